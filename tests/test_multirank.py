"""The N > 1 bench path on CPU: two gloo ranks in separate processes.

Every rank builds its own replica of the workload (no data-path collective);
the only exchange is the maximum of the per-rank step times, after which rank 0
reports the whole-job rate.  These tests run that exchange and the reference
arm's rank handling with world_size 2 on the host.
"""
import json
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # rank r timed [step ms, e2e ms] = [10 + r, 30 - r]
    got = bench.max_over_ranks([10.0 + rank, 30.0 - rank])
    rate = bench.whole_job_rate(1000, world, got[0])
    dist.barrier()
    dist.destroy_process_group()
    with open(os.path.join(out_dir, f"r{rank}.json"), "w") as f:
        json.dump({"max": got, "rate": rate}, f)


def test_max_over_ranks_two_gloo_ranks(tmp_path):
    port = _free_port()
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True,
                       start_method="spawn")
    for r in range(2):
        with open(tmp_path / f"r{r}.json") as f:
            j = json.load(f)
        assert j["max"] == [11.0, 30.0]          # slowest rank's time on every rank
        assert j["rate"] == pytest.approx(2 * 1000 / 11e-3)


def test_max_over_ranks_without_group_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks([1.5, 2.5]) == [1.5, 2.5]
    assert bench.whole_job_rate(10, 1, 1000.0) == pytest.approx(10.0)


def test_reference_arm_other_ranks_print_nothing(capsys):
    sys.path.insert(0, ROOT)
    import bench
    from paper_2605_10135_gb300 import configs

    class A:
        warmup = 3
        steps = 1

    assert bench.run_reference(A(), configs.GAUSS_10K, 2, 1) is None
    assert capsys.readouterr().out == ""


def test_reference_arm_line_has_the_contract_keys(capsys):
    """--impl reference on rank 0: one JSON line with the metric, the oracle as the
    CPU baseline and an e2e block without host-device bytes."""
    sys.path.insert(0, ROOT)
    import bench
    from paper_2605_10135_gb300 import configs

    class A:
        warmup = 3
        steps = 1
        precision = "exact"
        epsilon = None

    bench.run_reference(A(), configs.GAUSS_10K, 1, 0)
    lines = [ln for ln in capsys.readouterr().out.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    j = json.loads(lines[0])
    assert j["impl"] == "reference" and j["metric"] == bench.METRIC
    assert j["unit"] == "vectors/s" and j["higher_is_better"] is True and j["value"] > 0
    assert j["cpu_baseline"]["kind"] == "oracle" and j["cpu_baseline"]["cores"] >= 1
    assert j["cpu_baseline"]["value"] == j["value"]
    assert j["e2e"]["h2d_bytes_per_step"] == 0 and j["e2e"]["d2h_bytes_per_step"] == 0
    assert j["config"]["workload"] == configs.GAUSS_10K.name
    # the same workload description the GPU arm prints
    assert j["config"] == bench.workload_config(configs.GAUSS_10K, A())
    assert j["warmup"] == 3 and j["extrapolated"] is True and j["wall_ms_per_step"] > 0
