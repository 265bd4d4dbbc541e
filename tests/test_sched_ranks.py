"""The live scheduler over worker processes (Sec. IV): a coordinator and two
workers meet at a TCPStore on 127.0.0.1; failures are made on the host (a
worker process that exits in the middle of a task, a worker that announces its
end).  No GPU: a task is a sleep of its estimated length."""
import json
import os
import socket
import sys
import time

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


EST = [0.6, 0.5, 0.4, 0.3, 0.2, 0.2]


def _main(rank, world, port, out_dir, scenario):
    sys.path.insert(0, ROOT)
    from datetime import timedelta

    import torch.distributed as dist
    from paper_2605_10135_gb300 import sched

    store = dist.TCPStore("127.0.0.1", port, world, rank == 0, timeout=timedelta(seconds=60))
    if rank == 0:
        try:
            done, log = sched.coordinator(store, list(range(1, world)), EST, timeout_s=2.0,
                                          join_s=120.0)
            res = {"done": {str(k): v for k, v in done.items()}, "log": log}
        except Exception as e:  # reported to the test instead of a silent hang
            res = {"error": repr(e)}
        with open(os.path.join(out_dir, "coord.json"), "w") as f:
            json.dump(res, f)
        time.sleep(0.3)  # let the workers read their stop message
        return

    def run(t):
        if scenario == "crash" and rank == 2:
            time.sleep(EST[t] / 2)
            os._exit(3)  # the process dies in the middle of its first task
        time.sleep(EST[t])

    end = time.time() + 0.45 if (scenario == "notice" and rank == 2) else None
    try:
        sched.worker(store, rank, run, end_time=end)
    except Exception:
        pass  # a worker past its announced end gets no stop message


def _run(tmp_path, scenario):
    port = _free_port()
    ctx = mp.start_processes(_main, args=(3, port, str(tmp_path), scenario), nprocs=3,
                             join=False, start_method="spawn")
    deadline = time.time() + 180
    while not os.path.exists(tmp_path / "coord.json") and time.time() < deadline:
        time.sleep(0.1)
    for p in ctx.processes:
        p.join(timeout=5)
        if p.is_alive():
            p.kill()
    with open(tmp_path / "coord.json") as f:
        out = json.load(f)
    assert "error" not in out, out["error"]
    return out


def test_crashed_worker_task_is_reallocated(tmp_path):
    out = _run(tmp_path, "crash")
    done = {int(k): v for k, v in out["done"].items()}
    assert sorted(done) == list(range(len(EST)))
    assert set(done.values()) == {1}        # worker 2 died: worker 1 did everything
    lost = [e for e in out["log"] if e[0] == "lost"]
    assert len(lost) == 1 and lost[0][2] == 2
    t = lost[0][1]
    starts = [e for e in out["log"] if e[0] == "start" and e[1] == t]
    assert [s[2] for s in starts] == [2, 1]  # first on the crashed worker, then on worker 1


def test_announced_end_gets_only_fitting_tasks(tmp_path):
    out = _run(tmp_path, "notice")
    done = {int(k): v for k, v in out["done"].items()}
    assert sorted(done) == list(range(len(EST)))
    assert not [e for e in out["log"] if e[0] == "lost"]  # nothing started that could not end
    for e in out["log"]:
        if e[0] == "start" and e[2] == 2:
            assert EST[e[1]] <= 0.45
