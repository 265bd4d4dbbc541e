"""Shard-task scheduler (Sec. IV): the library's decision, simulation and
estimation against scenarios worked by hand, against the plain restatement in
oracle/sched.py on random scenarios, and against the policy invariants
(availability, time fit, reallocation, cost formula).  Host code: no GPU."""
import math

import numpy as np
import pytest

from oracle import sched as osched
from paper_2605_10135_gb300 import ann, build

INF = math.inf


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()


def test_time_based_decision_by_hand():
    # Sec. IV: an instance that leaves in 10 minutes takes the 8-minute task, not
    # the 15-minute one; an instance with no announced end takes the longest task.
    got = ann.sched_decide(0.0, [0, 1], [15.0, 8.0], [0, 1], [10.0, INF])
    assert got.tolist() == [1, 0]
    # if no pending task fits it, the instance about to leave gets nothing
    got = ann.sched_decide(0.0, [0, 1], [15.0, 12.0], [0, 1], [10.0, INF])
    assert got.tolist() == [-1, 0]
    # availability only: longest task to the smallest idle instance id
    got = ann.sched_decide(0.0, [0, 1], [15.0, 12.0], [3, 1], [10.0, INF], ann.SCHED_AVAIL)
    assert got.tolist() == [1, 0]
    # the least remaining time that fits wins (best fit), ties to the smaller id
    got = ann.sched_decide(5.0, [7], [4.0], [2, 0, 1], [20.0, 9.0, 9.0])
    assert got.tolist() == [-1, 7, -1]


def test_simulation_by_hand():
    """Instances 0 (never leaves), 1 (leaves at 10, announced), 2 (joins at 5);
    tasks of 12, 8, 3 and 6 seconds.
      t=0  : 12 -> instance 0 (1 leaves too soon), 8 -> instance 1
      t=5  : instance 2 joins: 6 -> instance 2
      t=8  : instance 1 is free but leaves at 10: the 3-second task does not fit
      t=11 : 3 -> instance 2;  t=12, 14: the last two finish."""
    r = ann.sched_simulate([12, 8, 3, 6], [0, 0, 5], [INF, 10, INF], [0, 1, 0],
                           cpu_price=2.0, gpu_price=3.0)
    assert r["task_inst"].tolist() == [0, 1, 2, 2]
    assert r["task_start"].tolist() == [0.0, 0.0, 11.0, 5.0]
    assert r["task_end"].tolist() == [12.0, 8.0, 14.0, 11.0]
    s = r["summary"]
    assert s["makespan"] == 14.0 and s["gpu_active"] == 29.0 and s["lost"] == 0.0
    assert s["cost"] == 14.0 * 2.0 + 29.0 * 3.0


def test_unannounced_departure_reallocates():
    """Instance 0 leaves at 5 without notice while running the 10-second task: the
    run is lost (5 s) and the task restarts at 5 on instance 1 (free since 4)."""
    r = ann.sched_simulate([10, 4], [0, 0], [5, INF], [0, 0])
    assert r["tries"].tolist() == [2, 1]
    assert r["task_inst"].tolist() == [1, 1]
    assert r["task_end"].tolist() == [15.0, 4.0]
    s = r["summary"]
    assert s["reallocations"] == 1.0 and s["lost"] == 5.0 and s["gpu_active"] == 19.0
    # announced: the time-based policy never starts the long task there
    r = ann.sched_simulate([10, 4], [0, 0], [5, INF], [1, 0])
    assert r["tries"].tolist() == [1, 1] and r["summary"]["lost"] == 0.0
    assert r["task_inst"].tolist() == [1, 0]


def test_unfinished_when_nothing_fits():
    r = ann.sched_simulate([10], [0], [5], [1])
    assert r["summary"]["unfinished"] == 1.0 and r["task_inst"].tolist() == [-1]


@pytest.mark.parametrize("seed", range(30))
def test_matches_plain_restatement(seed):
    rng = np.random.default_rng(700 + seed)
    n, m = int(rng.integers(1, 25)), int(rng.integers(1, 6))
    est = rng.integers(1, 20, n).astype(float)
    actual = est * rng.choice([1.0, 0.5, 1.5, 2.0], n) if seed % 2 else None
    start = np.where(rng.random(m) < 0.3, rng.integers(0, 30, m), 0).astype(float)
    end = np.where(rng.random(m) < 0.5, start + rng.integers(0, 60, m), INF)
    end[0] = INF  # one instance stays, so every task can finish
    notice = (rng.random(m) < 0.5).astype(np.int32)
    policy = int(seed % 3 != 0)
    r = ann.sched_simulate(est, start, end, notice, actual, policy, 1.5, 4.0)
    ti, ts, te, tr, sm = osched.simulate(est.tolist(), None if actual is None else actual.tolist(),
                                         start.tolist(), end.tolist(), notice.tolist(), policy,
                                         1.5, 4.0)
    assert r["task_inst"].tolist() == ti
    assert r["tries"].tolist() == tr
    assert np.allclose(r["task_start"], ts) and np.allclose(r["task_end"], te)
    assert np.allclose(list(r["summary"].values()), sm)
    # invariants: every task done once; no instance runs two tasks at once
    assert all(i >= 0 for i in ti)
    runs = sorted((int(r["task_inst"][t]), r["task_end"][t] - (actual if actual is not None else est)[t],
                   r["task_end"][t]) for t in range(n))
    for (i1, _, e1), (i2, b2, _) in zip(runs, runs[1:]):
        if i1 == i2:
            assert b2 >= e1 - 1e-9
    if policy:  # time-based: a completed run on an announced instance fits before its end
        for t in range(n):
            j = int(r["task_inst"][t])
            if notice[j]:
                assert r["task_end"][t] <= end[j] + 1e-9


def test_decision_matches_restatement():
    rng = np.random.default_rng(800)
    for _ in range(200):
        n, m = int(rng.integers(0, 12)), int(rng.integers(0, 6))
        pid = rng.permutation(50)[:n]
        pes = rng.integers(1, 10, n).astype(float)
        iid = rng.permutation(20)[:m]
        ien = np.where(rng.random(m) < 0.5, rng.integers(1, 12, m).astype(float), INF)
        now = float(rng.integers(0, 3))
        pol = int(rng.integers(0, 2))
        got = ann.sched_decide(now, pid, pes, iid, ien, pol)
        ref = osched.decide(now, list(zip(pid.tolist(), pes.tolist())),
                            list(zip(iid.tolist(), ien.tolist())), pol)
        assert {int(i): int(t) for i, t in zip(iid, got) if t >= 0} == ref


def test_estimate_linear_and_quadratic():
    # exact data is reproduced exactly by the least-squares fit (Sec. IV: build time
    # linear in the shard size; the exact kNN graph: quadratic)
    s = np.array([1e3, 2e3, 5e3, 1e4])
    got = ann.sched_estimate(s, 0.5 + 2e-3 * s, [3e4, 1e5], model=0)
    assert np.allclose(got, 0.5 + 2e-3 * np.array([3e4, 1e5]))
    got = ann.sched_estimate(s, 0.1 + 1e-8 * s ** 2, [1e5], model=1)
    assert np.allclose(got, [0.1 + 1e-8 * 1e10])
    assert np.allclose(ann.sched_estimate(s, 3 * s + 1, [7.0]),
                       osched.estimate(s.tolist(), (3 * s + 1).tolist(), 0, [7.0]))
    with pytest.raises(ann.AnnError):
        ann.sched_estimate([5.0, 5.0], [1.0, 2.0], [1.0])


def test_restatement_pinned_by_hand():
    """The plain restatement itself on the hand-worked scenarios above."""
    ti, ts, te, tr, sm = osched.simulate([12, 8, 3, 6], None, [0, 0, 5], [INF, 10, INF],
                                         [0, 1, 0], 1, 2.0, 3.0)
    assert ti == [0, 1, 2, 2] and ts == [0.0, 0.0, 11.0, 5.0] and te == [12.0, 8.0, 14.0, 11.0]
    assert sm[0] == 14.0 and sm[1] == 29.0 and sm[5] == 14.0 * 2.0 + 29.0 * 3.0
    ti, ts, te, tr, sm = osched.simulate([10, 4], None, [0, 0], [5, INF], [0, 0], 1)
    assert tr == [2, 1] and te == [15.0, 4.0] and sm[2] == 5.0 and sm[3] == 1.0
    assert osched.decide(0.0, [(0, 15.0), (1, 8.0)], [(0, 10.0), (1, INF)], 1) == {0: 1, 1: 0}
    assert osched.decide(0.0, [(0, 15.0), (1, 12.0)], [(0, 10.0), (1, INF)], 1) == {1: 0}
    assert osched.estimate([1, 2, 3], [3, 5, 7], 0, [10]) == [21.0]
