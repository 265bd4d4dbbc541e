"""Shard tasks over worker processes that may leave (Sec. IV "Cloud Instance Task
Scheduler"), run live over a torch.distributed TCPStore.

The coordinator keeps the task list and the instance list (alive, busy or
idle, announced end time) and takes every decision with the library's
ann_sched_decide (availability- and time-based scheduling).  A worker reports
its end time when it knows it, beats a heartbeat, runs the tasks it is given
and reports each completion.  A worker whose heartbeat stops, or whose
announced end has passed, is taken off the list; the task it was running goes
back to the pending list and is given to another worker (reallocation).

Keys: alive/<rank> (heartbeat time), end/<rank> (announced end time),
task/<rank>/<n> (the n-th task id given to the rank, or "stop"),
done/<rank>/<n> (the rank finished its n-th task).
"""
from __future__ import annotations

import math
import threading
import time

from . import ann


def worker(store, rank: int, run_task, end_time: float | None = None,
           heartbeat_s: float = 0.05) -> int:
    """Serve tasks until told to stop; returns the number of tasks run."""
    if end_time is not None:
        store.set(f"end/{rank}", repr(float(end_time)))
    stop = threading.Event()

    def beat():
        while not stop.is_set():
            store.set(f"alive/{rank}", repr(time.time()))
            time.sleep(heartbeat_s)

    th = threading.Thread(target=beat, daemon=True)
    store.set(f"alive/{rank}", repr(time.time()))
    th.start()
    n = 0
    try:
        while True:
            key = f"task/{rank}/{n}"
            store.wait([key])
            msg = store.get(key).decode()
            if msg == "stop":
                break
            run_task(int(msg))
            store.set(f"done/{rank}/{n}", msg)
            n += 1
    finally:
        stop.set()
    return n


def coordinator(store, workers, est, policy: int = ann.SCHED_TIME, timeout_s: float = 1.0,
                poll_s: float = 0.01, max_s: float = 120.0, join_s: float = 10.0):
    """Give the tasks (estimated seconds est[t]) to the workers until all are done.

    Returns (done: task -> rank that completed it, log: list of (event, task, rank,
    time since start)) with events "start", "done", "lost".  Raises RuntimeError if
    every worker left with tasks pending, TimeoutError after max_s."""
    t0 = time.time()
    deadline = t0 + join_s
    for r in workers:  # every worker has beaten once
        while not store.check([f"alive/{r}"]):
            if time.time() > deadline:
                raise TimeoutError(f"worker {r} never joined")
            time.sleep(poll_s)
    pending = set(range(len(est)))
    running: dict[int, tuple[int, int]] = {}
    seq = {r: 0 for r in workers}
    alive = set(workers)
    done: dict[int, int] = {}
    log = []

    def end_of(r):
        return float(store.get(f"end/{r}")) if store.check([f"end/{r}"]) else math.inf

    while pending or running:
        now = time.time()
        for r, (n, t) in list(running.items()):
            if store.check([f"done/{r}/{n}"]):
                done[t] = r
                del running[r]
                seq[r] = n + 1
                log.append(("done", t, r, now - t0))
        for r in sorted(alive):
            hb = float(store.get(f"alive/{r}"))
            if now - hb > timeout_s or now >= end_of(r):
                alive.discard(r)
                if r in running:
                    n, t = running.pop(r)
                    pending.add(t)
                    log.append(("lost", t, r, now - t0))
        if not alive:
            raise RuntimeError(f"no worker left; tasks pending: {sorted(pending)}")
        idle = [r for r in sorted(alive) if r not in running]
        if pending and idle:
            ids = sorted(pending)
            pick = ann.sched_decide(now, ids, [est[t] for t in ids], idle,
                                    [end_of(r) for r in idle], policy)
            for r, t in zip(idle, pick.tolist()):
                if t < 0:
                    continue
                pending.discard(t)
                running[r] = (seq[r], t)
                store.set(f"task/{r}/{seq[r]}", str(t))
                log.append(("start", t, r, now - t0))
        if time.time() - t0 > max_s:
            raise TimeoutError("tasks not done in time")
        time.sleep(poll_s)
    for r in sorted(alive):
        store.set(f"task/{r}/{seq[r]}", "stop")
    return done, log
