"""Plain restatement of the shard-task scheduler (TEST INFRASTRUCTURE ONLY).

Sec. IV "Cloud Instance Task Scheduler": availability-based scheduling (busy
instances take no task), time-based scheduling (an instance whose remaining
time is known takes only tasks whose estimated run time fits it; an instance
about to leave gets a task that fits or none), reallocation of the task of an
instance that leaves.  Sec. IV "Spot instance cost analysis": cost = CPU time x
CPU price + aggregated GPU active time x GPU price.  Readings taken where the
paper is silent (order of tasks, choice among instances, simultaneous events)
are the ones stated in the library's header; this file writes them out as
plain loops, independently of the library.
"""
from __future__ import annotations

import math

TIME = 1


def decide(now, pending, idle, policy):
    """pending: list of (task id, estimate); idle: list of (instance id, end or
    inf).  Returns {instance id: task id}."""
    given = {}
    used = set()
    for tid, e in sorted(pending, key=lambda p: (-p[1], p[0])):
        choice = None
        for iid, end in idle:
            if iid in used:
                continue
            if policy & TIME:
                rem = end - now
                if rem < e:
                    continue
                if choice is None or rem < choice[1] or (rem == choice[1] and iid < choice[0]):
                    choice = (iid, rem)
            else:
                if choice is None or iid < choice[0]:
                    choice = (iid, 0.0)
        if choice is not None:
            given[choice[0]] = tid
            used.add(choice[0])
    return given


def simulate(est, actual, start, end, notice, policy, cpu_price=0.0, gpu_price=0.0):
    """Discrete events; returns (task_inst, task_start, task_end, tries, summary)."""
    n, m = len(est), len(start)
    dur = actual if actual is not None else est
    state = ["pending"] * n
    inst_task = [None] * m          # (task, begin, finish) while running
    gone = [False] * m
    t_inst, t_start, t_end, tries = [-1] * n, [math.nan] * n, [math.nan] * n, [0] * n
    now, busy, lost, makespan, realloc = 0.0, 0.0, 0.0, 0.0, 0
    while True:
        for j in range(m):          # completions
            run = inst_task[j]
            if run is not None and run[2] <= now:
                tid, b, f = run
                state[tid] = "done"
                t_inst[tid], t_end[tid] = j, f
                busy += f - b
                makespan = max(makespan, f)
                inst_task[j] = None
        for j in range(m):          # departures
            if not gone[j] and end[j] <= now:
                gone[j] = True
                if inst_task[j] is not None:
                    tid, b, _ = inst_task[j]
                    state[tid] = "pending"
                    busy += now - b
                    lost += now - b
                    realloc += 1
                    inst_task[j] = None
        pending = [(i, est[i]) for i in range(n) if state[i] == "pending"]
        idle = [(j, end[j] if (notice is not None and notice[j]) else math.inf)
                for j in range(m) if not gone[j] and start[j] <= now and inst_task[j] is None]
        if pending and idle:
            for j, tid in decide(now, pending, idle, policy).items():
                state[tid] = "running"
                inst_task[j] = (tid, now, now + dur[tid])
                if tries[tid] == 0:
                    t_start[tid] = now
                tries[tid] += 1
        if all(s == "done" for s in state):
            break
        times = []
        for j in range(m):
            if gone[j]:
                continue
            if inst_task[j] is not None:
                times.append(inst_task[j][2])
            if start[j] > now:
                times.append(start[j])
            else:
                times.append(end[j])
        nxt = min(times) if times else math.inf
        if nxt == math.inf:
            break
        now = nxt
    unfinished = sum(s != "done" for s in state)
    summary = [makespan, busy, lost, float(realloc), float(unfinished),
               makespan * cpu_price + busy * gpu_price]
    return t_inst, t_start, t_end, tries, summary


def estimate(sizes, times, model, task_sizes):
    """Least squares t = a + b f(s), f(s) = s (model 0) or s^2 (model 1)."""
    f = [s * s if model else s for s in sizes]
    n = len(f)
    mx, my = sum(f) / n, sum(times) / n
    b = sum((x - mx) * (y - my) for x, y in zip(f, times)) / sum((x - mx) ** 2 for x in f)
    a = my - b * mx
    return [a + b * (s * s if model else s) for s in task_sizes]
