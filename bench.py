"""Benchmark of one divide-and-merge index build on GB300.

A step is one pass of the whole build on the 10M-vector Deep-like workload
(N=1e7, d=96 float32, unit norm, 64 shards, r=2, k=64, R=32; --workload picks
another): k-means partition with replication -> exact per-shard kNN (tcgen05
distance tiles + fused top-k, FP32 re-rank) -> rank-detour prune ->
dedup-then-reprune merge, inputs resident in HBM.  The
build is captured once as a CUDA graph and every step replays it (all kernels
run again); --eager launches every kernel from the host instead.

Prints one JSON line (rank 0).  value = vectors indexed per second over all
ranks; e2e = the same with the vectors copied from pinned host memory and the
merged graph copied back inside every step; roofline = the distance-tile
kernel's algorithmic FLOP/s (sum over shards of n_s^2 * 2d per launch) against
the measured dense BF16 peak; cpu_baseline = the plain oracle on a bounded
sample, extrapolated.  --impl reference times the oracle alone.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

# Workspaces of the large builds are tens of GB; a cached block that large must not
# be split to serve the smaller buffers of the next step, or the next step's
# workspace no longer fits.  Set before the first CUDA allocation.
if "PYTORCH_CUDA_ALLOC_CONF" not in os.environ:
    os.environ.setdefault("PYTORCH_ALLOC_CONF", "max_split_size_mb:4096")

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "index-build vectors/s at recall@10>=0.95; distance TFLOP/s as % of GB300 peak"


def _kernel_source_sha256():
    """Hash of the distance-tile kernel's device code: knn.cu up to the host-side
    tables (the kernel and its device helpers) and the shared device helpers, with
    // comments and blank lines left out."""
    import hashlib
    import re

    def code(text):
        lines = (re.sub(r"//.*", "", ln).rstrip() for ln in text.splitlines())
        return "\n".join(ln for ln in lines if ln)

    with open(os.path.join(ROOT, "paper_2605_10135_gb300/csrc/knn.cu")) as f:
        src = f.read()
    cut = src.index("// ---- problem tables, gather and norms")
    h = hashlib.sha256(code(src[:cut]).encode())
    with open(os.path.join(ROOT, "paper_2605_10135_gb300/csrc/common.cuh")) as f:
        h.update(code(f.read()).encode())
    return h.hexdigest()


def _kernel_traffic(workload: str):
    """DRAM bytes per distance-tile launch from the committed ncu capture of this
    workload, or None when there is none or the kernel source has changed since
    the counters were taken."""
    p = os.path.join(ROOT, "profiles", f"k_knn_tiles_{workload}.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        j = json.load(f)
    if _kernel_source_sha256() != j.get("kernel_source_sha256"):
        return None
    return int(j["dram_bytes_read_per_launch"] + j["dram_bytes_write_per_launch"])


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            j = json.load(f)
        return j, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle samples while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.rows = []
        self.proc = None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", gpu_id], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4)
                          if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(self.rows)}


# ------------------------------------------------------------------ CPU oracle leg

class OracleLeg:
    """The plain oracle timed on a bounded sample of the workload, extrapolated to
    the whole build.

    Set-up (untimed): the oracle's own partition of all N vectors, which the kNN
    of sampled shard rows needs.  One step (timed): k-means (10 iterations on the
    whole k-means sample), the replicated assignment of `assign_rows` vectors
    spread evenly over X (scaled by N), the exact kNN of `budget_rows` shard rows
    spread evenly over all rows (scaled by rows), and prune + merge of a
    6000-vector graph of the same degrees (scaled by N)."""

    def __init__(self, w, X, assign_rows=200_000):
        import oracle

        self.o, self.w, self.X = oracle, w, X
        sample, init_rows = w.kmeans_inputs()
        self.sample = sample
        self.init = X[init_rows].astype(np.float32)
        self.arows = np.linspace(0, w.N - 1, min(assign_rows, w.N)).astype(np.int64)
        Xs = X[:6000]
        if w.uneven is None:
            self.cent, _ = oracle.kmeans(X, self.init, sample, 10)
            self.members, self.offsets = oracle.shards(oracle.assign(X, self.cent, w.r), w.C)
            self.small = (Xs, *oracle.shards(oracle.assign(Xs, self.cent, w.r), w.C))
        else:  # the partition is an input: no k-means, no assignment
            self.members, self.offsets = w.shards()
            from paper_2605_10135_gb300 import datagen
            self.small = (Xs, *datagen.uneven_shards(len(Xs), w.C, w.r, 20, 160, seed=w.seed))
        self.rows_total = int(self.offsets[-1])

    def step(self, budget_rows=1500):
        """Returns (vectors/s, threads, description, extrapolated seconds, wall seconds)."""
        o, w, X = self.o, self.w, self.X
        wall0 = time.perf_counter()
        t_kmeans = t_assign = 0.0
        if w.uneven is None:
            t0 = time.perf_counter()
            o.kmeans(X, self.init, self.sample, 10)
            t_kmeans = time.perf_counter() - t0
            Xa = X[self.arows]
            t0 = time.perf_counter()
            o.assign(Xa, self.cent, w.r)
            t_assign = (time.perf_counter() - t0) * (w.N / len(self.arows))
        rows = np.linspace(0, max(self.rows_total - 1, 0), budget_rows).astype(np.int64)
        t0 = time.perf_counter()
        o.shard_knn(X, self.members, self.offsets, w.k, rows=rows)
        t_knn = (time.perf_counter() - t0) / budget_rows * self.rows_total
        Xs, ms_, os_ = self.small
        kid, kd = o.shard_knn(Xs, ms_, os_, w.k)
        t0 = time.perf_counter()
        pid, pd = o.prune(kid, kd, ms_, os_, w.R)
        o.merge(pid, pd, ms_, os_, Xs.shape[0])
        t_pm = (time.perf_counter() - t0) * (w.N / Xs.shape[0])
        total = t_kmeans + t_assign + t_knn + t_pm
        part = (f"k-means (10 iterations on the {len(self.sample)}-row sample) in full; the "
                f"replicated assignment of {len(self.arows)} of the {w.N} vectors, scaled by N"
                if w.uneven is None else "the partition is given (synthetic uneven shards)")
        desc = (f"oracle: {part}; the exact kNN of {budget_rows} shard rows spread evenly over "
                f"all {self.rows_total} rows, scaled by rows; prune+merge of a 6000-vector "
                f"graph, scaled by N")
        return w.N / total, o.num_threads(), desc, total, time.perf_counter() - wall0


def workload_config(w, args):
    """The workload a line measures, identical in both arms' JSON lines."""
    return {"workload": w.name, "N": w.N, "d": w.d, "elem": w.dtype, "shards": w.C,
            "replicas": w.r, "k": w.k, "R": w.R,
            "partition": ("k-means, 10 iterations" if w.uneven is None else
                          "synthetic uneven shards, sizes log-uniform on [%d, %d] rescaled to "
                          "r N rows" % tuple(w.uneven)),
            "tile_launch": ("one per shard" if getattr(args, "per_shard", False) else
                            "one grouped launch over all shards (a CTA per row block, "
                            "largest shard first)"),
            "precision": args.precision, "epsilon": args.epsilon,
            "l2": "flushed (512 MB write) before every timed GPU step"}


# ------------------------------------------------------------------ multi-rank helpers

def max_over_ranks(values, device=None):
    """Element-wise maximum of per-rank values over all ranks of the default
    process group (the values themselves when no group is initialised)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return [float(v) for v in values]
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.tolist()


def whole_job_rate(units_per_rank, world, ms):
    """Units processed by all ranks per second, timed by the slowest rank (weak scaling:
    every rank builds its own replica of the workload)."""
    return world * units_per_rank / (ms * 1e-3)


def screening_error(X, row_vecs, ids, dist):
    """(max, mean) of |dist - d| / d over the listed (row, id) pairs with d > 0, d the
    squared distance in float64 (a measurement of the screening keys' error)."""
    rel = []
    for r in range(ids.shape[0]):
        ok = ids[r] != 0xFFFFFFFF
        if not ok.any():
            continue
        c = ids[r][ok].astype(np.int64)
        d = ((X[c].astype(np.float64) - X[int(row_vecs[r])].astype(np.float64)) ** 2).sum(1)
        pos = d > 0
        rel.append(np.abs(dist[r][ok][pos] - d[pos]) / d[pos])
    if not rel:
        return 0.0, 0.0
    a = np.concatenate(rel)
    return float(a.max()), float(a.mean())


def union_recall_at_10(ann, Xd, out, N, nq, seed):
    """Mean over nq sampled vectors of |10 nearest in the union of the vector's
    shard kNN lists  intersect  its exact 10 nearest over all N| / 10."""
    import torch
    rng = np.random.default_rng(seed)
    vs = np.sort(rng.choice(N, min(nq, N), replace=False))
    dev = out["graph"].device
    q = (Xd[torch.from_numpy(vs).to(Xd.device)] if Xd.is_cuda
         else Xd[torch.from_numpy(vs)]).to(dev)
    gt_id, _ = ann.knn_query(Xd, q, 11)
    gt = gt_id.cpu().numpy().view(np.uint32)
    members = out["members"].cpu().numpy().view(np.uint32)
    kid = out["knn_id"].cpu().numpy().view(np.uint32)
    kd = out["knn_d"].cpu().numpy()
    order = np.argsort(members, kind="stable")
    ms = members[order]
    lo, hi = np.searchsorted(ms, vs, "left"), np.searchsorted(ms, vs, "right")
    hit = 0
    for i, v in enumerate(vs):
        truth = [int(t) for t in gt[i] if int(t) != int(v)][:10]
        cand = {}
        for p in order[lo[i]:hi[i]]:
            for t, dd in zip(kid[p], kd[p]):
                t = int(t)
                if t != 0xFFFFFFFF and (t not in cand or dd < cand[t]):
                    cand[t] = float(dd)
        top = sorted(cand.items(), key=lambda e: (e[1], e[0]))[:10]
        hit += len({t for t, _ in top} & set(truth))
    return hit / (10.0 * len(vs))


# ------------------------------------------------------------------ main

def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="deep10m_d96_f32")
    ap.add_argument("--nq", type=int, default=1000)
    ap.add_argument("--no-baseline", action="store_true")
    ap.add_argument("--n", type=int, default=0, help="override N (smaller case for profiling)")
    ap.add_argument("--shards", type=int, default=0,
                    help="override the shard count C (with --n: a small case whose shards are "
                         "as large as the full workload's)")
    ap.add_argument("--precision", default="exact",
                    choices=["exact", "bf16", "f16", "fp8", "learned"],
                    help="distance-tile form: exact (uint8 / FP32 split), BF16 / scaled FP16 / "
                         "E4M3 screening with an FP32 re-rank of the top 128, or learned "
                         "(32-d MLP embedding screened, re-ranked exactly)")
    ap.add_argument("--rerank-k", type=int, default=0, help="screened list width (0: default)")
    ap.add_argument("--graph", action="store_true",
                    help="capture one whole build as a CUDA graph and time its replays (the "
                         "default where the build is capturable)")
    ap.add_argument("--eager", action="store_true",
                    help="time eager builds (every kernel launched from the host each step)")
    ap.add_argument("--autotune", action="store_true",
                    help="time the candidate tile plans during the first warm-up step")
    ap.add_argument("--learn-steps", type=int, default=300)
    ap.add_argument("--learn-batch", type=int, default=512)
    ap.add_argument("--sample-frac", type=float, default=0.01)
    ap.add_argument("--learn-lr", type=float, default=1e-3)
    ap.add_argument("--min-recall", type=float, default=0.9,
                    help="learned form: recall estimate below which the exact form is used")
    ap.add_argument("--epsilon", type=float, default=None,
                    help="selective replication (Sec. V) with this eps; default: every vector "
                         "in its r nearest shards")
    ap.add_argument("--tau0", type=float, default=2.0)
    ap.add_argument("--sel-block", type=int, default=65536, help="vectors per assignment block")
    ap.add_argument("--capacity", type=int, default=0, help="members per shard, 0 = no limit")
    ap.add_argument("--cand", type=int, default=8, help="candidate centroids per vector")
    ap.add_argument("--host-x", action="store_true",
                    help="leave the vectors in pinned host memory: the kernels read them over "
                         "the host link (NVLink-C2C) instead of from a device copy")
    ap.add_argument("--streamed", action="store_true",
                    help="build one shard at a time (kNN lists of one shard resident at a time)")
    ap.add_argument("--no-tile-prune", action="store_true",
                    help="sweep every distance tile (no exact skipping by the triangle "
                         "inequality)")
    ap.add_argument("--entries", type=int, default=1024,
                    help="search also from the nearest of this many sampled entry vectors")
    ap.add_argument("--per-shard", action="store_true",
                    help="one distance-tile launch per shard instead of one grouped launch "
                         "over all shards (same lists)")
    ap.add_argument("--tile-counters", action="store_true",
                    help="after timing, run one step with the counting kernel variant and "
                         "report its per-role cycle counters")
    args = ap.parse_args()

    from paper_2605_10135_gb300 import configs

    w = configs.BY_NAME[args.workload]
    if args.n or args.shards:
        import dataclasses
        n, c = args.n or w.N, args.shards or w.C
        w = dataclasses.replace(w, N=n, C=c, name=f"{w.name}@N={n},C={c}")
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        return run_reference(args, w, world, rank)

    import torch
    from paper_2605_10135_gb300 import ann

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if dist is not None:
            dist.barrier()

    X, Qn = w.vectors_and_queries(args.nq)
    sample, init_rows = w.kmeans_inputs()
    init = X[init_rows].astype(np.float32)
    Xh = torch.from_numpy(X).pin_memory()
    Xd = Xh if args.host_x else Xh.to(dev)
    init_d = torch.from_numpy(init).to(dev)
    samp_d = torch.from_numpy(sample.view(np.int32)).to(dev)
    shards = None  # synthetic uneven partition: (members, offsets, per-shard host offsets)
    if w.uneven is not None:
        mem_np, off_np = w.shards()
        shards = (torch.from_numpy(mem_np.view(np.int32)).to(dev), torch.from_numpy(off_np).to(dev),
                  off_np.tolist() if args.per_shard else None)
    prec = {"exact": ann.EXACT, "bf16": ann.BF16_RERANK, "f16": ann.F16_RERANK,
            "fp8": ann.FP8_RERANK, "learned": ann.LEARNED}[args.precision]
    sel = None
    if args.epsilon is not None:
        sel = ann.SelectiveConfig(epsilon=args.epsilon, tau0=args.tau0, block=args.sel_block,
                                  capacity=args.capacity, cand=args.cand)
    cfg = ann.BuildConfig(C=w.C, r=w.r, k=w.k, R=w.R, iters=10, precision=prec,
                          rerank_k=args.rerank_k, selective=sel)
    learned = None
    if prec == ann.LEARNED:
        from paper_2605_10135_gb300 import datagen
        ls = datagen.row_sample(w.N, args.sample_frac, 256, seed=w.seed + 11)
        learned = ann.LearnedInputs(
            sample=torch.from_numpy(ls.view(np.int32)).to(dev),
            draws=torch.from_numpy(datagen.triplet_draws(args.learn_steps, args.learn_batch,
                                                         seed=w.seed + 12).view(np.int32)).to(dev),
            params0=torch.from_numpy(datagen.mlp_init(w.d, seed=w.seed + 13)).to(dev),
            lr=args.learn_lr, min_recall=args.min_recall)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)  # > L2 (129 MB)

    captured = None

    def step(x):
        if captured is not None:
            if x.data_ptr() != captured.X.data_ptr():
                captured.X.copy_(x, non_blocking=True)
            return captured.replay()
        if shards is not None:
            return ann.build_from_shards(x, shards[0], shards[1], cfg, shards[2])
        if args.streamed:
            return ann.build_index_streamed(x, cfg, init_d, samp_d)
        return ann.build_index(x, cfg, init_d, samp_d, learned)

    ann.tile_prune(not args.no_tile_prune)
    if args.autotune:
        ann.autotune(1)
    for _ in range(max(args.warmup, 3)):
        out = step(Xd)
    torch.cuda.synchronize()
    ann.autotune(0)
    use_graph = args.graph or not args.eager
    if use_graph and (prec == ann.LEARNED or sel is not None or args.streamed):
        use_graph = False  # host decisions between stages: not capturable
    if use_graph:
        captured = ann.CapturedBuild(Xd, cfg, init_d, samp_d, shards)
        for _ in range(2):
            out = step(Xd)
        torch.cuda.synchronize()
    tuned = (ann.autotune_lookup(w.d, Xd.dtype, w.k, out.get("precision", prec), args.rerank_k,
                                 int(out["members"].numel()), w.C) if args.autotune else None)

    uuid = str(torch.cuda.get_device_properties(dev).uuid)
    clocks = ClockSampler(uuid if uuid.startswith("GPU-") else f"GPU-{uuid}")
    time.sleep(0.5)
    ann.timing_read()
    ann.tile_prune_stats()  # clears the tile counters (synchronises; outside the timed region)
    ann.timing_enable(True)
    l0 = ann.launch_count()
    st = torch.cuda.current_stream()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    barrier()
    torch.cuda.synchronize()
    for i in range(args.steps):
        flush.zero_()
        evs[i][0].record(st)
        out = step(Xd)
        evs[i][1].record(st)
    torch.cuda.synchronize()
    barrier()
    launches = (ann.launch_count() - l0) // args.steps
    if captured is not None:  # replays launch the captured kernels without host calls
        launches = captured.kernels
    ann.timing_enable(False)
    tile_ms, tile_n = ann.timing_read()
    pst = ann.tile_prune_stats()
    pst = {key: v / args.steps for key, v in pst.items()}  # per step
    step_ms = [a.elapsed_time(b) for a, b in evs]
    ms = float(np.mean(step_ms))
    tile_source = "timed steps"
    tile_steps = args.steps

    # e2e: vectors from pinned host memory in, merged graph out, every step
    e2e_ms = []
    graph_h = torch.empty((w.N, w.R), dtype=torch.int32).pin_memory()
    gdist_h = torch.empty((w.N, w.R), dtype=torch.float32).pin_memory()
    deg_h = torch.empty(w.N, dtype=torch.int32).pin_memory()
    # half the timed steps (at least 3; 3 when a step takes over a second)
    n_e2e = 3 if ms > 1000.0 else max(3, args.steps // 2)
    for i in range(n_e2e):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        xd = Xh if args.host_x else Xh.to(dev, non_blocking=True)
        o = step(xd)
        graph_h.copy_(o["graph"], non_blocking=True)
        gdist_h.copy_(o["gdist"], non_blocking=True)
        deg_h.copy_(o["degree"], non_blocking=True)
        torch.cuda.synchronize()
        e2e_ms.append((time.perf_counter() - t0) * 1e3)
    clocks.stop()
    # the graph (and its workspace) is not replayed again: release it, so that the
    # eager steps below have the memory of one workspace, not two
    if captured is not None:
        out = {key: (v.clone() if isinstance(v, torch.Tensor) else v) for key, v in out.items()}
        captured = o = None
        import gc
        gc.collect()
        torch.cuda.empty_cache()
    if tile_n == 0:  # graph replays record no host-side kernel events: one eager step
        flush.zero_()
        ann.timing_enable(True)
        step(Xd)
        torch.cuda.synchronize()
        ann.timing_enable(False)
        tile_ms, tile_n = ann.timing_read()
        tile_source = "one eager step after the timed graph replays"
        tile_steps = 1

    # quality: the exact form gives the exact graph by construction; a screening form
    # is scored against the exact form's lists on the same partition
    graph_recall = 1.0
    if out.get("precision", prec) != ann.EXACT and "knn_id" in out:
        ex_id, _ = ann.shard_knn(Xd, out["members"], out["offsets"], w.k, ann.EXACT)
        graph_recall = float(ann.recall(out["knn_id"], ex_id, 10).item())
        del ex_id
    union_recall = (union_recall_at_10(ann, Xd, out, w.N, args.nq, w.seed + 21)
                    if "knn_id" in out else None)  # the streamed build keeps no kNN lists
    # search recall@10 from the medoid
    Q = torch.from_numpy(Qn).to(dev)
    gt, _ = ann.knn_query(Xd, Q, 10)
    entry = int(ann.medoid(Xd).item())
    ids, cnt = ann.search(out["graph"], out["degree"], Xd, Q, entry, 64, 10)
    recall = float(ann.recall(ids, gt, 10).item())
    ent = torch.from_numpy(np.sort(np.random.default_rng(w.seed + 22).choice(
        w.N, min(args.entries, w.N), replace=False)).astype(np.int32)).to(dev)
    ids_e, cnt_e = ann.search_entries(out["graph"], out["degree"], Xd, Q, ent, 64, 10)
    recall_e = float(ann.recall(ids_e, gt, 10).item())
    # the merged graph with reverse edges (an alternative merge, not timed in the
    # step): its own time, and search recall from the medoid and from the entries
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    rg, _, rdeg = ann.merge_reverse(out["graph"], out["gdist"], out["degree"])
    ev1.record()
    torch.cuda.synchronize()
    ids_r, cnt_r = ann.search(rg, rdeg, Xd, Q, entry, 64, 10)
    ids_re, _ = ann.search_entries(rg, rdeg, Xd, Q, ent, 64, 10)
    reverse = {"merge_ms": ev0.elapsed_time(ev1),
               "search_recall_at_10": float(ann.recall(ids_r, gt, 10).item()),
               "mean_dist_count": float(cnt_r.float().mean().item()),
               "search_recall_at_10_from_entries": float(ann.recall(ids_re, gt, 10).item()),
               "mean_degree": float(rdeg.float().mean().item())}
    del rg, rdeg, ids_r, ids_re
    # screening error of float forms (the screened lists before the exact re-rank)
    # against the FP64 distances, on 2000 sampled rows
    screening = None
    if w.dtype != "u8" and prec != ann.LEARNED and shards is None:
        cid, cd = ann.shard_knn_screen(Xd, out["members"], out["offsets"], w.k, prec,
                                       args.rerank_k)
        rows_s = torch.from_numpy(np.linspace(0, cid.shape[0] - 1, 2000).astype(np.int64)).to(dev)
        sid = cid.index_select(0, rows_s).cpu().numpy().view(np.uint32)
        sdd = cd.index_select(0, rows_s).cpu().numpy().astype(np.float64)
        mem_h = out["members"].index_select(0, rows_s).cpu().numpy().view(np.uint32)
        mx, mean = screening_error(X, mem_h, sid, sdd)
        screening = {"rows_sampled": 2000, "list_width": int(cid.shape[1]),
                     "max_rel_error": mx, "mean_rel_error": mean,
                     "definition": "|screening distance - d64| / d64 over every listed "
                                   "(row, id) with d64 > 0, before the FP32 re-rank"}
        del cid, cd
    status = ann.device_status()

    # one more step with events between the stages (not timed above)
    torch.cuda.synchronize()
    sev = [torch.cuda.Event(enable_timing=True) for _ in range(6)]
    sev[0].record(st)
    if shards is not None:
        mem_s, off_s = shards[0], shards[1]
    elif sel is None:
        cent_s, mem_s, off_s = ann.partition(Xd, cfg.C, cfg.r, init_d, samp_d, cfg.iters)
    else:
        cent_s, mem_s, off_s, _, _ = ann.partition_selective(Xd, cfg.C, cfg.r, init_d, samp_d,
                                                             cfg.iters, sel)
    sev[1].record(st)
    prec_s, model_s = cfg.precision, None
    if prec_s == ann.LEARNED:
        model_s = learned.params0.clone()
        _, est_s = ann.learned_train(Xd, learned.sample, learned.draws, model_s, learned.kk,
                                     learned.kpos, learned.lr, learned.margin)
        if float(est_s.item()) < learned.min_recall:
            prec_s, model_s = ann.EXACT, None
    sev[2].record(st)
    if shards is not None and shards[2] is not None:
        kid_s, kd_s = ann.shard_knn_per_shard(Xd, mem_s, shards[2], cfg.k, prec_s, cfg.rerank_k)
    else:
        kid_s, kd_s = ann.shard_knn(Xd, mem_s, off_s, cfg.k, prec_s, cfg.rerank_k, model_s)
    sev[3].record(st)
    pid_s, pd_s = ann.prune(kid_s, kd_s, mem_s, off_s, cfg.R, cfg.rule, N=w.N)
    sev[4].record(st)
    ann.merge(pid_s, pd_s, mem_s, off_s, w.N)
    sev[5].record(st)
    torch.cuda.synchronize()
    stages_ms = {name: sev[i].elapsed_time(sev[i + 1]) for i, name in
                 enumerate(["partition", "learn", "shard_knn", "prune", "merge"])}
    if model_s is not None:  # the embedding alone (part of the learned shard_knn)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        ann.learned_embed(Xd, model_s)
        e1.record(st)
        torch.cuda.synchronize()
        stages_ms["of_which_embed"] = e0.elapsed_time(e1)
    del kid_s, kd_s, pid_s, pd_s

    counters = None
    if args.tile_counters:
        ann.tile_counters_read()
        ann.tile_counters_enable(True)
        step(Xd)  # eager (the graph is released above)
        counters = ann.tile_counters_read()
        ann.tile_counters_enable(False)

    ms, e2e_mean = max_over_ranks([ms, float(np.mean(e2e_ms))], dev)

    off = out["offsets"].cpu().numpy()
    sizes = np.diff(off).astype(np.float64)
    d_tile = 32 if out.get("precision") == ann.LEARNED else w.d
    pairs_all = float(np.sum(sizes ** 2))
    # exact tile skipping: the sweep computes only the pairs of the tiles it keeps
    pairs = pst["pairs"] if pst["tiles"] > 0 else pairs_all
    flops = float(pairs * 2 * d_tile)
    # per step: one launch over all shards (or one per shard when streamed)
    tile_avg_ms = tile_ms / max(tile_steps, 1)
    tile_launches_per_step = tile_n / max(tile_steps, 1)
    achieved = flops / (tile_avg_ms * 1e-3) / 1e12
    peaks, src = _peaks()
    peak = float(peaks.get("bf16_tflops_sustained", peaks["bf16_tflops"]))
    peak_note = f"{src} bf16_tflops_sustained"
    if prec == ann.FP8_RERANK:
        peak *= 2.0  # nominal dense E4M3 / BF16 ratio (4.5 / 2.25 PFLOP/s)
        peak_note += " x 2 (nominal fp8/bf16 ratio)"
    if w.dtype == "u8" and prec not in (ann.FP8_RERANK, ann.LEARNED):
        dtype, operands, products = "u8", "bf16 (exact for uint8), fp32 accumulate", 1
    elif prec == ann.EXACT:
        dtype = "f32"
        operands = "bf16 hi/lo split, three products, fp32 accumulate; fp32 re-rank of k+16"
        products = 3
    elif prec == ann.BF16_RERANK:
        dtype, operands, products = "bf16", "bf16, fp32 accumulate; fp32 re-rank of top 128", 1
    elif prec == ann.F16_RERANK:
        dtype, operands, products = ("f16", "fp16 (power-of-two global scale), fp32 accumulate; "
                                     "fp32 re-rank of top 128", 1)
    elif prec == ann.FP8_RERANK:
        dtype, operands, products = "fp8", "e4m3 (one global scale), fp32 accumulate; fp32 re-rank of top 128", 1
    else:
        dtype, operands, products = ("learned32-f16", "32-d MLP embedding (fp32 GEMMs) screened "
                                     "with scaled fp16, fp32 accumulate; fp32 re-rank in the "
                                     "original space", 1)
    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return
    line = {
        "metric": METRIC,
        "value": whole_job_rate(w.N, world, ms),
        "unit": "vectors/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": max(args.warmup, 3),
        "ms_per_step": ms,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": dtype,
        "data": "synthetic",
        "config": workload_config(w, args),
        "quality": {
            "recall_at_10": graph_recall,
            "recall_definition": ("graph recall@10 vs the exact kNN graph (exact build: 1.0 by "
                                  "construction, checked against the oracle in the parity tests)"
                                  if prec == ann.EXACT else
                                  "graph recall@10 of the shard kNN lists vs the exact form's "
                                  "lists on the same partition"),
            "union_recall_at_10": union_recall,
            "union_recall_definition": ("for nq sampled vectors: the 10 nearest of the union of "
                                        "the vector's shard kNN lists vs its exact 10 nearest "
                                        "over all N (partition locality)"),
            "search_recall_at_10": recall, "search_Ls": 64, "queries": args.nq,
            "mean_dist_count": float(cnt.float().mean().item()),
            "search_recall_at_10_from_entries": recall_e, "search_entries": int(ent.numel()),
            "mean_dist_count_from_entries": float(cnt_e.float().mean().item()),
            "reverse_edges": reverse,
            "reverse_edges_definition": ("the merged graph with reverse edges (ann_merge_reverse, "
                                         "an alternative merge timed on its own) searched the "
                                         "same way"),
        },
        "detail": {
            "learned": (None if prec != ann.LEARNED else {
                "steps": args.learn_steps, "batch": args.learn_batch,
                "sample_rows": int(learned.sample.numel()),
                "recall_estimate": out.get("recall_estimate"),
                "fell_back_to_exact": out.get("precision") != ann.LEARNED,
                "timed_step_includes_training": True}),
            "tile_operands": operands, "tensor_products_per_pair": products,
            "screening_error": screening,
            "selective": (None if sel is None else {
                "epsilon": sel.epsilon, "tau0": sel.tau0, "block": sel.block,
                "capacity": sel.capacity, "cand": sel.cand,
                "replicated_share": float(out["selective_stats"][0].item()) / w.N,
                "overflowed_originals": int(out["selective_stats"][1].item()),
                "member_rows": int(out["offsets"][-1].item())}),
            "shard_sizes_min_max": [int(sizes.min()), int(sizes.max())],
            "distance_tflops": achieved,
            "tile_skipping": ({"pairs_all": pairs_all, "pairs_swept": pairs,
                               "tiles_swept_fraction": pst["swept"] / max(pst["tiles"], 1),
                               "all_pairs_rate_tflops": pairs_all * 2 * d_tile /
                               (tile_avg_ms * 1e-3) / 1e12}
                              if pst["tiles"] > 0 else None),
            "stages_ms": stages_ms,
            "tile_plan_autotuned": tuned,
            "cuda_graph": bool(use_graph),
            "vectors_in": ("pinned host memory, read by the kernels over NVLink-C2C"
                           if args.host_x else "device memory"),
            "streamed_shards": bool(args.streamed),
            "device_status": status,
        },
        "roofline": {
            "kernel": "k_knn_tiles", "bound": "tensor", "achieved": achieved, "peak": peak,
            "unit": "TFLOP/s", "frac": achieved / peak,
            "traffic": _kernel_traffic(w.name) if prec == ann.EXACT else None,
            "peak_source": peak_note,
            "algorithmic_flops_per_step": flops,
            "algorithmic_flops_per_launch": flops / max(tile_launches_per_step, 1.0),
            "kernel_ms": tile_avg_ms,
            "kernel_ms_source": tile_source, "kernel_launches_per_step": tile_launches_per_step,
        },
        "e2e": {
            "value": whole_job_rate(w.N, world, e2e_mean), "unit": "vectors/s",
            "h2d_bytes_per_step": int(X.nbytes),
            "d2h_bytes_per_step": int(graph_h.numel() * 4 + gdist_h.numel() * 4 + deg_h.numel() * 4),
            "ms_per_step": e2e_mean,
        },
        "gpu_launches": int(launches) * args.steps,
        "clocks": clocks.summary(),
    }
    if counters is not None:
        line["tile_counters"] = counters
    if world == 1 and not args.no_baseline:
        v, cores, desc, _, _ = OracleLeg(w, X).step(budget_rows=1500)
        line["cpu_baseline"] = {"value": v, "unit": "vectors/s", "cores": cores, "kind": "oracle",
                                "sample": desc}
    print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()


def run_reference(args, w, world, rank):
    """The oracle as it stands, on the host cores, a bounded sample per step."""
    if rank != 0:
        return
    X = w.vectors()
    leg = OracleLeg(w, X)
    warm = max(args.warmup, 3)
    for _ in range(warm):
        leg.step(budget_rows=400)
    vals, tms, walls = [], [], []
    desc, cores = "", 0
    for _ in range(args.steps):
        v, cores, desc, total, wall = leg.step(budget_rows=400)
        vals.append(v)
        tms.append(total * 1e3)
        walls.append(wall * 1e3)
    v = float(np.mean(vals))
    ms = float(np.mean(tms))
    dtype = {"u8": "u8", "f32": "f64", "f16": "f64"}[w.dtype]
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": "vectors/s", "n_gpus": world,
        "steps": args.steps, "warmup": warm, "ms_per_step": ms,
        "extrapolated": True, "wall_ms_per_step": float(np.mean(walls)),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": dtype,
        "data": "synthetic", "config": workload_config(w, args),
        "cpu_baseline": {"value": v, "unit": "vectors/s", "cores": cores, "kind": "oracle",
                         "sample": desc},
        "e2e": {"value": v, "unit": "vectors/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


if __name__ == "__main__":
    main()
