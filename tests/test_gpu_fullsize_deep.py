"""Parity at the benchmark's default full size: the Deep-like 10M build (N = 1e7
FP32, d = 96, 64 shards, r = 2, k = 64, R = 32, exact form) in the configuration
bench.py times, checked on outputs the oracle computes one by one: the whole
partition (bit for bit: decisions in FP32 on both sides), the kNN lists of sampled
rows (the float rule: every sure neighbour present, no id beyond the k-th distance,
distances within 1e-5 of FP64, sorted), the pruned lists of sampled rows (the
oracle's prune of the GPU's own lists of those rows and their neighbours: integer
logic, bit for bit) and the merged lists of sampled vectors (the oracle's merge of
the GPU's pruned lists of their rows, bit for bit).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2605_10135_gb300 import ann, build, configs
from tests.parity import as_u32, check_float_lists

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def T(a):
    a = np.ascontiguousarray(a)
    if a.dtype == np.uint32:
        a = a.view(np.int32)
    return torch.from_numpy(a).to(DEV)


@pytest.fixture(scope="module")
def run():
    build.build()
    ann.device_status()
    w = configs.DEEP_10M
    X = w.vectors()
    sample, init_rows = w.kmeans_inputs()
    init = X[init_rows].astype(np.float32)
    out = ann.build_index(T(X), ann.BuildConfig(C=w.C, r=w.r, k=w.k, R=w.R, iters=10), T(init),
                          T(sample))
    torch.cuda.synchronize()
    cent_o, _, mem_o, off_o = oracle.partition(X, init, sample, 10, w.C, w.r)
    yield w, X, out, cent_o, mem_o, off_o
    assert ann.device_status() == 0


def test_partition_bit_exact_at_full_size(run):
    w, X, out, cent_o, mem_o, off_o = run
    assert np.array_equal(out["centroids"].cpu().numpy().view(np.uint32), cent_o.view(np.uint32))
    assert np.array_equal(out["offsets"].cpu().numpy(), off_o)
    assert np.array_equal(as_u32(out["members"]), mem_o)


def test_shard_knn_sampled_rows_float_rule(run):
    w, X, out, cent_o, mem_o, off_o = run
    rows = np.sort(np.random.default_rng(17).choice(len(mem_o), 256, replace=False))
    oid, od = oracle.shard_knn(X, mem_o, off_o, w.k, rows=rows)
    gid = as_u32(out["knn_id"].index_select(0, T(rows.astype(np.int64))))
    gd = out["knn_d"].index_select(0, T(rows.astype(np.int64))).cpu().numpy()
    assert check_float_lists(X, mem_o[rows], gid, gd, oid, od) == len(rows)


def _gpu_lists(out, rows):
    idx = T(np.asarray(rows, dtype=np.int64))
    return (as_u32(out["knn_id"].index_select(0, idx)),
            out["knn_d"].index_select(0, idx).cpu().numpy().astype(np.float64))


def _oracle_prune_of_gpu_lists(out, mem_o, off_o, rows, k, R):
    """The oracle's prune of row p, given the GPU's kNN lists of p and of its
    neighbours' rows in p's shard (the prune reads only those)."""
    res = {}
    for p in rows:
        s = int(np.searchsorted(off_o, p, side="right") - 1)
        m0, m1 = int(off_o[s]), int(off_o[s + 1])
        mem_s = mem_o[m0:m1]
        offs_s = np.array([0, m1 - m0], dtype=np.int64)
        own, _ = _gpu_lists(out, [p])
        nb = [int(np.searchsorted(mem_s, v)) for v in own[0] if v != oracle.PAD]
        need = np.array(sorted(set([p - m0] + nb)), dtype=np.int64)
        kid = np.full((m1 - m0, k), oracle.PAD, dtype=np.uint32)
        kd = np.full((m1 - m0, k), np.inf)
        kid[need], kd[need] = _gpu_lists(out, need + m0)
        pid, pd = oracle.prune(kid, kd, mem_s, offs_s, R)
        res[p] = (pid[p - m0], pd[p - m0])
    return res


def test_prune_sampled_rows_bit_exact(run):
    w, X, out, cent_o, mem_o, off_o = run
    rows = np.sort(np.random.default_rng(19).choice(len(mem_o), 24, replace=False))
    ref = _oracle_prune_of_gpu_lists(out, mem_o, off_o, rows, w.k, w.R)
    idx = T(rows.astype(np.int64))
    gp = as_u32(out["pr_id"].index_select(0, idx))
    gd = out["pr_d"].index_select(0, idx).cpu().numpy().astype(np.float64)
    for q, p in enumerate(rows):
        assert np.array_equal(gp[q], ref[p][0])
        assert np.array_equal(gd[q], ref[p][1])


def test_merge_sampled_vectors_bit_exact(run):
    """The oracle's merge over the GPU's pruned lists of the sampled vectors' rows
    (every other row empty) gives those vectors' merged lists."""
    w, X, out, cent_o, mem_o, off_o = run
    vecs = np.random.default_rng(23).choice(w.N, 8, replace=False)
    rows = []
    for v in vecs:
        for s in range(w.C):
            seg = mem_o[off_o[s]:off_o[s + 1]]
            j = int(np.searchsorted(seg, v))
            if j < len(seg) and seg[j] == v:
                rows.append(int(off_o[s]) + j)
    rows = np.asarray(rows, dtype=np.int64)
    pid = np.full((len(mem_o), w.R), oracle.PAD, dtype=np.uint32)
    pd = np.full((len(mem_o), w.R), np.inf)
    pid[rows] = as_u32(out["pr_id"].index_select(0, T(rows)))
    pd[rows] = out["pr_d"].index_select(0, T(rows)).cpu().numpy().astype(np.float64)
    og, ogd, odeg = oracle.merge(pid, pd, mem_o, off_o, w.N)
    vi = T(vecs.astype(np.int64))
    g = as_u32(out["graph"].index_select(0, vi))
    gd = out["gdist"].index_select(0, vi).cpu().numpy().astype(np.float64)
    deg = as_u32(out["degree"].index_select(0, vi))
    for q, v in enumerate(vecs):
        assert deg[q] == odeg[v]
        assert np.array_equal(g[q], og[v])
        assert np.array_equal(gd[q], ogd[v])
