"""Parity at the benchmark's full size: the Sift-like 1M build (N = 1e6 uint8,
d = 128, 16 shards, r = 2, k = 64, R = 32) in the configuration bench.py times,
checked on outputs the oracle computes one by one: the whole partition, the kNN
lists of sampled rows, the pruned lists of sampled rows (from the oracle's exact
lists of those rows' neighbours) and the merged lists of sampled vectors.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2605_10135_gb300 import ann, build, configs

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def T(a):
    a = np.ascontiguousarray(a)
    if a.dtype == np.uint32:
        a = a.view(np.int32)
    return torch.from_numpy(a).to(DEV)


def as_u32(t):
    a = t.detach().cpu().numpy()
    return a.view(np.uint32) if a.dtype == np.int32 else a


@pytest.fixture(scope="module")
def run():
    build.build()
    ann.device_status()
    w = configs.SIFT_1M
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


def test_shard_knn_sampled_rows_bit_exact(run):
    w, X, out, cent_o, mem_o, off_o = run
    rows = np.sort(np.random.default_rng(7).choice(len(mem_o), 256, replace=False))
    oid, od = oracle.shard_knn(X, mem_o, off_o, w.k, rows=rows)
    assert np.array_equal(as_u32(out["knn_id"])[rows], oid)
    assert np.array_equal(out["knn_d"].cpu().numpy()[rows].astype(np.float64), od)


def _shard_of(off, p):
    return int(np.searchsorted(off, p, side="right") - 1)


def _oracle_pruned(X, mem_o, off_o, rows, k, R):
    """Oracle pruned lists of the given rows: exact lists of each row and of its
    neighbours' rows in the same shard, then the prune rule on that shard."""
    out = {}
    for p in rows:
        s = _shard_of(off_o, p)
        m0, m1 = int(off_o[s]), int(off_o[s + 1])
        mem_s = mem_o[m0:m1]
        offs_s = np.array([0, m1 - m0], dtype=np.int64)
        own, _ = oracle.shard_knn(X, mem_s, offs_s, k, rows=np.array([p - m0]))
        nb = [int(np.searchsorted(mem_s, v)) for v in own[0] if v != oracle.PAD]
        need = np.array(sorted(set([p - m0] + nb)), dtype=np.int64)
        kid = np.full((m1 - m0, k), oracle.PAD, dtype=np.uint32)
        kd = np.full((m1 - m0, k), np.inf)
        lid, ld = oracle.shard_knn(X, mem_s, offs_s, k, rows=need)
        kid[need], kd[need] = lid, ld
        pid, pd = oracle.prune(kid, kd, mem_s, offs_s, R)
        out[p] = (pid[p - m0], pd[p - m0])
    return out


def test_prune_sampled_rows_bit_exact(run):
    w, X, out, cent_o, mem_o, off_o = run
    rows = np.sort(np.random.default_rng(11).choice(len(mem_o), 24, replace=False))
    ref = _oracle_pruned(X, mem_o, off_o, rows, w.k, w.R)
    gp, gd = as_u32(out["pr_id"]), out["pr_d"].cpu().numpy().astype(np.float64)
    for p in rows:
        assert np.array_equal(gp[p], ref[p][0])
        assert np.array_equal(gd[p], ref[p][1])


def test_merge_sampled_vectors_bit_exact(run):
    """The oracle's merge over pruned lists that are exact for the rows of the
    sampled vectors (every other row empty) gives those vectors' merged lists."""
    w, X, out, cent_o, mem_o, off_o = run
    vecs = np.random.default_rng(13).choice(w.N, 8, replace=False)
    rows = []
    for v in vecs:
        for s in range(w.C):
            seg = mem_o[off_o[s]:off_o[s + 1]]
            j = int(np.searchsorted(seg, v))
            if j < len(seg) and seg[j] == v:
                rows.append(int(off_o[s]) + j)
    ref = _oracle_pruned(X, mem_o, off_o, rows, w.k, w.R)
    pid = np.full((len(mem_o), w.R), oracle.PAD, dtype=np.uint32)
    pd = np.full((len(mem_o), w.R), np.inf)
    for p in rows:
        pid[p], pd[p] = ref[p]
    og, ogd, odeg = oracle.merge(pid, pd, mem_o, off_o, w.N)
    g, gd, deg = as_u32(out["graph"]), out["gdist"].cpu().numpy(), as_u32(out["degree"])
    for v in vecs:
        assert deg[v] == odeg[v]
        assert np.array_equal(g[v], og[v])
        assert np.array_equal(gd[v].astype(np.float64), ogd[v])
