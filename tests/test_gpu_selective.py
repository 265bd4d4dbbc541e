"""Blockwise-adaptive assignment with selective replication (Sec. V) on the GPU,
through the C-ABI, against the CPU oracle: centroids, per-vector shard lists,
statistics and member lists bit for bit, with and without a shard capacity,
ragged blocks, screened centroids (C > 32), the Fig. 2 example, and a whole
build on selectively replicated shards.
"""
import os

import numpy as np
import pytest
import torch

import oracle
from paper_2605_10135_gb300 import ann, build, datagen
from tests.parity import as_u32

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
GOLD = os.path.join(os.path.dirname(__file__), "golden")


def T(a):
    a = np.ascontiguousarray(a)
    if a.dtype == np.uint32:
        a = a.view(np.int32)
    return torch.from_numpy(a).to(DEV)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    ann.lib()
    ann.device_status()
    yield
    assert ann.device_status() == 0


def _run(X, C, omega, iters, sel, seed):
    sample, init_rows = datagen.kmeans_sample(X.shape[0], C, seed)
    init = X[init_rows].astype(np.float32)
    cent, mem, off, stats, assign = ann.partition_selective(
        T(X), C, omega, T(init), T(sample), iters, sel, with_assign=True)
    torch.cuda.synchronize()
    got = (cent.cpu().numpy(), as_u32(mem), off.cpu().numpy(), stats.cpu().numpy(),
           as_u32(assign))
    cent_o, _ = oracle.kmeans(X, init, sample, iters)
    a_o, st_o = oracle.selective(X, cent_o, omega, M=min(sel.cand, C), eps=sel.epsilon,
                                 tau0=sel.tau0, block=sel.block, cap=sel.capacity)
    mem_o, off_o = oracle.shards(a_o, C)
    return got, (cent_o, mem_o, off_o, st_o, a_o)


def _check(got, ref):
    cent, mem, off, stats, assign = got
    cent_o, mem_o, off_o, st_o, a_o = ref
    assert np.array_equal(cent.view(np.uint32), cent_o.view(np.uint32))
    assert np.array_equal(assign, a_o)
    assert stats.tolist() == st_o.tolist()
    assert np.array_equal(off, off_o)
    assert np.array_equal(mem, mem_o[:int(off_o[-1])])


@pytest.mark.parametrize("kind", ["u8", "f32"])
@pytest.mark.parametrize("eps,tau0", [(1.2, 2.0), (1.1, 1.0), (1.5, 4.0), (float("inf"), 1.0)])
def test_selective_no_capacity_bit_exact(kind, eps, tau0):
    if kind == "u8":
        X = datagen.clustered_u8(5000, 64, 40, seed=201)
    else:
        X = datagen.gaussian_mixture_f32(5003, 48, 24, 2.0, seed=202)
    sel = ann.SelectiveConfig(epsilon=eps, tau0=tau0, block=777, capacity=0, cand=8)
    got, ref = _run(X, 12, 2, 5, sel, seed=203)
    _check(got, ref)
    if np.isinf(eps):
        assert got[3][0] == X.shape[0]  # every vector replicated once
    else:
        assert 0 < got[3][0] < X.shape[0]


@pytest.mark.parametrize("kind", ["u8", "f32"])
@pytest.mark.parametrize("cap_factor,omega,block", [(1.6, 2, 1000), (1.1, 3, 333), (0.7, 2, 4096),
                                                    (1.3, 2, 1)])
def test_selective_with_capacity_bit_exact(kind, cap_factor, omega, block):
    """Capacity binds (cap_factor < 1 also overflows); the sequential block walk
    must give the oracle's id-order result, including where 32 vectors compete."""
    n = 2500 if block == 1 else 6000
    if kind == "u8":
        X = datagen.clustered_u8(n, 32, 30, seed=211)
    else:
        X = datagen.gaussian_mixture_f32(n, 32, 20, 2.0, seed=212)
    C = 10
    cap = int(np.ceil(cap_factor * n / C))
    sel = ann.SelectiveConfig(epsilon=1.5, tau0=2.0, block=block, capacity=cap, cand=10)
    got, ref = _run(X, C, omega, 4, sel, seed=213)
    _check(got, ref)
    counts = np.diff(got[2])
    if cap_factor >= 1.5:  # room to spare: nobody overflows, no shard above capacity
        assert got[3][1] == 0 and counts.max() <= cap
    elif cap_factor < 1.0:  # fewer slots than vectors: some originals must overflow
        assert got[3][1] > 0


def test_capacity_equal_to_no_capacity_when_it_never_binds():
    X = datagen.clustered_u8(4000, 32, 30, seed=221)
    free = ann.SelectiveConfig(epsilon=1.3, tau0=3.0, block=500, capacity=0, cand=6)
    loose = ann.SelectiveConfig(epsilon=1.3, tau0=3.0, block=500, capacity=4000 * 2, cand=6)
    g1, _ = _run(X, 8, 2, 3, free, seed=222)
    g2, _ = _run(X, 8, 2, 3, loose, seed=222)
    for a, b in zip(g1, g2):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("kind", ["u8", "f32"])
def test_selective_screened_centroids(kind):
    """C > 32: the candidate lists come from the tensor-core screen plus d32."""
    if kind == "u8":
        X = datagen.clustered_u8(6000, 128, 64, seed=231)
    else:
        X = datagen.gaussian_mixture_f32(6000, 64, 64, 2.0, seed=232)
    sel = ann.SelectiveConfig(epsilon=1.2, tau0=2.0, block=2048, capacity=0, cand=12)
    got, ref = _run(X, 48, 2, 3, sel, seed=233)
    _check(got, ref)
    sel = ann.SelectiveConfig(epsilon=1.2, tau0=2.0, block=2048, capacity=300, cand=12)
    got, ref = _run(X, 48, 3, 3, sel, seed=233)
    _check(got, ref)


def test_fig2_example_on_the_gpu():
    X = np.array([[2, 4], [9, 1], [4, 6]], np.float32)
    cent = np.array([[0, 0], [10, 0], [5, 8]], np.float32)
    sample = np.arange(3, dtype=np.uint32)
    cases = [(1.2, 2.0, 3, 2, [[0, 2], [1, PADI], [2, PADI]], [1, 0]),
             (1.2, 1.0, 3, 2, [[0, PADI], [1, PADI], [2, PADI]], [0, 0]),
             (float("inf"), 1.0, 1, 2, [[0, 2], [1, 2], [0, 1]], [3, 0])]
    for eps, tau0, block, cap, want, st in cases:
        sel = ann.SelectiveConfig(epsilon=eps, tau0=tau0, block=block, capacity=cap, cand=3)
        _, mem, off, stats, assign = ann.partition_selective(T(X), 3, 2, T(cent), T(sample), 0,
                                                             sel, with_assign=True)
        torch.cuda.synchronize()
        assert as_u32(assign).tolist() == [[int(v) for v in row] for row in want]
        assert stats.cpu().tolist() == st


PADI = 0xFFFFFFFF


def test_build_on_selective_shards():
    """The rest of the path runs on the variable replication: kNN lists of the
    selective shards bit-exact (uint8), merged graph valid."""
    X = datagen.clustered_u8(4000, 64, 32, seed=241)
    C, k, R = 8, 16, 8
    sample, init_rows = datagen.kmeans_sample(X.shape[0], C, 242)
    init = X[init_rows].astype(np.float32)
    cfg = ann.BuildConfig(C=C, r=2, k=k, R=R, iters=4,
                          selective=ann.SelectiveConfig(epsilon=1.2, tau0=2.0, block=1000))
    out = ann.build_index(T(X), cfg, T(init), T(sample))
    torch.cuda.synchronize()
    mem, off = as_u32(out["members"]), out["offsets"].cpu().numpy()
    rows = int(off[-1])
    st = out["selective_stats"].cpu().numpy()
    assert rows == X.shape[0] + st[0] and 0 < st[0] < X.shape[0]
    ids_o, ds_o = oracle.shard_knn(X, mem, off, k)
    assert np.array_equal(as_u32(out["knn_id"]), ids_o)
    assert np.array_equal(out["knn_d"].cpu().numpy().astype(np.float64), ds_o)
    pid_o, pd_o = oracle.prune(ids_o, ds_o, mem, off, R)
    assert np.array_equal(as_u32(out["pr_id"]), pid_o)
    g_o, gd_o, deg_o = oracle.merge(pid_o, pd_o, mem, off, X.shape[0])
    assert np.array_equal(as_u32(out["graph"]), g_o)
    assert np.array_equal(as_u32(out["degree"]), deg_o)
