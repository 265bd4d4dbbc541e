"""Vectors left in page-locked host memory: the kernels read them over the host
link (NVLink-C2C on Grace-Blackwell) and every result equals the one from a
device copy of the same vectors; pageable host memory is refused before any
launch."""
import ctypes as ct

import numpy as np
import pytest
import torch

from paper_2605_10135_gb300 import ann, build, datagen
from tests.parity import as_u32

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    ann.lib()
    ann.device_status()
    yield
    assert ann.device_status() == 0


def _pinned(a):
    return torch.from_numpy(np.ascontiguousarray(a)).pin_memory()


def _same(a, b):
    if isinstance(a, torch.Tensor):
        return torch.equal(a.cpu(), b.cpu())
    return a == b


@pytest.mark.parametrize("kind", ["u8", "f32"])
def test_build_from_host_vectors_equals_device(kind):
    if kind == "u8":
        X = datagen.clustered_u8(5000, 128, 32, seed=301)
    else:
        X = datagen.gaussian_mixture_f32(5000, 96, 24, 2.0, seed=302)
    C = 6
    sample, init_rows = datagen.kmeans_sample(X.shape[0], C, 303)
    init = torch.from_numpy(X[init_rows].astype(np.float32)).to(DEV)
    samp = torch.from_numpy(sample.view(np.int32)).to(DEV)
    cfg = ann.BuildConfig(C=C, r=2, k=24, R=12, iters=4)
    ref = ann.build_index(torch.from_numpy(X).to(DEV), cfg, init, samp)
    got = ann.build_index(_pinned(X), cfg, init, samp)
    torch.cuda.synchronize()
    for key in ("centroids", "members", "offsets", "knn_id", "knn_d", "pr_id", "graph", "gdist",
                "degree"):
        assert _same(ref[key], got[key]), key
    sel = ann.SelectiveConfig(epsilon=1.2, tau0=2.0, block=1024)
    a = ann.partition_selective(torch.from_numpy(X).to(DEV), C, 2, init, samp, 4, sel, True)
    b = ann.partition_selective(_pinned(X), C, 2, init, samp, 4, sel, True)
    for x, y in zip(a, b):
        assert _same(x, y)


def test_queries_and_search_from_host_vectors():
    X = datagen.clustered_u8(4000, 64, 16, seed=311)
    Q = datagen.clustered_u8(100, 64, 16, seed=312)
    Xd, Qd = torch.from_numpy(X).to(DEV), torch.from_numpy(Q).to(DEV)
    Xh, Qh = _pinned(X), _pinned(Q)
    gi, gd = ann.knn_query(Xd, Qd, 10)
    hi, hd = ann.knn_query(Xh, Qh, 10)
    assert torch.equal(gi, hi) and torch.equal(gd, hd)
    assert int(ann.medoid(Xd).item()) == int(ann.medoid(Xh).item())
    C = 4
    sample, init_rows = datagen.kmeans_sample(X.shape[0], C, 313)
    init = torch.from_numpy(X[init_rows].astype(np.float32)).to(DEV)
    samp = torch.from_numpy(sample.view(np.int32)).to(DEV)
    out = ann.build_index(Xd, ann.BuildConfig(C=C, r=2, k=16, R=8, iters=3), init, samp)
    ent = torch.arange(0, 4000, 97, dtype=torch.int32, device=DEV)
    a = ann.search_entries(out["graph"], out["degree"], Xd, Qd, ent, 32)
    b = ann.search_entries(out["graph"], out["degree"], Xh, Qh, ent, 32)
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])


def test_pageable_host_memory_is_refused_before_any_launch():
    X = np.ascontiguousarray(datagen.clustered_u8(2000, 32, 8, seed=321))
    with pytest.raises(ValueError):
        ann.medoid(torch.from_numpy(X))  # the binding refuses unpinned CPU tensors
    L = ann.lib()
    n = ct.c_size_t(0)
    assert L.ann_medoid_workspace(2000, 32, ct.byref(n)) == 0
    ws = torch.empty(max(n.value, 1), dtype=torch.uint8, device=DEV)
    out = torch.full((1,), -1, dtype=torch.int32, device=DEV)
    l0 = ann.launch_count()
    rc = L.ann_medoid(X.ctypes.data_as(ct.c_void_p), 2000, 32, 3, ct.c_void_p(out.data_ptr()),
                      ct.c_void_p(ws.data_ptr()), n.value, None)
    torch.cuda.synchronize()
    if rc == 0:  # a platform that maps pageable memory for the device: result must hold
        assert int(out.item()) == int(ann.medoid(torch.from_numpy(X).to(DEV)).item())
    else:
        assert rc == 1 and b"page-locked" in L.ann_last_error()
        assert ann.launch_count() == l0


@pytest.mark.parametrize("kind,host", [("u8", False), ("u8", True), ("f32", True)])
def test_streamed_build_equals_whole_build(kind, host):
    """One shard at a time (kNN lists of one shard resident at a time) gives the
    same partition, pruned lists and merged graph as the all-shard build."""
    if kind == "u8":
        X = datagen.clustered_u8(6000, 64, 24, seed=331)
    else:
        X = datagen.gaussian_mixture_f32(5000, 48, 16, 2.0, seed=332)
    C = 7
    sample, init_rows = datagen.kmeans_sample(X.shape[0], C, 333)
    init = torch.from_numpy(X[init_rows].astype(np.float32)).to(DEV)
    samp = torch.from_numpy(sample.view(np.int32)).to(DEV)
    cfg = ann.BuildConfig(C=C, r=2, k=20, R=10, iters=4)
    ref = ann.build_index(torch.from_numpy(X).to(DEV), cfg, init, samp)
    Xs = _pinned(X) if host else torch.from_numpy(X).to(DEV)
    got = ann.build_index_streamed(Xs, cfg, init, samp)
    torch.cuda.synchronize()
    for key in ("centroids", "members", "offsets", "pr_id", "pr_d", "graph", "gdist", "degree"):
        assert _same(ref[key], got[key]), key
    cfg_s = ann.BuildConfig(C=C, r=2, k=20, R=10, iters=4,
                            selective=ann.SelectiveConfig(epsilon=1.2, tau0=2.0, block=2000))
    ref = ann.build_index(torch.from_numpy(X).to(DEV), cfg_s, init, samp)
    got = ann.build_index_streamed(Xs, cfg_s, init, samp)
    for key in ("members", "offsets", "pr_id", "graph", "degree"):
        assert _same(ref[key], got[key]), key
