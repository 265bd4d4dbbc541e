"""The C-ABI library builds for sm_103a, loads, and exports every symbol that
include/ann.h declares; argument checks run on the host without a GPU."""
import ctypes as ct
import os
import re

import pytest

from paper_2605_10135_gb300 import ann, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "ann.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ann_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def L():
    build.build()
    return ann.lib()


def test_every_declared_symbol_is_exported(L):
    names = _declared()
    assert len(names) >= 15
    for n in names:
        assert hasattr(L, n), n


def test_version_and_error_string(L):
    assert L.ann_version() >= 100
    assert isinstance(L.ann_last_error(), bytes)


def test_workspace_queries_validate_on_host(L):
    n = ct.c_size_t(0)
    assert L.ann_partition_workspace(1000, 64, 4, 2, 100, ct.byref(n)) == 0 and n.value > 0
    assert L.ann_partition_workspace(1000, 64, 4, 5, 100, ct.byref(n)) == 1  # r > C
    assert b"r <= C" in L.ann_last_error()
    assert L.ann_shard_knn_workspace(1000, 128, 3, 16, 2000, 64, 0, 0, ct.byref(n)) == 0
    small = n.value
    assert L.ann_shard_knn_workspace(1000, 128, 3, 16, 4000, 64, 0, 0, ct.byref(n)) == 0
    assert n.value > small
    assert L.ann_shard_knn_workspace(1000, 128, 3, 16, 2000, 0, 0, 0, ct.byref(n)) == 1  # k = 0
    assert L.ann_shard_knn_workspace(1000, 128, 3, 16, 2000, 64, 1, 0, ct.byref(n)) == 0  # BF16 form
    assert L.ann_shard_knn_workspace(1000, 128, 0, 16, 2000, 64, 2, 0, ct.byref(n)) == 0  # E4M3 form
    assert L.ann_shard_knn_workspace(1000, 128, 0, 16, 2000, 64, 4, 0, ct.byref(n)) == 0  # FP16 form
    assert L.ann_shard_knn_workspace(1000, 128, 0, 2000, 2000, 64, 0, 0, ct.byref(n)) == 1  # C
    assert L.ann_shard_knn_workspace(1000, 128, 0, 16, 2000, 64, 2, 32, ct.byref(n)) == 1  # < k
    assert L.ann_shard_knn_workspace(1000, 768, 0, 16, 2000, 64, 3, 0, ct.byref(n)) == 0  # learned
    assert L.ann_shard_knn_workspace(1000, 768, 0, 16, 2000, 64, 0, 0, ct.byref(n)) == 0  # f32 split
    assert L.ann_shard_knn_workspace(1000, 768, 0, 16, 2000, 64, 4, 0, ct.byref(n)) == 0  # streamed
    assert L.ann_shard_knn_workspace(1000, 1024, 1, 16, 2000, 64, 0, 0, ct.byref(n)) == 0  # f16
    assert L.ann_shard_knn_workspace(1000, 512, 3, 16, 2000, 64, 0, 0, ct.byref(n)) == 2  # u8
    assert L.ann_shard_knn_workspace(1000, 128, 3, 16, 2000, 64, 5, 0, ct.byref(n)) == 1  # bad


def test_learned_workspace_queries_validate_on_host(L):
    n = ct.c_size_t(0)
    assert L.ann_learned_train_workspace(10000, 96, 0, 100, 40, 256, ct.byref(n)) == 0
    assert n.value > 10000 * 32 * 4
    assert L.ann_learned_train_workspace(10000, 5000, 0, 100, 40, 256, ct.byref(n)) == 1  # d
    assert L.ann_learned_train_workspace(30, 96, 0, 10, 40, 256, ct.byref(n)) == 1       # N < kk+2
    assert L.ann_learned_embed_workspace(10000, 1024, ct.byref(n)) == 0 and n.value > 0
    f = ct.c_float
    assert L.ann_learned_train(None, 10000, 96, 0, None, 100, 40, 40, None, 1, 256, f(1e-3),
                               f(1e-3), None, None, None, None, 0, None) == 1  # kpos = kk
    assert L.ann_shard_knn_workspace(1000, 512, 3, 16, 2000, 64, 0, 0, ct.byref(n)) == 2  # d > 256
    assert L.ann_merge_workspace(1000, 2000, ct.byref(n)) == 0 and n.value > 0
    assert L.ann_prune(None, None, None, None, 4, 10, 100, 0, 8, 0, None, None, None, 0,
                       None) == 1  # k = 0
    assert L.ann_prune(None, None, None, None, 4, 10, 100, 8, 8, 7, None, None, None, 0,
                       None) == 1  # rule


def test_null_workspace_is_rejected(L):
    n = ct.c_size_t(0)
    assert L.ann_merge_workspace(1000, 2000, ct.byref(n)) == 0
    rc = L.ann_merge(ct.c_void_p(16), ct.c_void_p(16), ct.c_void_p(16), ct.c_void_p(16), 4, 2000,
                     1000, 8, ct.c_void_p(16), ct.c_void_p(16), ct.c_void_p(16), None, 0, None)
    assert rc == 5 and b"workspace" in L.ann_last_error()


def test_host_side_failures_return_status_codes(L):
    """Argument and workspace failures are caught on the host before any launch."""
    n = ct.c_size_t(0)
    assert L.ann_wait_selftest(2, 100, None) == 1
    assert L.ann_wait_selftest(0, 0, None) == 1
    dummy = ct.c_void_p(16)  # never dereferenced: the calls fail before using it
    buf = (ct.c_int64 * 3)(0, 1000, 2000)
    assert L.ann_shard_knn_workspace(1000, 64, 3, 2, 2000, 16, 0, 0, ct.byref(n)) == 0
    rc = L.ann_shard_knn(dummy, 1000, 64, 3, dummy, ct.cast(buf, ct.c_void_p), 2, 2000, 16, 0, 0,
                         None, dummy, dummy, None, 0, None)
    assert rc == 5 and b"workspace" in L.ann_last_error().lower()


def test_selective_partition_arguments_validate_on_host(L):
    n = ct.c_size_t(0)
    P = ann._SelectiveParams
    ok = P(1.2, 2.0, 4096, 0, 2, 8)
    assert L.ann_partition_selective_workspace(10000, 96, 16, 1000, ct.byref(ok), ct.byref(n)) == 0
    small = n.value
    assert small > 10000 * 8 * 8
    capped = P(1.2, 2.0, 4096, 3000, 2, 8)
    assert L.ann_partition_selective_workspace(10000, 96, 16, 1000, ct.byref(capped),
                                               ct.byref(n)) == 0
    inf = P(float("inf"), 1.0, 1, 0, 3, 16)
    assert L.ann_partition_selective_workspace(10000, 96, 16, 1000, ct.byref(inf), ct.byref(n)) == 0
    bad = [P(1.2, 2.0, 4096, 0, 9, 8),            # omega > cand
           P(1.2, 2.0, 4096, 0, 2, 17),           # cand > C
           P(1.2, 2.0, 0, 0, 2, 8),               # block
           P(float("nan"), 2.0, 4096, 0, 2, 8),   # eps
           P(-1.0, 2.0, 4096, 0, 2, 8),
           P(1.2, float("inf"), 4096, 0, 2, 8),   # tau0
           P(1.2, 2.0, 4096, -5, 2, 8)]           # capacity
    for p in bad:
        assert L.ann_partition_selective_workspace(10000, 96, 16, 1000, ct.byref(p),
                                                   ct.byref(n)) == 1
    assert L.ann_partition_selective_workspace(10000, 96, 16, 1000, None, ct.byref(n)) == 1
    big = P(1.2, 2.0, 4096, 0, 2, 33)
    assert L.ann_partition_selective_workspace(10000, 96, 64, 1000, ct.byref(big), ct.byref(n)) == 1
    dummy = ct.c_void_p(16)
    rc = L.ann_partition_selective(dummy, 10000, 96, 0, 16, dummy, dummy, 1000, 5, ct.byref(ok),
                                   dummy, None, dummy, dummy, None, None, 0, None)
    assert rc == 5 and b"workspace" in L.ann_last_error().lower()


def test_pageable_vectors_are_refused_before_any_launch(L):
    """Vectors must be device memory or page-locked host memory mapped for the
    device; a plain host array is refused on the host (here, with no GPU at all,
    the pointer query itself fails) after the workspace checks pass."""
    import numpy as np
    import torch
    if torch.cuda.is_available():
        pytest.skip("checks the no-device path; tests/test_gpu_host_vectors.py covers GPUs")
    X = np.zeros((100, 16), np.uint8)
    n = ct.c_size_t(0)
    assert L.ann_medoid_workspace(100, 16, ct.byref(n)) == 0
    ws = (ct.c_char * max(n.value, 1))()
    l0 = L.ann_launch_count()
    rc = L.ann_medoid(X.ctypes.data_as(ct.c_void_p), 100, 16, 3, ct.c_void_p(16),
                      ct.cast(ws, ct.c_void_p), n.value, None)
    assert rc == 1
    assert L.ann_launch_count() == l0
