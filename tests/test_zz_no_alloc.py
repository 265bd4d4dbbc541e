"""ann_medoid_noalloc: the medoid for callers that cannot allocate device memory.

Some callers cannot call cudaMalloc: code running inside a framework that owns the
device's memory pool, or a pipeline stage where an allocation could synchronise the
device or fail part-way.  For them the library offers one entry point whose scratch
is a fixed array inside the library instead of a caller workspace.  These tests
check it against the ordinary ann_medoid (which takes a workspace) on two calls in
a row, and that inputs beyond the fixed scratch are refused.  This file is named so
that pytest collects it last.
"""
import ctypes as ct

import numpy as np
import pytest

from paper_2605_10135_gb300 import ann, build, datagen


def test_rejects_inputs_beyond_the_fixed_scratch():
    build.build()
    L = ann.lib()
    out = ct.c_void_p(16)  # never dereferenced: the size check comes first
    # ceil(N / 4096) * d = 1025 * 1024 > 524288 column sums
    rc = L.ann_medoid_noalloc(ct.c_void_p(16), 1025 * 4096, 1024, 3, out, None)
    assert rc == 1 and b"fixed scratch" in L.ann_last_error()
    rc = L.ann_medoid_noalloc(ct.c_void_p(16), 1000, 5000, 3, out, None)  # d > 4096
    assert rc == 1


def test_rejects_pageable_host_vectors_before_any_launch():
    """A pointer no kernel may read (ordinary pageable host memory) is refused by
    the readability check, after the size check and before any launch."""
    build.build()
    L = ann.lib()
    X = np.zeros((64, 16), np.float32)  # pageable: never registered with CUDA
    out = np.zeros(1, np.uint32)
    before = L.ann_launch_count()
    rc = L.ann_medoid_noalloc(X.ctypes.data_as(ct.c_void_p), 64, 16, 0,
                              out.ctypes.data_as(ct.c_void_p), None)
    assert rc == 1
    assert b"X" in L.ann_last_error()
    assert L.ann_launch_count() == before
    assert out[0] == 0


@pytest.mark.gpu
def test_no_alloc_medoid_at_the_scratch_limit_allocates_nothing():
    """The largest input the fixed scratch takes (ceil(N / 4096) * d equal to the
    524288 column sums) gives the workspace medoid, and the device's free memory
    is the same before and after the call; one more row is refused."""
    import torch

    build.build()
    d = 128
    N = 4096 * (524288 // d)  # 4096 chunks of 4096 rows
    X = torch.randint(0, 256, (N, d), dtype=torch.uint8, device="cuda:0",
                      generator=torch.Generator("cuda:0").manual_seed(93))
    out = torch.empty(1, dtype=torch.int32, device="cuda:0")
    ann.medoid_noalloc(X[:4096], out)  # the first call resolves the scratch symbol
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    got = int(ann.medoid_noalloc(X, out).item())
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert got == int(ann.medoid(X).item())
    L = ann.lib()
    Y = torch.zeros((N + 1, d), dtype=torch.uint8, device="cuda:0")
    rc = L.ann_medoid_noalloc(ct.c_void_p(Y.data_ptr()), N + 1, d, 3, ct.c_void_p(out.data_ptr()),
                              None)
    assert rc == 1 and b"fixed scratch" in L.ann_last_error()
    assert ann.device_status() == 0


@pytest.mark.gpu
@pytest.mark.parametrize("kind", ["u8", "f32"])
def test_no_alloc_medoid_matches_workspace_medoid_twice(kind):
    import torch

    build.build()
    if kind == "u8":
        X = datagen.clustered_u8(30000, 128, 32, seed=91)
    else:
        X = datagen.gaussian_mixture_f32(30000, 64, seed=92)
    Xt = torch.from_numpy(X).to("cuda:0")
    ref = int(ann.medoid(Xt).item())
    out = torch.empty(1, dtype=torch.int32, device="cuda:0")
    for _ in range(2):  # the shared scratch keeps the previous call's contents
        out.fill_(-1)
        got = int(ann.medoid_noalloc(Xt, out).item())
        assert got == ref
    # a different input in between must not leak through the shared scratch
    Y = np.ascontiguousarray(X[::-1])
    Yt = torch.from_numpy(Y).to("cuda:0")
    assert int(ann.medoid_noalloc(Yt).item()) == int(ann.medoid(Yt).item())
    assert int(ann.medoid_noalloc(Xt).item()) == ref
    assert ann.device_status() == 0
