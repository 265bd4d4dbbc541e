"""Comparison rules between the CUDA path and the oracle.

Integer data: bit-exact ids and distances.  Float data (the kNN lists): the
rule fixed for the exact build - with d_k the oracle's k-th distance of a row,
the GPU list must (1) contain every id whose FP64 distance is below
d_k (1 - 1e-5), (2) hold only ids whose FP64 distance is at most
d_k (1 + 1e-5), (3) report each distance within 1e-5 relative of FP64 (exact
zeros exactly), and (4) be sorted by (distance, id); padding must match.
"""
from __future__ import annotations

import numpy as np

PAD = 0xFFFFFFFF
RTOL = 1e-5


def as_u32(t) -> np.ndarray:
    a = t.detach().cpu().numpy() if hasattr(t, "detach") else np.asarray(t)
    return a.view(np.uint32) if a.dtype == np.int32 else a.astype(np.uint32)


def d64_pairs(X: np.ndarray, u: int, ids: np.ndarray) -> np.ndarray:
    x = X[u].astype(np.float64)
    return ((X[ids].astype(np.float64) - x[None, :]) ** 2).sum(axis=1)


def check_float_lists(X, row_vec_ids, gpu_id, gpu_d, or_id, or_d, rtol=RTOL):
    """Apply the float rule row by row; returns the number of rows checked."""
    gpu_id = as_u32(gpu_id)
    gpu_d = np.asarray(gpu_d, dtype=np.float64)
    for q, u in enumerate(row_vec_ids):
        oi, od = or_id[q], or_d[q]
        gi, gd = gpu_id[q], gpu_d[q]
        ov = oi != PAD
        gv = gi != PAD
        assert np.array_equal(ov, gv), f"row {q}: padding differs"
        if not ov.any():
            continue
        dk = od[ov][-1]
        must = oi[ov][od[ov] < dk * (1 - rtol)]
        assert set(must.tolist()) <= set(gi[gv].tolist()), f"row {q}: missing a sure neighbour"
        true_d = d64_pairs(X, int(u), gi[gv].astype(np.int64))
        assert np.all(true_d <= dk * (1 + rtol) + 0.0), f"row {q}: an id beyond the k-th distance"
        err = np.abs(gd[gv] - true_d)
        assert np.all(err <= rtol * true_d), f"row {q}: distance error {err.max()}"
        assert np.all(gd[gv][true_d == 0] == 0)
        key = list(zip(gd[gv].tolist(), gi[gv].tolist()))
        assert key == sorted(key), f"row {q}: not sorted by (distance, id)"
        assert len(set(gi[gv].tolist())) == int(gv.sum()), f"row {q}: duplicate ids"
    return len(row_vec_ids)
