"""FP64 oracle of the precision forms' screening (TEST INFRASTRUCTURE ONLY).

Only the tests and the benchmark's measurement legs import this module.  It
shares no code with the CUDA library.

The paper builds every shard graph from exact distances (Sec. II-B, Sec. IV
Workflow (2)) and fixes no arithmetic precision.  The precision forms are an
addition beside the method: distance tiles in a narrow operand type screen a
widened candidate list, which an exact re-rank then orders.  This file writes
that definition out plainly:

* operands   x is rounded element by element to the operand type, round to
             nearest even, finite values saturated to the largest finite value:
             BF16 (8 significant bits); FP16 after one power-of-two scale that
             puts max|x| in [2^13, 2^14); E4M3 (4 significant bits, largest
             finite 448, subnormal step 2^-9) after the scale 448 / max|x|.
             The scale is one float32 number for the whole array and the scaled
             value is the float32 product x * scale.
* key        for row u and member v of its shard, key = |s v|^2 / 2 - q(u) . q(v),
             where s v is the scaled float32 vector, q() its rounded copy, and
             the arithmetic is FP64; the screening distance is |s u|^2 + 2 key,
             divided by scale^2.
* screening  the kprime members v != u of smallest (key, id).
* re-rank    those candidates by exact FP64 squared distance (ties to the
             smaller id), first k kept.
"""
from __future__ import annotations

import numpy as np

from . import oracle as _o

E4M3_MAX = 448.0
BF16, F16, E4M3 = "bf16", "f16", "e4m3"


def _round_to_bits(v: np.ndarray, mant_bits: int, min_exp: int, max_val: float) -> np.ndarray:
    """Round float64 values to a binary format with `mant_bits` fraction bits,
    smallest normal exponent `min_exp` (subnormals below it), largest finite
    value `max_val`; round to nearest even, saturating."""
    v = np.asarray(v, dtype=np.float64)
    a = np.abs(v)
    with np.errstate(divide="ignore"):
        e = np.floor(np.log2(np.where(a > 0, a, 1.0)))
    e = np.maximum(e, min_exp)
    quantum = np.exp2(e - mant_bits)
    q = np.round(a / quantum) * quantum  # np.round: half to even
    q = np.minimum(q, max_val)
    return np.copysign(q, v)


def round_bf16(v) -> np.ndarray:
    """BF16: 7 fraction bits, exponent range of float32."""
    return _round_to_bits(v, 7, -126, float(np.finfo(np.float32).max))


def round_e4m3(v) -> np.ndarray:
    """E4M3: 3 fraction bits, smallest normal 2^-6, largest finite 448."""
    return _round_to_bits(v, 3, -6, E4M3_MAX)


def round_f16(v) -> np.ndarray:
    """IEEE half: 10 fraction bits, smallest normal 2^-14, largest finite 65504."""
    return _round_to_bits(v, 10, -14, 65504.0)


def operand_scale(X: np.ndarray, form: str) -> np.float32:
    """The one float32 scale of the whole array (1 for BF16)."""
    am = np.float32(np.max(np.abs(X.astype(np.float32)))) if X.size else np.float32(0)
    if form == E4M3:
        return np.float32(E4M3_MAX) / am if am > 0 else np.float32(1)
    if form == F16:
        if am <= 0:
            return np.float32(1)
        _, ex = np.frexp(am)  # am = m 2^ex, m in [0.5, 1)
        return np.float32(np.ldexp(1.0, 14 - int(ex)))
    return np.float32(1)


def operands(X: np.ndarray, form: str):
    """(scaled float32 vectors as float64, their rounded copies, scale)."""
    s = operand_scale(X, form)
    v = (X.astype(np.float32) * s).astype(np.float64)
    q = {BF16: round_bf16, F16: round_f16, E4M3: round_e4m3}[form](v)
    return v, q, float(s)


def screen_rows(X, members, offsets, form, kprime, k, rows):
    """For each shard row in `rows` (positions into members): the screening list
    (ids [kprime], screening distances [kprime], unscaled) and the re-ranked
    result (ids [k], exact FP64 distances [k]); PAD / inf past the shard's end."""
    members = np.asarray(members, dtype=np.int64)
    offsets = np.asarray(offsets, dtype=np.int64)
    v, q, s = operands(X, form)
    nv = (v * v).sum(1)
    Xd = X.astype(np.float64)
    n = len(rows)
    sid = np.full((n, kprime), _o.PAD, np.uint32)
    sdist = np.full((n, kprime), np.inf)
    rid = np.full((n, k), _o.PAD, np.uint32)
    rdist = np.full((n, k), np.inf)
    for i, p in enumerate(rows):
        sh = int(np.searchsorted(offsets, p, side="right") - 1)
        mem = members[offsets[sh]:offsets[sh + 1]]
        u = int(members[p])
        cand = mem[mem != u]
        key = nv[cand] / 2.0 - q[cand] @ q[u]
        order = np.lexsort((cand, key))[:kprime]
        c = cand[order]
        sid[i, :len(c)] = c
        sdist[i, :len(c)] = (nv[u] + 2.0 * key[order]) / (s * s)
        de = ((Xd[c] - Xd[u]) ** 2).sum(1)
        o2 = np.lexsort((c, de))[:k]
        rid[i, :len(o2)] = c[o2]
        rdist[i, :len(o2)] = de[o2]
    return sid, sdist, rid, rdist


def distance_error_rows(X, row_vecs, ids, dist):
    """Relative error |dist - d64| / d64 of each listed (row, id) distance, for
    rows whose vectors are X[row_vecs]: (max, mean) over entries with d64 > 0."""
    Xd = X.astype(np.float64)
    rel = []
    for r in range(ids.shape[0]):
        ok = ids[r] != _o.PAD
        if not ok.any():
            continue
        c = ids[r][ok].astype(np.int64)
        de = ((Xd[c] - Xd[int(row_vecs[r])]) ** 2).sum(1)
        pos = de > 0
        rel.append(np.abs(dist[r][ok][pos] - de[pos]) / de[pos])
    if not rel:
        return 0.0, 0.0
    allr = np.concatenate(rel)
    return float(allr.max()), float(allr.mean())
