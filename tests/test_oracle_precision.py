"""Pins of the precision forms' screening oracle (oracle/precision.py), on the CPU.

The rounding functions are checked against the formats' definitions (largest
finite values, subnormal steps, ties to even) and against library conversions
of the same formats; the screening is checked by reductions to the exact kNN:
a list that keeps every member, and integer data that BF16 holds exactly.
"""
import numpy as np
import pytest
import torch

import oracle
from oracle import precision as P
from paper_2605_10135_gb300 import datagen


def test_e4m3_rounding_at_the_format_boundaries():
    # 3 fraction bits: 1 + 1/16 is halfway between 1 and 1.125 -> even (1.0);
    # 1 + 3/16 halfway between 1.125 and 1.25 -> even (1.25)
    assert P.round_e4m3([1.0625, 1.1875]).tolist() == [1.0, 1.25]
    # largest finite 448 = 1.75 * 2^8; beyond it saturates
    assert P.round_e4m3([448.0, 460.0, 1e6, -1e6]).tolist() == [448.0, 448.0, 448.0, -448.0]
    # subnormal step 2^-9: 2^-10 ties to 0 (even), 3 * 2^-10 ties to 2^-8 (even)
    assert P.round_e4m3([2.0 ** -10, 3 * 2.0 ** -10, 2.0 ** -9]).tolist() == \
        [0.0, 2.0 ** -8, 2.0 ** -9]
    # smallest normal 2^-6 and the step just below it
    assert P.round_e4m3([2.0 ** -6, 2.0 ** -6 - 2.0 ** -9]).tolist() == \
        [2.0 ** -6, 2.0 ** -6 - 2.0 ** -9]


def test_rounding_equals_library_conversions():
    rng = np.random.default_rng(5)
    x = (rng.normal(size=20000) * rng.choice([1e-3, 1.0, 30.0], 20000)).astype(np.float32)
    assert np.array_equal(P.round_bf16(x), torch.from_numpy(x).to(torch.bfloat16).double().numpy())
    assert np.array_equal(P.round_f16(x * 100), (x * 100).astype(np.float16).astype(np.float64))
    y = np.clip(x * 10, -448, 448)  # the library's E4M3 conversion does not saturate
    assert np.array_equal(P.round_e4m3(y),
                          torch.from_numpy(y).to(torch.float8_e4m3fn).double().numpy())


def test_scales():
    X = np.array([[0.5, -3.0], [2.0, 1.0]], np.float32)
    assert P.operand_scale(X, P.E4M3) == np.float32(448.0) / np.float32(3.0)
    s = P.operand_scale(X, P.F16)
    assert s == 2.0 ** 12 and 2.0 ** 13 <= 3.0 * s < 2.0 ** 14
    assert P.operand_scale(X, P.BF16) == 1.0


@pytest.mark.parametrize("form", [P.BF16, P.F16, P.E4M3])
def test_screening_that_keeps_every_member_is_the_exact_knn(form):
    X = datagen.gaussian_mixture_f32(600, 24, 4, 2.0, seed=11)
    a = oracle.assign(X, X[:3].astype(np.float32), 2)
    mem, off = oracle.shards(a, 3)
    rows = np.arange(0, len(mem), 7)
    big = int(np.diff(off).max())
    _, _, rid, rdist = P.screen_rows(X, mem, off, form, big, 10, rows)
    oid, od = oracle.shard_knn(X, mem, off, 10, rows=rows)
    assert np.array_equal(rid, oid)
    assert np.allclose(rdist, od, rtol=1e-12, atol=0)  # summation order only


def test_bf16_screening_of_integer_data_is_exact():
    X = datagen.clustered_u8(800, 32, 6, seed=12).astype(np.float32)
    a = oracle.assign(X, X[:2].astype(np.float32), 1)
    mem, off = oracle.shards(a, 2)
    rows = np.arange(0, len(mem), 5)
    sid, sdist, rid, rdist = P.screen_rows(X, mem, off, P.BF16, 16, 16, rows)
    oid, od = oracle.shard_knn(X, mem, off, 16, rows=rows)
    assert np.array_equal(sid, oid) and np.array_equal(rid, oid)
    assert np.array_equal(sdist, od)  # integer keys: the screening distance is exact
    mx, mean = P.distance_error_rows(X, mem[rows], sid, sdist)
    assert mx == 0.0 and mean == 0.0


def test_e4m3_screening_error_is_within_the_rounding_bound():
    """Each E4M3 operand is within 2^-4 relative of its scaled value, so a
    screening distance is off by at most about 2 * 2^-4 * |s u| |s v| / s^2 plus
    the norm term's rounding: check the observed errors against that bound."""
    X = datagen.anisotropic_mixture(500, 32, 4, 0.25, True, np.float32, seed=13)
    a = oracle.assign(X, X[:2].astype(np.float32), 1)
    mem, off = oracle.shards(a, 2)
    rows = np.arange(0, len(mem), 9)
    sid, sdist, _, _ = P.screen_rows(X, mem, off, P.E4M3, 20, 10, rows)
    Xd = X.astype(np.float64)
    for r, p in enumerate(rows):
        u = int(mem[p])
        ok = sid[r] != oracle.PAD
        c = sid[r][ok].astype(np.int64)
        de = ((Xd[c] - Xd[u]) ** 2).sum(1)
        bound = 2 * (2.0 ** -4 + 2.0 ** -8) * np.linalg.norm(Xd[u]) * np.linalg.norm(Xd[c], axis=1)
        assert np.all(np.abs(sdist[r][ok] - de) <= bound + 1e-12)
