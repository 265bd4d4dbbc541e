"""Exact pruning of distance tiles (uint8, ANN_EXACT): the pruned sweep returns
the same kNN lists as the full sweep, bit for bit, on clustered data where most
far tiles are skipped, on data with many duplicate vectors and ties, and against
the oracle."""
import numpy as np
import pytest
import torch

import oracle
from paper_2605_10135_gb300 import ann, build, datagen
from tests.parity import as_u32

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    ann.lib()
    ann.device_status()
    ann.tile_prune(True)
    yield
    ann.tile_prune(True)
    assert ann.device_status() == 0


def _shards(X, C, seed):
    sample, init_rows = datagen.kmeans_sample(X.shape[0], C, seed)
    init = torch.from_numpy(X[init_rows].astype(np.float32)).to(DEV)
    samp = torch.from_numpy(sample.view(np.int32)).to(DEV)
    _, mem, off = ann.partition(torch.from_numpy(X).to(DEV), C, min(2, C), init, samp, 4)
    return mem, off


def _both(X, mem, off, k):
    Xd = torch.from_numpy(X).to(DEV)
    ann.tile_prune(False)
    a = ann.shard_knn(Xd, mem, off, k)
    torch.cuda.synchronize()
    ann.tile_prune_stats()
    ann.tile_prune(True)
    b = ann.shard_knn(Xd, mem, off, k)
    st = ann.tile_prune_stats()
    return a, b, st


@pytest.mark.parametrize("n,d,centres,C,k,expect", [(40000, 128, 16, 1, 64, 0.8),
                                                   (30000, 64, 96, 2, 32, None),
                                                   (20000, 128, 48, 3, 64, None),
                                                   (9001, 32, 12, 1, 16, None)])
def test_pruned_sweep_equals_full_sweep(n, d, centres, C, k, expect):
    X = datagen.clustered_u8(n, d, centres, seed=400 + d)
    mem, off = _shards(X, C, 401)
    (ia, da), (ib, db), st = _both(X, mem, off, k)
    assert torch.equal(ia, ib) and torch.equal(da, db)
    assert 0 < st["swept"] <= st["tiles"]
    if expect is not None:  # clusters of thousands of rows: most far tiles are skipped
        assert st["swept"] < expect * st["tiles"]


def test_pruned_sweep_with_duplicates_and_ties():
    """Few distinct vectors: many columns at exactly the k-th distance."""
    rng = np.random.default_rng(411)
    base = rng.integers(0, 256, size=(60, 48)).astype(np.uint8)
    X = np.repeat(base, 150, axis=0)
    X[::7, 0] ^= 1  # some near-duplicates one unit away
    X = X[rng.permutation(len(X))]
    mem, off = _shards(X, 2, 412)
    (ia, da), (ib, db), st = _both(X, mem, off, 24)
    assert torch.equal(ia, ib) and torch.equal(da, db)


def test_pruned_sweep_matches_the_oracle():
    X = datagen.clustered_u8(16000, 96, 8, seed=421)
    mem, off = _shards(X, 2, 422)
    Xd = torch.from_numpy(X).to(DEV)
    ann.tile_prune(True)
    ids, ds = ann.shard_knn(Xd, mem, off, 32)
    ann.tile_prune_stats()
    m, o = as_u32(mem), off.cpu().numpy()
    rows = np.random.default_rng(423).choice(len(m), 400, replace=False)
    oid, od = oracle.shard_knn(X, m, o, 32, rows=rows)
    assert np.array_equal(as_u32(ids)[rows], oid)
    assert np.array_equal(ds.cpu().numpy()[rows].astype(np.float64), od)


@pytest.mark.parametrize("kind", ["deep", "gauss"])
def test_float_pruned_sweep_equals_full_sweep(kind):
    """FP32 data (split BF16 keys, screened list re-ranked in FP32): the skipping
    keeps a margin for the key error, so the lists equal the full sweep's."""
    if kind == "deep":
        X = datagen.anisotropic_mixture(30000, 96, 16, 0.25, True, np.float32, seed=431)
    else:
        X = datagen.gaussian_mixture_f32(30000, 64, 12, 6.0, seed=432)
    mem, off = _shards(X, 2, 433)
    (ia, da), (ib, db), st = _both(X, mem, off, 32)
    assert torch.equal(ia, ib) and torch.equal(da, db)
    assert 0 < st["swept"] <= st["tiles"]


@pytest.mark.parametrize("prec", [ann.BF16_RERANK, ann.F16_RERANK])
@pytest.mark.parametrize("kind", ["deep", "gauss"])
def test_screening_forms_pruned_sweep_equals_full_sweep(kind, prec):
    """The BF16 and scaled FP16 screening forms skip tiles too, with the margin of
    their own key error (one rounding of each operand): the screened lists, and so
    the re-ranked ones, equal the full sweep's bit for bit."""
    if kind == "deep":
        X = datagen.anisotropic_mixture(30000, 96, 16, 0.25, True, np.float32, seed=441)
    else:
        X = datagen.gaussian_mixture_f32(30000, 64, 12, 6.0, seed=442)
    mem, off = _shards(X, 2, 443)
    Xd = torch.from_numpy(X).to(DEV)
    ann.tile_prune(False)
    sa = ann.shard_knn_screen(Xd, mem, off, 32, prec, 96)
    a = ann.shard_knn(Xd, mem, off, 32, precision=prec, rerank_k=96)
    torch.cuda.synchronize()
    ann.tile_prune_stats()
    ann.tile_prune(True)
    sb = ann.shard_knn_screen(Xd, mem, off, 32, prec, 96)
    b = ann.shard_knn(Xd, mem, off, 32, precision=prec, rerank_k=96)
    st = ann.tile_prune_stats()
    assert torch.equal(sa[0], sb[0]) and torch.equal(sa[1], sb[1])
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])
    assert 0 < st["swept"] < st["tiles"]
