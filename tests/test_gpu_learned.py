"""Learned candidate form on the GPU (through the C-ABI) against the FP64 oracle.

The MLP runs in FP32 on the GPU and in FP64 in the oracle, so embeddings and
training trajectories are compared within tolerances derived from FP32
rounding; the learned kNN lists are compared through what is unique: exact
distances of every returned id, the list order, and - with a model that makes
the embedding the identity - bit-exact equality with the exact shard kNN.
"""
import numpy as np
import pytest
import torch

import oracle
from oracle import learned as OL
from paper_2605_10135_gb300 import ann, build, datagen
from tests.parity import as_u32

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


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


def _fp16_operands(X, p):
    """What the tensor-core layer 1 multiplies: FP16(x * (1 / max|x|)) and FP16(W1)."""
    d = X.shape[1]
    inv = np.float32(1.0) / np.float32(np.abs(X.astype(np.float32)).max())
    xs = (X.astype(np.float32) * inv).astype(np.float16).astype(np.float64)
    q = np.asarray(p, dtype=np.float64).copy()
    q[:OL.HIDDEN * d] = np.asarray(p[:OL.HIDDEN * d], dtype=np.float32).astype(np.float16)
    return xs, q


@pytest.mark.parametrize("kind,d", [("f32", 96), ("u8", 64), ("f16", 1000)])
def test_embedding_matches_oracle(kind, d):
    """Layer 1 on the tensor cores (FP16 operands, FP32 accumulation), layer 2 in
    FP32: against the FP64 forward pass of the same FP16-rounded operands."""
    if kind == "f32":
        X = datagen.anisotropic_mixture(5000, d, 32, 0.25, True, np.float32, seed=61)
    elif kind == "u8":
        X = datagen.clustered_u8(70000, d, 64, seed=62)   # more than one 65536-row chunk
    else:
        X = datagen.anisotropic_mixture(3000, d, 16, 0.25, False, np.float16, seed=64)
    p = datagen.mlp_init(X.shape[1], seed=63)
    E = ann.learned_embed(T(X), T(p)).cpu().numpy().astype(np.float64)
    xs, q = _fp16_operands(X, p)
    ref = OL.forward(q, xs, X.shape[1])[2]
    # FP32 sums of d + 256 products: error well below 1e-4 of the embedding scale
    assert np.abs(E - ref).max() <= 1e-4 * np.abs(ref).max()
    # and the FP16 rounding itself moves the embedding by well under 1% of its scale
    assert np.abs(E - OL.embed(X, p)).max() <= 1e-2 * np.abs(ref).max()


def _train_case(steps, batch, seed):
    X = datagen.gaussian_mixture_f32(4000, 32, 8, 3.0, seed=seed)
    sample = datagen.row_sample(4000, 0.02, 64, seed=seed + 1)
    draws = datagen.triplet_draws(steps, batch, seed=seed + 2)
    p0 = datagen.mlp_init(32, seed=seed + 3)
    return X, sample, draws, p0


def test_training_steps_match_oracle():
    """Three Adam steps: the per-step losses agree to FP32 rounding, and the
    parameters agree except where a gradient component is so close to zero that
    its FP32 and FP64 signs differ (Adam's first steps move every parameter by
    about lr, whatever the gradient's size)."""
    X, sample, draws, p0 = _train_case(3, 256, 71)
    lr, margin, kk, kpos = 1e-3, 1e-3, 40, 10
    p = T(p0.copy())
    losses, _ = ann.learned_train(T(X), T(sample), T(draws), p, kk, kpos, lr, margin,
                                  estimate=False)
    knn = OL.sample_knn(X, sample, kk)
    ref_p, ref_l = OL.train(X, sample, knn, draws, lr, margin, p0, kpos)
    got_l = losses.cpu().numpy().astype(np.float64)
    assert np.allclose(got_l, ref_l, rtol=1e-4, atol=1e-7)
    dp = np.abs(p.cpu().numpy().astype(np.float64) - ref_p)
    assert dp.max() <= 2 * 3 * lr + 1e-6
    assert (dp > 1e-5).mean() < 0.01


def test_training_lowers_loss_and_estimates_recall():
    X, sample, draws, p0 = _train_case(300, 256, 81)
    p = T(p0.copy())
    losses, est = ann.learned_train(T(X), T(sample), T(draws), p, 40, 10, 1e-3, 1e-3)
    l = losses.cpu().numpy()
    assert np.isfinite(l).all()
    assert l[-30:].mean() < 0.5 * l[:5].mean()
    e = float(est.item())
    assert 0.5 < e <= 1.0


def _identity_params(d):
    W1 = np.zeros((OL.HIDDEN, d)); b1 = np.zeros(OL.HIDDEN)
    W1[:d] = np.eye(d); W1[d:2 * d] = -np.eye(d)
    W2 = np.zeros((OL.OUT, OL.HIDDEN)); b2 = np.zeros(OL.OUT)
    W2[:d, :d] = np.eye(d); W2[:d, d:2 * d] = -np.eye(d)
    return OL.pack(W1, b1, W2, b2).astype(np.float32)


def _shards(X, C, r, seed):
    sample, init_rows = datagen.kmeans_sample(X.shape[0], C, seed)
    cent, _ = oracle.kmeans(X, X[init_rows].astype(np.float32), sample, 4)
    return oracle.shards(oracle.assign(X, cent, r), C)


def test_identity_model_gives_the_exact_shard_knn():
    """f(x) = x / s: candidates in embedding space are the exact candidates up to
    the rounding of x / s and of the FP16 screening, which only reorders near-ties;
    a screened list of 64 for k = 16 leaves the re-rank the exact answer."""
    X = datagen.clustered_u8(5000, 32, 24, sigma=8.0, seed=91)
    mem, off = _shards(X, 3, 2, seed=92)
    p = _identity_params(32)
    gid, gd = ann.shard_knn(T(X), T(mem), T(off), 16, precision=ann.LEARNED, rerank_k=64,
                            model=T(p))
    oid, od = oracle.shard_knn(X, mem, off, 16)
    assert np.array_equal(as_u32(gid), oid)
    assert np.array_equal(gd.cpu().numpy().astype(np.float64), od)


def test_trained_model_lists_are_exactly_scored_and_close_to_the_oracle():
    X, sample, draws, p0 = _train_case(200, 256, 101)
    p = T(p0.copy())
    ann.learned_train(T(X), T(sample), T(draws), p, 40, 10, 1e-3, 1e-3, estimate=False)
    pt = p.cpu().numpy()
    mem, off = _shards(X, 3, 2, seed=102)
    k, kp = 16, 64
    gid, gd = ann.shard_knn(T(X), T(mem), T(off), k, precision=ann.LEARNED, rerank_k=kp,
                            model=T(pt))
    gid, gd = as_u32(gid), gd.cpu().numpy().astype(np.float64)
    # every returned id carries its exact distance (FP32 direct form) and lists are sorted
    Xd = X.astype(np.float64)
    rows = np.arange(0, len(mem), 37)
    for r in rows:
        u = int(mem[r])
        ids = gid[r]
        ex = ((Xd[ids.astype(np.int64)] - Xd[u]) ** 2).sum(1)
        assert np.allclose(gd[r], ex, rtol=1e-5, atol=0)
        key = list(zip(gd[r], ids))
        assert key == sorted(key)
    # the same model in the oracle (FP64 screening) proposes nearly the same lists
    oid, _ = OL.learned_shard_knn(X, mem, off, pt, k, kp)
    assert oracle.recall_at(gid[rows], oid[rows], k) > 0.98
    # and both find the same share of the exact graph (the model's own quality)
    eid, _ = oracle.shard_knn(X, mem, off, 10, rows=rows)
    r_gpu = oracle.recall_at(gid[rows], eid, 10)
    r_or = oracle.recall_at(oid[rows], eid, 10)
    assert abs(r_gpu - r_or) <= 0.02 and r_gpu > 0.7


def test_learned_without_model_is_the_exact_form():
    X = datagen.clustered_u8(3000, 64, 16, seed=111)
    mem, off = _shards(X, 3, 2, seed=112)
    gid, gd = ann.shard_knn(T(X), T(mem), T(off), 12, precision=ann.LEARNED)
    eid, ed = ann.shard_knn(T(X), T(mem), T(off), 12)
    assert torch.equal(gid, eid) and torch.equal(gd, ed)
