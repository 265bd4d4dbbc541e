"""Learned candidate form on the GPU (through the C-ABI) against the FP64 oracle.

The MLP's layer 1 runs on the tensor cores (FP16 operands for the embedding,
split BF16 operands for the training step, FP32 accumulation), the rest in
FP32; the oracle is FP64.  Embeddings, gradients and training trajectories are
compared within tolerances derived from those roundings, the embedding against
the oracle on the same rounded operands; the learned kNN lists are compared
through what is unique: exact
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


# Layer 1 of the training step runs on the tensor cores with each FP32 operand
# (x / s, W1, dU) split into two BF16 parts, hi + lo, and three products (hi.hi +
# lo.hi + hi.lo): each product is within about 2^-16 of its FP32 value.  The
# triplet gradients cancel (anchor, positive and negative terms of opposite sign),
# which can raise a tensor's relative error by an order of magnitude; 1e-2 of each
# tensor's norm leaves a wide margin, and the loss agrees to 1e-4.
GRAD_RTOL = 1e-2


@pytest.mark.parametrize("kind,d,B", [("f32", 48, 256), ("u8", 128, 100), ("f16", 300, 64)])
def test_batch_gradient_matches_the_oracle(kind, d, B):
    """ann_learned_grad (the training step's loss and gradient kernels) against the
    FP64 loss_and_grads of the oracle on the same triplets, per parameter tensor:
    |g - g64| / |g64| for W1, b1, W2, b2."""
    rng = np.random.default_rng(71)
    n = 3000
    if kind == "f32":
        X = datagen.gaussian_mixture_f32(n, d, 8, 3.0, seed=72)
    elif kind == "u8":
        X = datagen.clustered_u8(n, d, 8, seed=73)
    else:
        X = datagen.anisotropic_mixture(n, d, 8, 0.25, False, np.float16, seed=74)
    p = datagen.mlp_init(d, seed=75)
    rows = rng.integers(0, n, size=3 * B).astype(np.uint32)
    margin = 0.05
    g, loss = ann.learned_grad(T(X), T(p), T(rows), margin)
    g = g.cpu().numpy().astype(np.float64)
    Xs = X.astype(np.float64) / OL.input_scale(X)
    a, pp, ng = rows[:B], rows[B:2 * B], rows[2 * B:]
    l64, g64, hinge = OL.loss_and_grads(p, Xs[a], Xs[pp], Xs[ng], margin, d)
    assert (hinge > 0).sum() > B // 4  # a batch with active and inactive triplets
    assert abs(float(loss.item()) - l64) <= 1e-4 * abs(l64)
    o = 0
    for name, size in (("W1", OL.HIDDEN * d), ("b1", OL.HIDDEN), ("W2", OL.OUT * OL.HIDDEN),
                       ("b2", OL.OUT)):
        got, ref = g[o:o + size], g64[o:o + size]
        o += size
        if name == "b2":
            # each triplet adds c (zn - zp) + c (zp - za) + c (za - zn) = 0: the exact
            # b2 gradient vanishes, so only rounding remains, small against the rest
            assert np.linalg.norm(ref) <= 1e-12 * np.linalg.norm(g64)
            assert np.linalg.norm(got) <= GRAD_RTOL * np.linalg.norm(g64), name
            continue
        err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        assert err <= GRAD_RTOL, (name, err)


def test_batch_gradient_is_zero_when_every_margin_holds():
    """Negatives far beyond their positives and a zero margin: no hinge is active,
    so the loss and every gradient entry are exactly zero."""
    X = np.zeros((40, 16), np.float32)
    X[20:] = 50.0
    p = datagen.mlp_init(16, seed=76)
    B = 10
    rows = np.concatenate([np.arange(10), np.arange(10), np.arange(20, 30)]).astype(np.uint32)
    g, loss = ann.learned_grad(T(X), T(p), T(rows), 0.0)
    if float(loss.item()) == 0.0:
        assert not torch.any(g != 0)
    else:  # the random model may not separate the groups; the oracle decides
        Xs = X.astype(np.float64) / OL.input_scale(X)
        l64, _, hinge = OL.loss_and_grads(p, Xs[rows[:B]], Xs[rows[B:2 * B]], Xs[rows[2 * B:]],
                                          0.0, 16)
        assert l64 > 0


def _train_case(steps, batch, seed):
    X = datagen.gaussian_mixture_f32(4000, 32, 8, 3.0, seed=seed)
    sample = datagen.row_sample(4000, 0.02, 64, seed=seed + 1)
    draws = datagen.triplet_draws(steps, batch, seed=seed + 2)
    p0 = datagen.mlp_init(32, seed=seed + 3)
    return X, sample, draws, p0


def test_training_steps_match_oracle():
    """Three Adam steps: the per-step losses agree to the rounding of layer 1's
    split BF16 products (well under 1e-3), and the parameters agree except where a
    gradient component is so close to zero that its rounded and FP64 signs differ
    (Adam's first steps move every parameter by about lr, whatever the gradient's
    size).  The gradients themselves are compared in
    test_batch_gradient_matches_the_oracle."""
    X, sample, draws, p0 = _train_case(3, 256, 71)
    lr, margin, kk, kpos = 1e-3, 1e-3, 40, 10
    p = T(p0.copy())
    losses, _ = ann.learned_train(T(X), T(sample), T(draws), p, kk, kpos, lr, margin,
                                  estimate=False)
    knn = OL.sample_knn(X, sample, kk)
    ref_p, ref_l = OL.train(X, sample, knn, draws, lr, margin, p0, kpos)
    got_l = losses.cpu().numpy().astype(np.float64)
    assert np.allclose(got_l, ref_l, rtol=1e-3, atol=1e-7)
    dp = np.abs(p.cpu().numpy().astype(np.float64) - ref_p)
    assert dp.max() <= 2 * 3 * lr + 1e-6
    assert (dp > 1e-5).mean() < 0.05


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
