"""Pins of the FP64 learned-form oracle against facts that do not come from it:
finite differences, closed forms, a hand-worked example, an identity model that
reduces the learned form to the exact shard kNN, and scipy's exact kNN."""
import numpy as np
import pytest

import oracle
from oracle import learned as L
from paper_2605_10135_gb300 import datagen


def _rand_params(d, seed, scale=0.3):
    rng = np.random.default_rng(seed)
    return rng.normal(0.0, scale, size=L.n_params(d))


def test_gradient_matches_central_differences():
    """The analytic gradient against (L(p + h e_i) - L(p - h e_i)) / 2h, at a point
    where no pre-activation or hinge lies within reach of the step."""
    d, B, margin = 5, 4, 0.5
    rng = np.random.default_rng(7)
    for attempt in range(50):
        p = _rand_params(d, 100 + attempt)
        Xa, Xp, Xn = (rng.uniform(-1, 1, size=(B, d)) for _ in range(3))
        U = L.forward(p, np.concatenate([Xa, Xp, Xn]), d)[0]
        _, g, hinge = L.loss_and_grads(p, Xa, Xp, Xn, margin, d)
        if np.abs(U).min() > 1e-3 and np.abs(hinge).min() > 1e-3 and (hinge > 0).any():
            break
    else:
        pytest.fail("no smooth point found")
    h = 1e-6
    num = np.empty_like(p)
    for i in range(p.size):
        e = np.zeros_like(p)
        e[i] = h
        num[i] = (L.loss_and_grads(p + e, Xa, Xp, Xn, margin, d)[0]
                  - L.loss_and_grads(p - e, Xa, Xp, Xn, margin, d)[0]) / (2 * h)
    assert np.allclose(g, num, rtol=1e-5, atol=1e-7)  # atol: cancellation in the quotient


def test_forward_hand_worked_example():
    """d = 2, hidden unit 0 = relu(x0 - x1 + 0.5), unit 1 = relu(-x0), others 0;
    z0 = 2 h0 - h1 + 1, z1 = h1, other outputs 0."""
    d = 2
    W1 = np.zeros((L.HIDDEN, d)); b1 = np.zeros(L.HIDDEN)
    W1[0] = [1.0, -1.0]; b1[0] = 0.5
    W1[1] = [-1.0, 0.0]
    W2 = np.zeros((L.OUT, L.HIDDEN)); b2 = np.zeros(L.OUT)
    W2[0, 0] = 2.0; W2[0, 1] = -1.0; b2[0] = 1.0
    W2[1, 1] = 1.0
    p = L.pack(W1, b1, W2, b2)
    X = np.array([[0.25, 0.5], [-0.5, 0.25]])
    Z = L.forward(p, X, d)[2]
    # row 0: h0 = relu(0.25) = 0.25, h1 = 0 -> z0 = 1.5, z1 = 0
    # row 1: h0 = relu(-0.25) = 0, h1 = 0.5 -> z0 = 0.5, z1 = 0.5
    assert np.allclose(Z[:, :2], [[1.5, 0.0], [0.5, 0.5]], atol=0, rtol=0)
    assert not Z[:, 2:].any()


def test_loss_is_zero_when_every_margin_is_met():
    d = 3
    p = np.zeros(L.n_params(d))
    W1, b1, W2, b2 = L.unpack(p, d)
    W1 = W1.copy(); W2 = W2.copy()
    W1[:3] = np.eye(3); W1[3:6] = -np.eye(3)
    W2[:3, :3] = np.eye(3); W2[:3, 3:6] = -np.eye(3)   # identity embedding
    p = L.pack(W1, b1, W2, b2)
    Xa = np.zeros((2, 3)); Xp = np.full((2, 3), 0.1); Xn = np.ones((2, 3))
    loss, g, hinge = L.loss_and_grads(p, Xa, Xp, Xn, 0.5, d)
    assert loss == 0.0 and not g.any()
    assert np.allclose(hinge, 3 * 0.01 - 3 + 0.5)


def test_adam_closed_form():
    """Under a constant gradient g the bias-corrected moments equal g and g^2
    exactly, so every step moves each parameter by lr * g / (|g| + eps)."""
    p0 = np.array([1.0, -2.0, 0.5])
    g = np.array([0.3, -4.0, 1e-3])
    m = np.zeros(3); v = np.zeros(3)
    p = p0.copy()
    lr = 0.01
    for t in range(1, 6):
        p, m, v = L.adam(p, g, m, v, t, lr)
    step = lr * g / (np.abs(g) + L.EPS)
    assert np.allclose(p, p0 - 5 * step, rtol=1e-12, atol=1e-12)


def _identity_params(d):
    W1 = np.zeros((L.HIDDEN, d)); b1 = np.zeros(L.HIDDEN)
    W1[:d] = np.eye(d); W1[d:2 * d] = -np.eye(d)
    W2 = np.zeros((L.OUT, L.HIDDEN)); b2 = np.zeros(L.OUT)
    W2[:d, :d] = np.eye(d); W2[:d, d:2 * d] = -np.eye(d)
    return L.pack(W1, b1, W2, b2)


def test_identity_model_reduces_to_exact_shard_knn():
    """With f(x) = x / s (d <= 32) the embedding order is the exact order up to the
    rounding of x / s, which can only reorder exact ties; with kprime well above k
    the re-rank restores them, so the learned form returns exactly the exact shard
    kNN (ties by id on both sides)."""
    X = datagen.clustered_u8(600, 24, 8, sigma=6.0, seed=31)
    cent = X[:3].astype(np.float32)
    a = oracle.assign(X, cent, 2)
    mem, off = oracle.shards(a, 3)
    p = _identity_params(24)
    assert np.allclose(L.embed(X, p)[:, :24], X / L.input_scale(X))
    lid, ld = L.learned_shard_knn(X, mem, off, p, 10, 40)
    eid, ed = oracle.shard_knn(X, mem, off, 10)
    assert np.array_equal(lid, eid)
    assert np.array_equal(ld, ed)


def test_sample_knn_matches_scipy():
    from scipy.spatial import cKDTree
    X = datagen.gaussian_mixture_f32(2000, 8, 4, seed=5)
    sample = np.array([3, 50, 777, 1999], dtype=np.uint32)
    got = L.sample_knn(X, sample, 6)
    _, ref = cKDTree(X.astype(np.float64)).query(X[sample].astype(np.float64), k=7)
    for j, a in enumerate(sample):
        assert set(got[j].tolist()) == set(int(v) for v in ref[j] if v != a)


def test_triplets_follow_the_draws():
    sample = np.array([10, 20, 30], dtype=np.uint32)
    knn = np.array([[1, 2, 7, 8, 9], [3, 4, 11, 12, 13], [5, 6, 14, 15, 16]], dtype=np.uint32)
    # kpos = 2: positive = knn[j, r1 % 2]; even r2 -> knn[j, 2 + (r2 >> 1) % 3],
    # odd r2 -> row (r2 >> 1) % N
    draws = np.array([[4, 3, 2015], [2, 0, 10]], dtype=np.uint32)
    a, p, n = L.triplets(sample, knn, draws, 1000, 2)
    assert a.tolist() == [20, 30] and p.tolist() == [4, 5]
    assert n.tolist() == [7, 16]    # 2015 odd: 1007 % 1000; 10 even: knn[2, 2 + 5 % 3]


def test_training_lowers_the_loss_and_finds_neighbours():
    N = 3000
    X = datagen.gaussian_mixture_f32(N, 16, 8, 3.0, seed=9)
    rng = np.random.default_rng(3)
    sample = np.sort(rng.choice(N, 100, replace=False)).astype(np.uint32)
    knn = L.sample_knn(X, sample, 40)
    draws = datagen.triplet_draws(400, 64, seed=5)
    p0 = datagen.mlp_init(16, seed=4)
    p, losses = L.train(X, sample, knn, draws, 1e-3, 1e-3, p0, 10)
    assert losses[-20:].mean() < 0.5 * losses[:5].mean()
    mem = np.arange(N, dtype=np.uint32)
    off = np.array([0, N], dtype=np.int64)
    rows = np.arange(0, N, 60)
    eid, _ = oracle.shard_knn(X, mem, off, 10, rows=rows)
    lid0, _ = L.learned_shard_knn(X, mem, off, p0, 10, 40)
    lid, _ = L.learned_shard_knn(X, mem, off, p, 10, 40)
    r0 = oracle.recall_at(lid0[rows], eid, 10)
    r1 = oracle.recall_at(lid[rows], eid, 10)
    assert r1 > r0 and r1 > 0.9
