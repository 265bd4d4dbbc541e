"""FP64 oracle of the learned candidate form (TEST INFRASTRUCTURE ONLY).

Only the tests, the smoke check and the CPU-baseline leg of the benchmark import
this module.  It shares no code with the CUDA library.

The paper builds every shard graph with an exact-distance graph builder
(Sec. II-B, Sec. IV Workflow (2)); it has no learned component.  The learned
form is an addition beside the method: a small MLP maps every vector to 32
dimensions, the nearest rows in that space are proposed as candidates, and the
candidates are re-ranked with exact distances in the original space.  This file
is its definition, written out plainly:

* model      f(x) = W2 relu(W1 (x / s) + b1) + b2, W1 [256 x d], W2 [32 x 256];
             s = max |x| over all vectors (one scalar that brings every input
             into [-1, 1]).  Parameters are one flat float array
             [W1 (row-major) | b1 | W2 (row-major) | b2].
* training   triplet margin loss over (anchor, positive, negative):
             L = (1/B) sum_i max(0, |f(a)-f(p)|^2 - |f(a)-f(n)|^2 + margin),
             anchors from a seeded sample of the vectors; with L the anchor's
             exact kk nearest vectors (all N, itself excluded, by (distance,
             id)), the positive is L[r1 mod kpos] and the negative is, for an
             even r2, the near miss L[kpos + (r2 >> 1) mod (kk - kpos)], for an
             odd r2 the uniform row (r2 >> 1) mod N.  The random picks are
             inputs (draws[t, i] = three uint32: anchor slot, r1, r2).
* optimiser  Adam (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected), the
             parameters updated once per step.
* proposal   per shard row: the kprime members nearest in embedding space
             (ties to the smaller id), re-ranked by exact squared distance in
             the original space (ties to the smaller id), first k kept.
"""
from __future__ import annotations

import numpy as np

from . import oracle as _o

HIDDEN = 256
OUT = 32
BETA1, BETA2, EPS = 0.9, 0.999, 1e-8


def n_params(d: int) -> int:
    return HIDDEN * d + HIDDEN + OUT * HIDDEN + OUT


def unpack(params: np.ndarray, d: int):
    p = np.asarray(params, dtype=np.float64)
    o = 0
    W1 = p[o:o + HIDDEN * d].reshape(HIDDEN, d); o += HIDDEN * d
    b1 = p[o:o + HIDDEN]; o += HIDDEN
    W2 = p[o:o + OUT * HIDDEN].reshape(OUT, HIDDEN); o += OUT * HIDDEN
    b2 = p[o:o + OUT]
    return W1, b1, W2, b2


def pack(W1, b1, W2, b2) -> np.ndarray:
    return np.concatenate([W1.ravel(), b1.ravel(), W2.ravel(), b2.ravel()])


def input_scale(X: np.ndarray) -> float:
    s = float(np.abs(X.astype(np.float64)).max()) if X.size else 0.0
    return s if s > 0.0 else 1.0


def forward(params, Xs: np.ndarray, d: int):
    """Xs: inputs already divided by s.  Returns (U, H, Z): pre-activations,
    hidden activations and embeddings."""
    W1, b1, W2, b2 = unpack(params, d)
    U = Xs @ W1.T + b1
    H = np.maximum(U, 0.0)
    Z = H @ W2.T + b2
    return U, H, Z


def loss_and_grads(params, Xa, Xp, Xn, margin: float, d: int):
    """Triplet margin loss of one batch and its gradient (same layout as params)."""
    W1, b1, W2, b2 = unpack(params, d)
    B = Xa.shape[0]
    X = np.concatenate([Xa, Xp, Xn])
    U, H, Z = forward(params, X, d)
    za, zp, zn = Z[:B], Z[B:2 * B], Z[2 * B:]
    dp = ((za - zp) ** 2).sum(1)
    dn = ((za - zn) ** 2).sum(1)
    hinge = dp - dn + margin
    act = (hinge > 0.0).astype(np.float64)
    loss = float((hinge * act).sum() / B)
    c = (2.0 / B) * act[:, None]
    dZ = np.concatenate([c * (zn - zp), c * (zp - za), c * (za - zn)])
    dW2 = dZ.T @ H
    db2 = dZ.sum(0)
    dH = dZ @ W2
    dU = dH * (U > 0.0)
    dW1 = dU.T @ X
    db1 = dU.sum(0)
    return loss, pack(dW1, db1, dW2, db2), hinge


def adam(params, grads, m, v, t: int, lr: float):
    """One bias-corrected Adam step (t counts from 1)."""
    m = BETA1 * m + (1.0 - BETA1) * grads
    v = BETA2 * v + (1.0 - BETA2) * grads * grads
    mh = m / (1.0 - BETA1 ** t)
    vh = v / (1.0 - BETA2 ** t)
    return params - lr * mh / (np.sqrt(vh) + EPS), m, v


def sample_knn(X: np.ndarray, sample: np.ndarray, kk: int) -> np.ndarray:
    """Exact kk nearest vectors (all N, by (distance, id)) of each sampled row,
    the row itself excluded."""
    ids, _ = _o.bruteforce(X, X[sample], kk + 1)
    out = np.empty((len(sample), kk), dtype=np.uint32)
    for j, a in enumerate(sample):
        row = [int(v) for v in ids[j] if int(v) != int(a)]
        out[j] = row[:kk]
    return out


def triplets(sample, knn, draws_t, N: int, kpos: int):
    """(anchor, positive, negative) row ids of one step from its draws [B, 3]."""
    S, kk = knn.shape
    j = draws_t[:, 0].astype(np.int64) % S
    a = sample[j].astype(np.int64)
    p = knn[j, draws_t[:, 1].astype(np.int64) % kpos].astype(np.int64)
    r2 = draws_t[:, 2].astype(np.int64)
    near = knn[j, kpos + (r2 >> 1) % (kk - kpos)].astype(np.int64)
    n = np.where(r2 & 1, (r2 >> 1) % N, near)
    return a, p, n


def train(X, sample, knn, draws, lr: float, margin: float, params0, kpos: int):
    """Adam on the triplet loss, one step per draws[t]; returns (params, losses)."""
    d = X.shape[1]
    Xs = X.astype(np.float64) / input_scale(X)
    p = np.asarray(params0, dtype=np.float64).copy()
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    losses = []
    for t in range(draws.shape[0]):
        a, pp, n = triplets(sample, knn, draws[t], X.shape[0], kpos)
        loss, g, _ = loss_and_grads(p, Xs[a], Xs[pp], Xs[n], margin, d)
        p, m, v = adam(p, g, m, v, t + 1, lr)
        losses.append(loss)
    return p, np.array(losses)


def embed(X, params) -> np.ndarray:
    d = X.shape[1]
    return forward(params, X.astype(np.float64) / input_scale(X), d)[2]


def learned_shard_knn(X, members, offsets, params, k: int, kprime: int):
    """Per shard row: kprime nearest members in embedding space (ties to the
    smaller id), re-ranked by exact squared distance, first k (PAD / inf after)."""
    E = embed(X, params)
    Xd = X.astype(np.float64)
    rows = int(offsets[-1])
    out_id = np.full((rows, k), _o.PAD, dtype=np.uint32)
    out_d = np.full((rows, k), np.inf, dtype=np.float64)
    for s in range(len(offsets) - 1):
        mem = members[offsets[s]:offsets[s + 1]].astype(np.int64)
        if len(mem) == 0:
            continue
        Es = E[mem]
        for li, u in enumerate(mem):
            de = ((Es - E[u]) ** 2).sum(1)
            order = np.lexsort((mem, de))
            cand = [int(mem[q]) for q in order if int(mem[q]) != int(u)][:kprime]
            dx = [(float(((Xd[c] - Xd[u]) ** 2).sum()), c) for c in cand]
            dx.sort()
            for e, (dd, c) in enumerate(dx[:k]):
                out_id[offsets[s] + li, e] = c
                out_d[offsets[s] + li, e] = dd
    return out_id, out_d
