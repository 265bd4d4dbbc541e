"""Seeded synthetic inputs shaped like the paper's workloads (Table 3 datasets).

This module holds no arithmetic of the indexing method itself: it only draws
vectors, query sets, the k-means sample and the k-means initial centroids.
Both the CPU oracle tests and the CUDA path take their inputs from here, so the
two sides always see bit-identical arrays.

The paper's datasets (Sift100M u8 d=128, Deep100M f32 d=96, Laion100M f32
d=768; Table 3) are not available; every generator below is a stand-in with the
same dimension, element type and clustered structure:

* ``gaussian_mixture_f32`` - isotropic mixture, centres ~ N(0, centre_std^2 I),
  points = centre + N(0, I) (small float workload).
* ``clustered_u8`` - Sift-like: centres ~ U[lo, hi]^d, points
  round(clip(centre + N(0, sigma^2 I), 0, 255)); duplicates occur.
* ``anisotropic_mixture`` - Deep/Laion-like: per component a random rotation Q
  and eigenvalues lambda_i ~ i^-1 scaled to a fixed trace; optionally
  L2-normalised; returned as f32 or f16.
* ``powerlaw_gaussian`` - embedding-like: one zero-mean Gaussian whose
  eigenvalues decay as i^-alpha, under a random rotation.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "gaussian_mixture_f32",
    "clustered_u8",
    "anisotropic_mixture",
    "powerlaw_gaussian",
    "kmeans_sample",
    "uneven_shards",
    "mlp_init",
    "triplet_draws",
    "row_sample",
]


def gaussian_mixture_f32(n: int, d: int, n_centres: int = 16, centre_std: float = 2.0,
                         seed: int = 1001, queries: int = 0):
    """Isotropic Gaussian mixture, equal weights, float32 [n, d] (plus a held-out
    query set from the same centres when queries > 0)."""
    rng = np.random.default_rng(seed)
    centres = rng.normal(0.0, centre_std, size=(n_centres, d))
    lab = rng.integers(0, n_centres, size=n)
    x = centres[lab] + rng.normal(0.0, 1.0, size=(n, d))
    x = np.ascontiguousarray(x.astype(np.float32))
    if queries:
        lq = rng.integers(0, n_centres, size=queries)
        q = centres[lq] + rng.normal(0.0, 1.0, size=(queries, d))
        return x, np.ascontiguousarray(q.astype(np.float32))
    return x


def clustered_u8(n: int, d: int, n_centres: int = 256, lo: float = 32.0, hi: float = 224.0,
                 sigma: float = 20.0, seed: int = 1002, queries: int = 0):
    """Sift-like clustered uint8 vectors [n, d] (rounded and clipped to 0..255).

    With queries > 0 also returns a held-out query set [queries, d] drawn from
    the same centres after the data (the data itself does not change)."""
    rng = np.random.default_rng(seed)
    centres = rng.uniform(lo, hi, size=(n_centres, d)).astype(np.float32)

    def draw(m):
        lab = rng.integers(0, n_centres, size=m)
        out = np.empty((m, d), dtype=np.uint8)
        step = 1 << 18
        for s in range(0, m, step):
            e = min(m, s + step)
            z = rng.standard_normal(size=(e - s, d), dtype=np.float32) * np.float32(sigma)
            v = np.rint(centres[lab[s:e]] + z)
            out[s:e] = np.clip(v, 0, 255).astype(np.uint8)
        return out

    # labels of the data are drawn before its noise, as a single block
    lab = rng.integers(0, n_centres, size=n)
    out = np.empty((n, d), dtype=np.uint8)
    step = 1 << 18
    for s in range(0, n, step):
        e = min(n, s + step)
        z = rng.standard_normal(size=(e - s, d), dtype=np.float32) * np.float32(sigma)
        v = np.rint(centres[lab[s:e]] + z)
        out[s:e] = np.clip(v, 0, 255).astype(np.uint8)
    if queries:
        return out, draw(queries)
    return out


def _random_orthogonal(rng: np.random.Generator, d: int) -> np.ndarray:
    q, r = np.linalg.qr(rng.normal(size=(d, d)))
    return q * np.sign(np.diag(r))[None, :]


def anisotropic_mixture(n: int, d: int, n_comp: int, trace: float = 0.25, normalise: bool = True,
                        out_dtype=np.float32, seed: int = 1003, rotations: int = 16) -> np.ndarray:
    """Anisotropic Gaussian mixture [n, d].

    Component c has centre ~ N(0, I) and covariance Q_c diag(lambda) Q_c^T with
    lambda_i proportional to i^-1, scaled so that sum(lambda) = trace.  To keep
    generation cheap at 10^7 points, components share ``rotations`` random
    orthogonal matrices (component c uses rotation c % rotations).
    """
    rng = np.random.default_rng(seed)
    lam = 1.0 / np.arange(1, d + 1, dtype=np.float64)
    lam *= trace / lam.sum()
    sd = np.sqrt(lam).astype(np.float32)
    centres = rng.normal(size=(n_comp, d)).astype(np.float32)
    rots = [(_random_orthogonal(rng, d).astype(np.float32)) for _ in range(rotations)]
    lab = rng.integers(0, n_comp, size=n)
    out = np.empty((n, d), dtype=out_dtype)
    step = 1 << 17
    for s in range(0, n, step):
        e = min(n, s + step)
        z = rng.standard_normal(size=(e - s, d), dtype=np.float32) * sd[None, :]
        lb = lab[s:e]
        v = centres[lb].copy()
        rid = lb % rotations
        for q in range(rotations):
            m = rid == q
            if m.any():
                v[m] += z[m] @ rots[q].T
        if normalise:
            v /= np.linalg.norm(v, axis=1, keepdims=True).astype(np.float32)
        out[s:e] = v.astype(out_dtype)
    return out


def powerlaw_gaussian(n: int, d: int, alpha: float = 0.8, seed: int = 1004) -> np.ndarray:
    """Zero-mean Gaussian with eigenvalues i^-alpha under a random rotation, f32 [n, d]."""
    rng = np.random.default_rng(seed)
    sd = np.power(np.arange(1, d + 1, dtype=np.float64), -alpha / 2.0).astype(np.float32)
    q = _random_orthogonal(rng, d).astype(np.float32)
    out = np.empty((n, d), dtype=np.float32)
    step = 1 << 16
    for s in range(0, n, step):
        e = min(n, s + step)
        z = rng.standard_normal(size=(e - s, d), dtype=np.float32) * sd[None, :]
        out[s:e] = z @ q.T
    return out


def kmeans_sample(n: int, n_centroids: int, seed: int) -> tuple[np.ndarray, np.ndarray]:
    """The k-means training sample and the initial centroid rows.

    Sample size S = min(n, max(256 * C, n // 100)), drawn without replacement
    and sorted; the initial centroids are the rows of the first C entries of a
    seeded permutation of the sample.  Returns (sample_idx [S] uint32,
    init_rows [C] uint32), both global row indices.
    """
    rng = np.random.default_rng(seed)
    s = min(n, max(256 * n_centroids, n // 100))
    sample = np.sort(rng.choice(n, size=s, replace=False)).astype(np.uint32)
    perm = rng.permutation(s)[:n_centroids]
    return sample, sample[perm].astype(np.uint32)


def uneven_shards(n: int, n_shards: int, r: int, lo: int, hi: int, seed: int
                  ) -> tuple[np.ndarray, np.ndarray]:
    """Synthetic uneven shards for the grouped form.

    Shard sizes are drawn log-uniform on [lo, hi] and rescaled so that they sum
    to r * n (largest remainders first); every vector is then placed in r
    distinct shards so that shard s holds exactly its size: the r * n slots
    (shard s repeated size[s] times) are shuffled and dealt r to a vector, and a
    vector dealt the same shard twice trades one slot with a random other
    vector until both hold distinct shards.  Returns (members [r*n] uint32
    sorted by id within each shard, offsets [n_shards + 1] int64).
    """
    rng = np.random.default_rng(seed)
    raw = np.exp(rng.uniform(np.log(lo), np.log(hi), size=n_shards))
    exact = raw / raw.sum() * r * n
    size = np.floor(exact).astype(np.int64)
    size[np.argsort(-(exact - size), kind="stable")[: r * n - size.sum()]] += 1
    if r > n_shards or size.max() > n:
        raise ValueError("each vector needs r distinct shards of at most n members")
    slots = np.repeat(np.arange(n_shards, dtype=np.int64), size)
    rng.shuffle(slots)
    owner = slots.reshape(n, r)

    def clash(rows):
        o = np.sort(owner[rows], axis=1)
        return (o[:, 1:] == o[:, :-1]).any(axis=1)

    bad = np.flatnonzero(clash(np.arange(n)))
    for g in bad:
        while True:
            row = owner[g]
            vals, cnt = np.unique(row, return_counts=True)
            if (cnt == 1).all():
                break
            a = int(np.flatnonzero(row == vals[np.argmax(cnt > 1)])[0])
            h = int(rng.integers(n))
            b = int(rng.integers(r))
            if h == g or owner[h, b] in row or row[a] in np.delete(owner[h], b):
                continue
            owner[g, a], owner[h, b] = owner[h, b], owner[g, a]
    offsets = np.zeros(n_shards + 1, dtype=np.int64)
    offsets[1:] = np.cumsum(size)
    flat_shard = owner.ravel()
    flat_id = np.repeat(np.arange(n, dtype=np.int64), r)
    order = np.lexsort((flat_id, flat_shard))
    members = flat_id[order].astype(np.uint32)
    return members, offsets


def mlp_init(d: int, hidden: int = 256, out: int = 32, seed: int = 1006) -> np.ndarray:
    """Initial parameters of the d -> hidden -> out projection MLP as one float32
    array [W1 (hidden x d) | b1 | W2 (out x hidden) | b2]: W1 ~ N(0, 2/d) (He),
    W2 ~ N(0, 1/hidden), biases zero."""
    rng = np.random.default_rng(seed)
    W1 = rng.normal(0.0, np.sqrt(2.0 / d), size=(hidden, d))
    W2 = rng.normal(0.0, np.sqrt(1.0 / hidden), size=(out, hidden))
    return np.concatenate([W1.ravel(), np.zeros(hidden), W2.ravel(), np.zeros(out)]
                          ).astype(np.float32)


def triplet_draws(steps: int, batch: int, seed: int = 1007) -> np.ndarray:
    """Uniform uint32 draws [steps, batch, 3] for the triplet picks (anchor slot,
    positive rank, negative row), reduced modulo their ranges by the method."""
    rng = np.random.default_rng(seed)
    return rng.integers(0, 2**32, size=(steps, batch, 3), dtype=np.uint64).astype(np.uint32)


def row_sample(n: int, frac: float = 0.01, minimum: int = 256, seed: int = 1008) -> np.ndarray:
    """Sorted uint32 sample of max(minimum, frac * n) distinct rows (at most n)."""
    rng = np.random.default_rng(seed)
    s = min(n, max(minimum, int(frac * n)))
    return np.sort(rng.choice(n, size=s, replace=False)).astype(np.uint32)
