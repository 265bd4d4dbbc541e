"""Named workloads: the paper's Table 3 shapes scaled to synthetic stand-ins.

Each entry gives the vector count N, dimension d, element type, shard count C,
replicas r, intermediate degree k (the paper's L) and final degree R, plus the
generator that draws the vectors (see datagen).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import datagen


@dataclass(frozen=True)
class Workload:
    name: str
    N: int
    d: int
    dtype: str
    C: int
    r: int
    k: int
    R: int
    seed: int
    # synthetic uneven shards (log-uniform sizes on [lo, hi], rescaled to r N rows)
    # in place of the k-means partition; None: the k-means partition
    uneven: tuple | None = None

    def vectors(self, n: int | None = None, seed_offset: int = 0) -> np.ndarray:
        n = self.N if n is None else n
        s = self.seed + seed_offset
        base = self.name.split("@")[0]
        if base.startswith("gauss"):
            return datagen.gaussian_mixture_f32(n, self.d, 16, 2.0, seed=s)
        if base.startswith("sift"):
            return datagen.clustered_u8(n, self.d, 256, seed=s)
        if base.startswith("deep"):
            return datagen.anisotropic_mixture(n, self.d, 1024, 0.25, True, np.float32, seed=s)
        if base.startswith("laion"):
            return datagen.powerlaw_gaussian(n, self.d, 0.8, seed=s)
        if base.startswith("embed"):
            return datagen.anisotropic_mixture(n, self.d, 4096, 0.25, False, np.float16, seed=s)
        raise KeyError(self.name)

    def vectors_and_queries(self, nq: int):
        """The vectors plus nq held-out queries from the same distribution."""
        base = self.name.split("@")[0]
        if base.startswith("gauss"):
            return datagen.gaussian_mixture_f32(self.N, self.d, 16, 2.0, seed=self.seed, queries=nq)
        if base.startswith("sift"):
            return datagen.clustered_u8(self.N, self.d, 256, seed=self.seed, queries=nq)
        X = self.vectors()
        return X, self.vectors(nq, seed_offset=777)

    def kmeans_inputs(self, n: int | None = None):
        return datagen.kmeans_sample(self.N if n is None else n, self.C, seed=self.seed + 7)

    def shards(self):
        """(members, offsets) of the synthetic uneven partition."""
        lo, hi = self.uneven
        return datagen.uneven_shards(self.N, self.C, self.r, lo, hi, seed=self.seed + 9)


# Small float mixture (oracle finishes in seconds): N=1e4, d=64, 4 shards.
GAUSS_10K = Workload("gauss10k_d64_f32", 10_000, 64, "f32", 4, 2, 32, 16, 1001)
# Sift-like integer-exact workload: N=1e6, d=128 uint8, 16 shards.
SIFT_1M = Workload("sift1m_d128_u8", 1_000_000, 128, "u8", 16, 2, 64, 32, 1002)
# Deep-like unit-norm floats: N=1e7, d=96, 64 shards.
DEEP_10M = Workload("deep10m_d96_f32", 10_000_000, 96, "f32", 64, 2, 64, 32, 1003)
# Laion-like power-law floats: N=2e6, d=768, 128 uneven shards (log-uniform sizes
# on [5e3, 4e5], rescaled to the 4e6 shard rows), no k-means.
LAION_2M = Workload("laion2m_d768_f32", 2_000_000, 768, "f32", 128, 2, 32, 32, 1004,
                    uneven=(5_000, 400_000))
# High-dimensional FP16 embeddings: N=1e7, d=1024, 128 shards.
EMBED_10M = Workload("embed10m_d1024_f16", 10_000_000, 1024, "f16", 128, 2, 64, 32, 1005)

ALL = [GAUSS_10K, SIFT_1M, DEEP_10M, LAION_2M, EMBED_10M]
BY_NAME = {w.name: w for w in ALL}
