"""Merge with reverse edges (ann_merge_reverse) against the oracle's
or_merge_reverse: ids, distances and degrees bit for bit, on synthetic graphs
(hubs whose in-degree passes 64, distance ties, empty and full lists, odd R) and
on the merged graph of a build."""
import numpy as np
import pytest
import torch

import oracle
from paper_2605_10135_gb300 import ann, build, datagen
from tests.parity import as_u32

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
PAD = 0xFFFFFFFF


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    ann.lib()
    ann.device_status()
    yield
    assert ann.device_status() == 0


def T(a):
    a = np.ascontiguousarray(a)
    if a.dtype == np.uint32:
        a = a.view(np.int32)
    return torch.from_numpy(a).to(DEV)


def _graph(N, R, seed):
    """Lists of distinct ids (no self-loops) sorted by (distance, id), integer
    distances (many ties), degrees 0..R; eight hubs sit in about half the lists."""
    rng = np.random.default_rng(seed)
    deg = rng.integers(0, R + 1, size=N).astype(np.uint32)
    deg[:7] = R
    deg[7:11] = 0
    hubs = rng.choice(N, 8, replace=False)
    graph = np.full((N, R), PAD, np.uint32)
    gdist = np.full((N, R), np.inf, np.float32)
    for u in range(N):
        d = int(deg[u])
        cand = [int(h) for h in hubs if h != u and rng.random() < 0.5][:d]
        seen = set(cand)
        while len(cand) < d:
            c = int(rng.integers(0, N))
            if c != u and c not in seen:
                seen.add(c)
                cand.append(c)
        ids = np.array(cand, np.uint32)
        dist = rng.integers(1, 40, size=d).astype(np.float32)
        o = np.lexsort((ids, dist))
        graph[u, :d] = ids[o]
        gdist[u, :d] = dist[o]
    return graph, gdist, deg


def _check(graph, gdist, deg):
    g, gd, dg = ann.merge_reverse(T(graph), T(gdist), T(deg))
    og, od, odeg = oracle.merge_reverse(graph, gdist.astype(np.float64), deg)
    assert np.array_equal(dg.cpu().numpy().view(np.uint32), odeg)
    assert np.array_equal(as_u32(g), og)
    assert np.array_equal(gd.cpu().numpy().astype(np.float64), od)
    return og, odeg


@pytest.mark.parametrize("R", [1, 8, 31, 32, 64])
def test_reverse_merge_matches_the_oracle_on_synthetic_graphs(R):
    graph, gdist, deg = _graph(3000, R, seed=700 + R)
    og, odeg = _check(graph, gdist, deg)
    # hubs: more than 64 reverse sources reach some vertices (several selection rounds)
    indeg = np.bincount(graph[graph != PAD].astype(np.int64), minlength=3000)
    assert indeg.max() > 64
    assert (odeg <= R).all() and (odeg >= np.minimum(deg, R)).all()


def test_reverse_merge_of_a_built_index():
    X = datagen.clustered_u8(20000, 64, 24, seed=711)
    cfg = ann.BuildConfig(C=8, r=2, k=32, R=16, iters=4)
    sample, init_rows = datagen.kmeans_sample(X.shape[0], cfg.C, 712)
    out = ann.build_index(T(X), cfg, T(X[init_rows].astype(np.float32)), T(sample))
    graph = as_u32(out["graph"])
    gdist = out["gdist"].cpu().numpy()
    deg = out["degree"].cpu().numpy().view(np.uint32)
    og, odeg = _check(graph, gdist, deg)
    # every own edge of the first half survives; the degree never drops
    half = (16 + 1) // 2
    for v in range(0, 20000, 997):
        keep = graph[v, :min(int(deg[v]), half)]
        assert set(keep.tolist()) <= set(og[v, :odeg[v]].tolist())
    assert (odeg >= deg).all()


def test_reverse_merge_of_an_empty_graph():
    graph = np.full((5, 4), PAD, np.uint32)
    gdist = np.full((5, 4), np.inf, np.float32)
    deg = np.zeros(5, np.uint32)
    og, odeg = _check(graph, gdist, deg)
    assert (odeg == 0).all() and (og == PAD).all()
