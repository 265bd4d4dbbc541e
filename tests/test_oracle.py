"""Pins of the CPU oracle against facts it does not compute itself.

Every function of the oracle is checked here against a hand-worked example,
a closed form, a library routine (scipy / scikit-learn) or an invariant the
method guarantees, chosen so that a dropped term, a wrong sign or index or a
transposed operand fails at least one test.  No test here needs a GPU.
"""
import os

import numpy as np
import pytest

import oracle
from paper_2605_10135_gb300 import datagen

GOLD = os.path.join(os.path.dirname(__file__), "golden")
PAD = oracle.PAD


def _gold(name):
    rows = []
    with open(os.path.join(GOLD, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append([float(v) for v in line.split()])
    return np.array(rows)


# ---------------------------------------------------------------- distances

def test_d64_closed_forms():
    assert oracle.d64(np.array([0, 0], np.float32), np.array([3, 4], np.float32)) == 25.0
    a = np.array([255, 0, 7], np.uint8)
    b = np.array([0, 255, 7], np.uint8)
    assert oracle.d64(a, b) == 2 * 255 ** 2
    rng = np.random.default_rng(0)
    x, y = rng.normal(size=(2, 37)).astype(np.float32)
    assert oracle.d64(x, y) == oracle.d64(y, x)
    assert oracle.d64(x, x) == 0.0
    # float16 elements are converted exactly (numpy's own float16 -> float64)
    h = rng.normal(size=(2, 19)).astype(np.float16)
    ref = float(np.sum((h[0].astype(np.float64) - h[1].astype(np.float64)) ** 2))
    assert abs(oracle.d64(h[0], h[1]) - ref) <= 1e-12 * ref
    # subnormal and extreme float16 values
    z = np.array([6e-8, 65504.0, -3.0e-5], np.float16)
    zz = np.zeros(3, np.float16)
    assert oracle.d64(z, zz) == float(np.sum(z.astype(np.float64) ** 2))


def test_d32_is_exact_on_integers_and_within_summation_bound():
    rng = np.random.default_rng(1)
    a, b = rng.integers(0, 256, size=(2, 128)).astype(np.uint8)
    assert oracle.d32(a, b) == oracle.d64(a, b)  # integers < 2^24 are exact in FP32
    for _ in range(20):
        x, y = rng.normal(size=(2, 96)).astype(np.float32)
        e = oracle.d64(x, y)
        # sequential FP32 summation of n terms: relative error <= (n + 2) u, u = 2^-24
        assert abs(oracle.d32(x, y) - e) <= (96 + 2) * 2.0 ** -24 * e


# ----------------------------------------------------------------- k-means

def test_kmeans_hand_example():
    X = np.array([[0], [1], [9], [10]], np.float32)
    init = np.array([[0], [1]], np.float32)
    for it, c0, c1 in _gold("kmeans_line4.txt"):
        cent, _ = oracle.kmeans(X, init, np.arange(4, dtype=np.uint32), int(it))
        assert cent[0, 0] == np.float32(c0) and cent[1, 0] == np.float32(c1)


def test_kmeans_single_centroid_is_sample_mean():
    X = datagen.gaussian_mixture_f32(500, 8, seed=5)
    idx = np.arange(0, 500, 3, dtype=np.uint32)
    cent, _ = oracle.kmeans(X, X[idx[:1]], idx, 3)
    ref = X[idx].astype(np.float64).mean(axis=0)
    assert np.all(np.abs(cent[0] - ref) <= 1e-6 * np.abs(ref) + 1e-7)


def test_kmeans_matches_sklearn_lloyd():
    sk = pytest.importorskip("sklearn.cluster")
    X = datagen.gaussian_mixture_f32(3000, 16, n_centres=6, centre_std=4.0, seed=7)
    idx = np.arange(3000, dtype=np.uint32)
    init = X[[0, 500, 1000, 1500, 2000, 2500]]
    cent, lab = oracle.kmeans(X, init, idx, 50)
    km = sk.KMeans(n_clusters=6, init=init.astype(np.float64), n_init=1, algorithm="lloyd",
                   max_iter=50, tol=0.0).fit(X.astype(np.float64))
    assert np.array_equal(lab, km.labels_)
    assert np.allclose(cent, km.cluster_centers_, rtol=1e-6, atol=1e-6)


def test_kmeans_objective_non_increasing_and_empty_cluster_kept():
    X = datagen.gaussian_mixture_f32(2000, 12, seed=9)
    idx = np.arange(0, 2000, 2, dtype=np.uint32)
    init = X[idx[:8]].copy()
    init[7] = 1e4  # far away: stays empty, must keep its initial value
    prev = np.inf
    for it in range(1, 7):
        cent, lab = oracle.kmeans(X, init, idx, it)
        pts = X[idx].astype(np.float64)
        obj = np.sum((pts - cent[lab].astype(np.float64)) ** 2)
        assert obj <= prev * (1 + 1e-9)
        prev = obj
        assert np.all(cent[7] == np.float32(1e4))


# -------------------------------------------------------------- assignment

def test_assign_r1_is_voronoi_and_r_equals_c_is_everything():
    sp = pytest.importorskip("scipy.spatial.distance")
    X = datagen.gaussian_mixture_f32(1000, 10, seed=11)
    cent = X[:5].copy() + 0.5
    a1 = oracle.assign(X, cent, 1)
    ref = np.argmin(sp.cdist(X.astype(np.float64), cent.astype(np.float64), "sqeuclidean"), axis=1)
    assert np.array_equal(a1[:, 0], ref)
    a5 = oracle.assign(X, cent, 5)
    assert np.all(np.sort(a5, axis=1) == np.arange(5)[None, :])


def test_assign_fp32_decision_agrees_with_fp64_up_to_near_ties():
    X = datagen.clustered_u8(5000, 32, n_centres=20, seed=13)
    cent = X[:7].astype(np.float32) + np.float32(0.37)
    a32 = oracle.assign(X, cent, 2)
    a64 = oracle.assign(X, cent, 2, use_d64=True)
    diff = np.nonzero(np.any(a32 != a64, axis=1))[0]
    for i in diff:  # any disagreement must be a tie within 1e-5 relative
        d = np.array([oracle.d64(X[i], c) for c in cent])
        s = np.sort(d)
        assert np.min(np.abs(np.diff(s[:3]))) <= 1e-5 * s[2]


def test_shards_invariants():
    X = datagen.gaussian_mixture_f32(2000, 8, seed=15)
    cent = X[:6].copy()
    a = oracle.assign(X, cent, 2)
    members, off = oracle.shards(a, 6)
    assert off[0] == 0 and off[-1] == 2 * 2000
    cnt = np.bincount(members, minlength=2000)
    assert np.all(cnt == 2)  # every vector in exactly r shards
    for c in range(6):
        seg = members[off[c]:off[c + 1]]
        assert np.all(np.diff(seg.astype(np.int64)) > 0)  # sorted, distinct
        assert np.all(np.any(a[seg] == c, axis=1))


# --------------------------------------------------------------- shard kNN

def test_shard_knn_single_shard_equals_kdtree():
    spat = pytest.importorskip("scipy.spatial")
    X = datagen.gaussian_mixture_f32(1500, 6, seed=17)
    members = np.arange(1500, dtype=np.uint32)
    off = np.array([0, 1500])
    ids, ds = oracle.shard_knn(X, members, off, 12)
    tree = spat.cKDTree(X.astype(np.float64))
    dd, ii = tree.query(X.astype(np.float64), k=13)
    assert np.array_equal(ids, ii[:, 1:].astype(np.uint32))
    assert np.allclose(ds, dd[:, 1:] ** 2, rtol=1e-12)


def test_shard_knn_ties_by_id_duplicates_and_padding():
    X = np.array([[5, 5], [5, 5], [5, 5], [6, 5], [0, 0]], np.uint8)
    members = np.array([0, 1, 2, 3, 4, 1, 4], np.uint32)
    off = np.array([0, 5, 7])
    ids, ds = oracle.shard_knn(X, members, off, 3)
    assert ids[0].tolist() == [1, 2, 3] and ds[0].tolist() == [0, 0, 1]
    assert ids[2].tolist() == [0, 1, 3]
    assert ids[3].tolist() == [0, 1, 2] and ds[3].tolist() == [1, 1, 1]
    # second shard has two members: one neighbour, then padding
    assert ids[5].tolist() == [4, PAD, PAD] and ds[5][0] == 50.0 and np.isinf(ds[5][1])


def test_shard_knn_symmetric_and_rows_subset():
    X = datagen.clustered_u8(600, 16, n_centres=8, seed=19)
    cent = X[:3].astype(np.float32)
    members, off = oracle.shards(oracle.assign(X, cent, 2), 3)
    ids, ds = oracle.shard_knn(X, members, off, 10)
    sub = np.array([3, 77, 500, 1199])
    ids2, ds2 = oracle.shard_knn(X, members, off, 10, rows=sub)
    assert np.array_equal(ids[sub], ids2) and np.array_equal(ds[sub], ds2)
    for p in range(0, len(members), 37):
        for v, dv in zip(ids[p], ds[p]):
            assert dv == oracle.d64(X[members[p]], X[v])


# ------------------------------------------------------------------- prune

def _line4():
    X = np.array([[0], [1], [3], [7]], np.float32)
    members = np.arange(4, dtype=np.uint32)
    off = np.array([0, 4])
    ids, ds = oracle.shard_knn(X, members, off, 3)
    return ids, ds, members, off


def test_prune_hand_example():
    ids, ds, members, off = _line4()
    pid, pd = oracle.prune(ids, ds, members, off, 2)
    g = _gold("prune_rank_detour_line4.txt")
    assert np.array_equal(pid, g[:, 1:3].astype(np.uint32))
    assert np.array_equal(pd, g[:, 3:5])
    tid, _ = oracle.prune(ids, ds, members, off, 2, rule=1)
    assert tid[2].tolist() == [1, 0]  # truncation differs from the detour rule


def _random_shard_graph(seed, n=40, k=8, shards=2, dtype=np.float32):
    X = datagen.gaussian_mixture_f32(n, 3, n_centres=4, seed=seed)
    cent = X[:shards].copy()
    members, off = oracle.shards(oracle.assign(X, cent, min(2, shards)), shards)
    ids, ds = oracle.shard_knn(X, members, off, k)
    return X, members, off, ids, ds


def test_prune_invariants():
    for seed in range(5):
        X, members, off, ids, ds = _random_shard_graph(seed)
        for R in (1, 3, 5, 8, 12):
            pid, pd = oracle.prune(ids, ds, members, off, R)
            for p in range(len(members)):
                valid = [v for v in ids[p] if v != PAD]
                out = [v for v in pid[p] if v != PAD]
                assert len(out) == min(R, len(valid))
                assert set(out) <= set(valid) and members[p] not in out
                pos = [valid.index(v) for v in out]
                assert pos == sorted(pos)  # emitted in list order (distance-sorted)
                assert all(pd[p][j] == ds[p][pos[j]] for j in range(len(out)))
            if R >= ids.shape[1]:
                assert np.array_equal(pid[:, :ids.shape[1]], ids)


def test_prune_brute_force_definition():
    """c_j recomputed from rank matrices (an independent formulation)."""
    for seed in range(4):
        X, members, off, ids, ds = _random_shard_graph(100 + seed, n=30, k=6, shards=1)
        n, k = ids.shape
        rank = np.full((n, n), 10 ** 6)
        for w in range(n):
            for t, v in enumerate(ids[w]):
                if v != PAD:
                    rank[w, v] = t
        R = 3
        pid, _ = oracle.prune(ids, ds, members, off, R)
        for u in range(n):
            L = [v for v in ids[u] if v != PAD]
            c = [sum(rank[L[i], L[j]] < j for i in range(j)) for j in range(len(L))]
            keep = sorted(sorted(range(len(L)), key=lambda j: (c[j], j))[:R])
            assert pid[u][:len(keep)].tolist() == [L[j] for j in keep]


def test_prune_all_zero_counts_equals_truncation():
    ids, ds, members, off = _line4()
    # rows 0 and 1 of the line example have all-zero counts
    pa, _ = oracle.prune(ids, ds, members, off, 2)
    pb, _ = oracle.prune(ids, ds, members, off, 2, rule=1)
    assert np.array_equal(pa[:2], pb[:2])


# ------------------------------------------------------------------- merge

def test_merge_r1_identity_and_hand_example():
    ids, ds, members, off = _line4()
    g, gd, deg = oracle.merge(ids, ds, members, off, 4)
    assert np.array_equal(g, ids) and np.array_equal(gd, ds) and np.all(deg == 3)
    # two shards sharing vector 0; duplicate edge 0->2 with equal distance
    members = np.array([0, 1, 2, 0, 2, 3], np.uint32)
    off = np.array([0, 3, 6])
    pr = np.array([[1, 2], [0, PAD], [0, PAD], [2, 3], [0, 3], [0, 2]], np.uint32)
    pd = np.array([[1.0, 4.0], [1.0, np.inf], [4.0, np.inf], [4.0, 9.0], [4.0, 1.0], [9.0, 1.0]])
    g, gd, deg = oracle.merge(pr, pd, members, off, 4)
    assert g[0].tolist() == [1, 2] and gd[0].tolist() == [1.0, 4.0] and deg[0] == 2
    g3, _, _ = oracle.merge(pr, pd, members, off, 4)
    assert g3[2].tolist() == [3, 0]


def test_merge_invariants_and_shard_order_independence():
    for seed in range(4):
        X, members, off, ids, ds = _random_shard_graph(200 + seed, n=50, k=8, shards=3)
        pid, pd = oracle.prune(ids, ds, members, off, 5)
        N = 50
        g, gd, deg = oracle.merge(pid, pd, members, off, N)
        for u in range(N):
            out = [v for v in g[u] if v != PAD]
            assert len(out) == deg[u] <= 5 and u not in out and len(set(out)) == len(out)
            rows = np.nonzero(members == u)[0]
            edges = {}
            for p in rows:
                for v, dv in zip(pid[p], pd[p]):
                    if v != PAD:
                        edges[v] = min(dv, edges.get(v, np.inf))
            assert set(out) <= set(edges)
            if deg[u] == 5:  # every shard edge ranking before the last kept one survives
                last = (gd[u][4], g[u][4])
                for v, dv in edges.items():
                    if (dv, v) <= last:
                        assert v in out
            else:
                assert set(out) == set(edges)
        # reversing the shard order gives the same graph
        C = len(off) - 1
        seg = [np.arange(off[c], off[c + 1]) for c in range(C)][::-1]
        perm = np.concatenate(seg)
        off2 = np.concatenate([[0], np.cumsum([len(s) for s in seg])])
        g2, gd2, deg2 = oracle.merge(pid[perm], pd[perm], members[perm], off2, N)
        assert np.array_equal(g, g2) and np.array_equal(gd, gd2) and np.array_equal(deg, deg2)


# ------------------------------------------------------------ search / GT

def test_bruteforce_matches_kdtree():
    spat = pytest.importorskip("scipy.spatial")
    X = datagen.gaussian_mixture_f32(2000, 5, seed=23)
    Q = datagen.gaussian_mixture_f32(50, 5, seed=24)
    ids, ds = oracle.bruteforce(X, Q, 10)
    dd, ii = spat.cKDTree(X.astype(np.float64)).query(Q.astype(np.float64), k=10)
    assert np.array_equal(ids, ii.astype(np.uint32))
    assert np.allclose(ds, dd ** 2, rtol=1e-12)


def test_medoid_hand_example():
    X = np.array([[0, 0], [10, 0], [4, 1], [0, 10]], np.float32)  # mean (3.5, 2.75)
    assert oracle.medoid(X) == 2


def test_search_complete_graph_is_exact_and_path_graph_walks():
    X = datagen.gaussian_mixture_f32(60, 4, seed=25)
    Q = datagen.gaussian_mixture_f32(12, 4, seed=26)
    N = 60
    graph = np.array([[v for v in range(N) if v != u] for u in range(N)], np.uint32)
    deg = np.full(N, N - 1, np.uint32)
    got, cnt = oracle.search(graph, deg, X, Q, entry=0, Ls=16)
    gt, _ = oracle.bruteforce(X, Q, 10)
    assert oracle.recall_at(got, gt) == 1.0
    assert np.all(cnt == N)  # every vertex is seen exactly once
    # a path 0-1-2-...-9 on the line: from vertex 0 greedy search walks to the query
    L = np.arange(10, dtype=np.float32)[:, None]
    path = np.array([[max(u - 1, 0), min(u + 1, 9)] for u in range(10)], np.uint32)
    path[0] = [1, PAD]
    path[9] = [8, PAD]
    pdeg = np.array([1] + [2] * 8 + [1], np.uint32)
    got, cnt = oracle.search(path, pdeg, L, np.array([[7.2]], np.float32), entry=0, Ls=2, topk=2)
    assert got[0].tolist() == [7, 8] and cnt[0] == 10


def test_recall_helper():
    a = np.array([[1, 2, 3], [4, 5, 6]], np.uint32)
    b = np.array([[3, 2, 9], [7, 8, 9]], np.uint32)
    assert oracle.recall_at(a, b, 3) == 2 / 6


# ------------------------------------------------------------- generators

def test_generators_shapes_and_determinism():
    a = datagen.clustered_u8(1000, 128, seed=3)
    assert a.dtype == np.uint8 and a.shape == (1000, 128)
    assert np.array_equal(a, datagen.clustered_u8(1000, 128, seed=3))
    b = datagen.anisotropic_mixture(500, 96, 32, seed=4)
    assert b.dtype == np.float32 and np.allclose(np.linalg.norm(b, axis=1), 1, atol=1e-5)
    s, init = datagen.kmeans_sample(100000, 16, seed=5)
    assert len(s) == 4096 and np.all(np.diff(s.astype(np.int64)) > 0) and np.all(np.isin(init, s))
