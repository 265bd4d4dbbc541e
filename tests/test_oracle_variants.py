"""Pins of the oracle's prune and merge variants (the occlusion prune of the
Vamana family of graph builders and a merge that adds reverse edges), the
alternatives to the rank-detour prune and the plain edge union.  Hand-worked
examples on four points of a line, reductions, invariants and a plain-Python
restatement on random inputs.  No GPU needed."""
import numpy as np
import pytest

import oracle

PAD = oracle.PAD
LINE = np.array([[0], [1], [3], [7]], np.float32)  # ids 0..3


def _lists(X, k):
    ids, ds = oracle.bruteforce(X, X, k + 1)
    out_i = np.full((len(X), k), PAD, np.uint32)
    out_d = np.full((len(X), k), np.inf)
    for u in range(len(X)):
        keep = [(int(i), float(d)) for i, d in zip(ids[u], ds[u]) if int(i) != u][:k]
        for j, (i, d) in enumerate(keep):
            out_i[u, j], out_d[u, j] = i, d
    return out_i, out_d


def test_occlusion_prune_by_hand():
    # lists (squared distances): 0: 1(1) 2(9) 3(49); 1: 0(1) 2(4) 3(36);
    # 2: 1(4) 0(9) 3(16); 3: 2(16) 1(36) 0(49).
    # alpha = 1 keeps the nearest point on each side: 0 -> [1]; 1 -> [0, 2]
    # (3 is occluded by 2: 16 <= 36); 2 -> [1, 3] (0 occluded by 1: 1 <= 9);
    # 3 -> [2].
    ki, kd = _lists(LINE, 3)
    pid, pd = oracle.prune_alpha(LINE, ki, kd, 3, alpha=1.0)
    got = [[int(v) for v in row if v != PAD] for row in pid]
    assert got == [[1], [0, 2], [1, 3], [2]]
    assert pd[1].tolist()[:2] == [1.0, 4.0]
    # alpha = 2 (alpha^2 = 4) occludes less: 0 -> [1, 2, 3] (4*4 = 16 > 9,
    # 4*36 > 49 and 4*16 > 49); 1 -> [0, 2, 3]; 2 -> [1, 3] (4*1 <= 9 still occludes 0)
    pid, _ = oracle.prune_alpha(LINE, ki, kd, 3, alpha=2.0)
    got = [[int(v) for v in row if v != PAD] for row in pid]
    assert got[0] == [1, 2, 3] and got[1] == [0, 2, 3] and got[2] == [1, 3]


def _prune_py(X, ki, kd, R, alpha):
    out = []
    for u in range(len(ki)):
        kept = []
        for v, duv in zip(ki[u], kd[u]):
            if v == PAD or len(kept) >= R:
                continue
            occ = any((alpha * alpha) * float(np.sum((X[w].astype(np.float64) -
                                                        X[v].astype(np.float64)) ** 2)) <= duv
                      for w, _ in kept)
            if not occ:
                kept.append((int(v), float(duv)))
        out.append(kept)
    return out


@pytest.mark.parametrize("seed", range(4))
def test_occlusion_prune_matches_restatement_and_invariants(seed):
    rng = np.random.default_rng(500 + seed)
    X = rng.normal(size=(60, 5)).astype(np.float32)
    ki, kd = _lists(X, 12)
    R, alpha = 6, [1.0, 1.2, 1.5, 3.0][seed]
    pid, pd = oracle.prune_alpha(X, ki, kd, R, alpha)
    ref = _prune_py(X, ki, kd, R, alpha)
    for u in range(len(X)):
        got = [(int(v), float(d)) for v, d in zip(pid[u], pd[u]) if v != PAD]
        assert got == ref[u]
        assert got and got[0][0] == int(ki[u, 0])   # the nearest is never occluded
        assert set(v for v, _ in got) <= set(int(v) for v in ki[u])
        pos = [list(ki[u]).index(v) for v, _ in got]
        assert pos == sorted(pos)                    # list order kept
    # a huge alpha occludes nothing (distinct points): truncation to R
    pid, _ = oracle.prune_alpha(X, ki, kd, R, 1e6)
    assert np.array_equal(pid, ki[:, :R])


def test_reverse_merge_by_hand():
    # path 0 -> 1 -> 2 -> 3 -> 2 on the line, R = 2 (one forward entry kept first):
    # 0: [1]; 1: forward 2, reverse 0 -> sorted [0 (1), 2 (4)];
    # 2: forward 3, reverse 1 (4) then 3 (taken) -> [1 (4), 3 (16)]; 3: [2].
    g = np.array([[1, PAD], [2, PAD], [3, PAD], [2, PAD]], np.uint32)
    gd = np.array([[1, np.inf], [4, np.inf], [16, np.inf], [16, np.inf]], np.float64)
    deg = np.array([1, 1, 1, 1], np.uint32)
    og, od, odeg = oracle.merge_reverse(g, gd, deg)
    got = [[int(v) for v in row[:n]] for row, n in zip(og, odeg)]
    assert got == [[1], [0, 2], [1, 3], [2]]
    assert od[1].tolist() == [1.0, 4.0] and od[2].tolist() == [4.0, 16.0]


def test_reverse_merge_leaves_a_symmetric_graph_unchanged():
    ki, kd = _lists(LINE, 3)
    pid, pd = oracle.prune_alpha(LINE, ki, kd, 3, 1.0)  # the path 0-1-2-3, symmetric
    deg = (pid != PAD).sum(1).astype(np.uint32)
    og, od, odeg = oracle.merge_reverse(pid, pd, deg)
    assert np.array_equal(og, pid) and np.array_equal(odeg, deg)


@pytest.mark.parametrize("seed", range(3))
def test_reverse_merge_invariants(seed):
    rng = np.random.default_rng(600 + seed)
    X = rng.normal(size=(80, 4)).astype(np.float32)
    ki, kd = _lists(X, 8)
    R = 6
    g, gd = ki[:, :R].copy(), kd[:, :R].copy()
    deg = np.full(len(X), R, np.uint32)
    og, od, odeg = oracle.merge_reverse(g, gd, deg)
    rev = {v: set() for v in range(len(X))}
    for u in range(len(X)):
        for v in g[u]:
            rev[int(v)].add(u)
    for v in range(len(X)):
        got = [int(x) for x in og[v, :odeg[v]]]
        assert len(got) == len(set(got)) <= R and v not in got
        assert set(got) <= set(int(x) for x in g[v]) | rev[v]
        assert set(int(x) for x in g[v, :(R + 1) // 2]) <= set(got)
        d = od[v, :odeg[v]].tolist()
        assert d == sorted(d)
