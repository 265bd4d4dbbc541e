"""Pins of the oracle's blockwise-adaptive assignment with selective replication
(Sec. V-A, Sec. V-B, Algorithm 1) against facts it does not compute itself:
the paper's three-cluster example (Fig. 2) worked by hand, the reductions to the
plain nearest-r assignment and to the Voronoi assignment, the absence of
replicas when eps <= 1, the monotone replication trend in eps (Table 4), and an
independent pure-Python restatement on tiny inputs.  No GPU needed.
"""
import os

import numpy as np
import pytest

import oracle
from paper_2605_10135_gb300 import datagen

GOLD = os.path.join(os.path.dirname(__file__), "golden")
PAD = oracle.PAD


def _fig2_cases():
    cases = []
    with open(os.path.join(GOLD, "selective_fig2_three_clusters.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            head, shards, stats = [p.strip() for p in line.split("|")]
            name, eps, tau0, block, cap = head.split()
            sets = [sorted(int(c) for c in s.strip().split(",")) for s in shards.split(";")]
            cases.append((name, float(eps), float(tau0), int(block), int(cap), sets,
                          [int(v) for v in stats.split()]))
    return cases


FIG2_X = np.array([[2, 4], [9, 1], [4, 6]], np.float32)
FIG2_C = np.array([[0, 0], [10, 0], [5, 8]], np.float32)


@pytest.mark.parametrize("case", _fig2_cases(), ids=lambda c: c[0])
def test_fig2_example_by_hand(case):
    _, eps, tau0, block, cap, sets, stats = case
    a, st = oracle.selective(FIG2_X, FIG2_C, 2, eps=eps, tau0=tau0, block=block, cap=cap)
    got = [sorted(int(c) for c in row if c != PAD) for row in a]
    assert got == sets
    assert st.tolist() == stats
    # the original comes first in each row
    for row, s in zip(a, sets):
        assert int(row[0]) in s


def _data(kind, n, d, seed):
    if kind == "u8":
        return datagen.clustered_u8(n, d, n_centres=12, seed=seed)
    return datagen.gaussian_mixture_f32(n, d, n_centres=12, seed=seed)


def _centroids(X, C, seed):
    rng = np.random.default_rng(seed)
    return X[rng.choice(len(X), C, replace=False)].astype(np.float32)


@pytest.mark.parametrize("kind", ["u8", "f32"])
@pytest.mark.parametrize("block", [1, 37, 1000])
def test_no_selectivity_no_capacity_is_nearest_r(kind, block):
    # eps = inf and no capacity: Algorithm 1 takes the first omega candidates,
    # i.e. the plain assignment to the omega nearest centroids (Sec. II-B).
    X = _data(kind, 500, 24, 11)
    cent = _centroids(X, 9, 1)
    for omega in (1, 2, 3):
        a, st = oracle.selective(X, cent, omega, block=block)
        ref = oracle.assign(X, cent, omega)
        assert np.array_equal(a, ref)
        assert st.tolist() == [500 * (omega - 1), 0]


@pytest.mark.parametrize("eps", [1.05, 1.5, float("inf")])
def test_omega_one_is_voronoi(eps):
    X = _data("f32", 400, 16, 12)
    cent = _centroids(X, 7, 2)
    a, st = oracle.selective(X, cent, 1, eps=eps, tau0=3.0, block=50)
    assert np.array_equal(a, oracle.assign(X, cent, 1))
    assert st.tolist() == [0, 0]


@pytest.mark.parametrize("eps", [0.5, 1.0])
def test_eps_at_most_one_replicates_nothing(eps):
    # d' < eps d <= d is impossible for a candidate after the nearest one.
    X = _data("u8", 300, 32, 13)
    cent = _centroids(X, 8, 3)
    a, st = oracle.selective(X, cent, 3, eps=eps, tau0=5.0, block=64)
    assert st[0] == 0
    assert np.all(a[:, 1:] == PAD)
    assert np.array_equal(a[:, 0], oracle.assign(X, cent, 1)[:, 0])


def test_replication_grows_with_eps_up_to_full():
    # Table 4: the share of replicated vectors rises with eps (33.3%, 54.3%,
    # 81.8% at 1.1, 1.2, 1.5) up to 100% for the original full replication.
    X = _data("f32", 2000, 32, 14)
    cent = _centroids(X, 16, 4)
    prev = -1
    shares = []
    for eps in (1.0, 1.05, 1.1, 1.2, 1.5, 2.0, 4.0, float("inf")):
        a, st = oracle.selective(X, cent, 2, eps=eps, tau0=2.0, block=256)
        n_rep = int(np.sum(a[:, 1] != PAD))
        assert n_rep == st[0]
        assert n_rep >= prev
        prev = n_rep
        shares.append(n_rep / len(X))
    assert shares[0] == 0.0 and shares[-1] == 1.0
    assert 0.0 < shares[2] < shares[4] < 1.0


def test_rows_are_valid_and_capacity_holds():
    X = _data("u8", 1200, 16, 15)
    cent = _centroids(X, 10, 5)
    cap = 260  # 10 x 260 = 2600 slots for 1200 originals + replicas
    a, st = oracle.selective(X, cent, 3, eps=1.6, tau0=2.0, block=100, cap=cap)
    assert st[1] == 0
    counts = np.bincount(a[a != PAD].astype(np.int64), minlength=10)
    assert counts.max() <= cap
    for row in a:
        vals = [int(c) for c in row if c != PAD]
        assert 1 <= len(vals) <= 3 and len(set(vals)) == len(vals)
        # pads only at the end
        assert all(c == PAD for c in row[len(vals):])
    members, offsets = oracle.shards(a, 10)
    assert offsets[-1] == len(X) + st[0]
    for c in range(10):
        m = members[offsets[c]:offsets[c + 1]]
        assert np.all(np.diff(m.astype(np.int64)) > 0)


# ---------------------------------------------- an independent restatement

def _d32(x, c):
    s = np.float32(0.0)
    for t in range(len(x)):
        df = np.float32(np.float32(x[t]) - np.float32(c[t]))
        s = np.float32(s + np.float32(df * df))
    return s


def _selective_py(X, cent, omega, M, eps, tau0, block, cap):
    """Algorithm 1 with the block schedule of Sec. V-A, written out plainly."""
    N, C = len(X), len(cent)
    dist = [[_d32(X[v], cent[c]) for c in range(C)] for v in range(N)]
    order = [sorted(range(C), key=lambda c: (dist[v][c], c))[:M] for v in range(N)]
    size = [0] * C
    originals = [0] * C
    replicas = [0] * C
    radius2 = [np.float32(0.0)] * C
    out = [[] for _ in range(N)]
    n_ovf = 0
    for b, b0 in enumerate(range(0, N, block), start=1):
        vs = range(b0, min(N, b0 + block))
        for v in vs:
            room = [c for c in order[v] if cap == 0 or size[c] < cap]
            if room:
                c = room[0]
            else:
                c = order[v][0]
                n_ovf += 1
            out[v].append(c)
            size[c] += 1
            originals[c] += 1
            radius2[c] = max(radius2[c], dist[v][c])
        seen = vs.stop
        limit = [None] * C
        if cap:
            for c in range(C):
                projected = -(-originals[c] * N // seen)
                limit[c] = max(0, cap - projected)
        tau = 1.0 + (tau0 - 1.0) / b
        for v in vs:
            c = out[v][0]
            for c2 in order[v]:
                if len(out[v]) >= omega:
                    break
                if c2 == c:
                    continue
                if cap and (replicas[c2] >= limit[c2] or size[c2] >= cap):
                    continue
                if not np.isinf(eps):
                    ok = float(dist[v][c2]) < (eps * eps) * float(dist[v][c])
                    ok = ok and float(dist[v][c2]) < ((eps * tau) * (eps * tau)) * float(radius2[c2])
                    if not ok:
                        continue
                out[v].append(c2)
                replicas[c2] += 1
                size[c2] += 1
    a = np.full((N, omega), PAD, np.uint32)
    for v in range(N):
        a[v, :len(out[v])] = out[v]
    return a, [sum(replicas), n_ovf]


@pytest.mark.parametrize("seed", range(18))
def test_matches_plain_python_on_tiny_inputs(seed):
    rng = np.random.default_rng(100 + seed)
    N, d, C = int(rng.integers(20, 60)), int(rng.integers(2, 6)), int(rng.integers(3, 7))
    if seed % 2:
        X = rng.integers(0, 8, size=(N, d)).astype(np.uint8)  # many exact ties
    else:
        X = rng.normal(size=(N, d)).astype(np.float32)
    cent = X[rng.choice(N, C, replace=False)].astype(np.float32)
    omega = int(rng.integers(1, min(C, 4) + 1))
    M = int(rng.integers(omega, C + 1))
    eps = [1.1, 1.3, 2.0, float("inf")][seed % 4]
    tau0 = [1.0, 2.0, 4.0][seed % 3]
    block = int(rng.integers(1, N + 1))
    cap = [0, int(np.ceil(1.3 * N / C)), int(np.ceil(0.8 * N / C))][seed % 3]
    a, st = oracle.selective(X, cent, omega, M=M, eps=eps, tau0=tau0, block=block, cap=cap)
    ref, rst = _selective_py(X, cent, omega, M, eps, tau0, block, cap)
    assert np.array_equal(a, ref)
    assert st.tolist() == rst
