"""CUDA path (through the C-ABI) against the CPU oracle on the same seeded inputs.

Integer data and integer logic are compared bit for bit; float kNN lists follow
the rule in tests/parity.py.  Sizes span several 128-row blocks and 256-column
tiles with ragged tails; edge cases cover tiny shards (padding), one shard,
r = C, duplicate vectors and empty shards.
"""
import numpy as np
import pytest
import torch

import oracle
from oracle import precision as OP
from paper_2605_10135_gb300 import ann, build, datagen
from tests.parity import PAD, as_u32, check_float_lists

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


def _part_inputs(X, C, seed):
    sample, init_rows = datagen.kmeans_sample(X.shape[0], C, seed)
    init = X[init_rows].astype(np.float32)
    return sample, init


def _gpu_partition(X, C, r, iters, seed):
    sample, init = _part_inputs(X, C, seed)
    cent, mem, off = ann.partition(T(X), C, r, T(init), T(sample), iters)
    torch.cuda.synchronize()
    return cent.cpu().numpy(), as_u32(mem), off.cpu().numpy(), (sample, init)


# ------------------------------------------------------------------- partition

@pytest.mark.parametrize("kind", ["u8", "f32", "f16"])
def test_partition_bit_exact(kind):
    if kind == "u8":
        X = datagen.clustered_u8(3000, 128, 32, seed=31)
    elif kind == "f32":
        X = datagen.gaussian_mixture_f32(3000, 64, seed=32)
    else:
        X = datagen.anisotropic_mixture(3000, 96, 64, 0.25, False, np.float16, seed=33)
    C, r, iters = 5, 2, 6
    cent, mem, off, (sample, init) = _gpu_partition(X, C, r, iters, seed=34)
    cent_o, _, mem_o, off_o = oracle.partition(X, init, sample, iters, C, r)
    assert np.array_equal(cent.view(np.uint32), cent_o.view(np.uint32))
    assert np.array_equal(off, off_o)
    assert np.array_equal(mem, mem_o)


@pytest.mark.parametrize("kind,d", [("u8", 128), ("f32", 64), ("f16", 700)])
def test_partition_screened_bit_exact(kind, d):
    """More than 32 centroids: tensor-core screening of r + 6 centroids, then d32 of
    those; the result must equal the oracle's full d32 scan (ids, centroids, lists).
    d = 700 streams the K blocks of the vector side."""
    if kind == "u8":
        X = datagen.clustered_u8(6000, d, 64, seed=131)
    elif kind == "f32":
        X = datagen.gaussian_mixture_f32(6000, d, 64, 2.0, seed=132)
    else:
        X = datagen.anisotropic_mixture(4000, d, 64, 0.25, False, np.float16, seed=133)
    C, r, iters = 48, 2, 4
    cent, mem, off, (sample, init) = _gpu_partition(X, C, r, iters, seed=134)
    cent_o, _, mem_o, off_o = oracle.partition(X, init, sample, iters, C, r)
    assert np.array_equal(cent.view(np.uint32), cent_o.view(np.uint32))
    assert np.array_equal(off, off_o)
    assert np.array_equal(mem, mem_o)


def test_partition_edge_cases():
    X = datagen.clustered_u8(700, 16, 4, seed=35)
    for C, r in [(1, 1), (3, 3), (7, 1)]:
        cent, mem, off, (sample, init) = _gpu_partition(X, C, r, 3, seed=36)
        cent_o, _, mem_o, off_o = oracle.partition(X, init, sample, 3, C, r)
        assert np.array_equal(cent.view(np.uint32), cent_o.view(np.uint32))
        assert np.array_equal(off, off_o) and np.array_equal(mem, mem_o)
    # a centroid far from every point leaves its shard empty
    sample = np.arange(700, dtype=np.uint32)
    init = np.vstack([X[:2].astype(np.float32), np.full((1, 16), 1e6, np.float32)])
    cent, mem, off = ann.partition(T(X), 3, 1, T(init), T(sample), 2)
    cent_o, _, mem_o, off_o = oracle.partition(X, init, sample, 2, 3, 1)
    assert np.array_equal(off.cpu().numpy(), off_o) and off_o[3] - off_o[2] == 0
    assert np.array_equal(as_u32(mem), mem_o)


# ------------------------------------------------------------------- shard kNN

def _oracle_shards(X, C, r, seed, iters=4):
    sample, init = _part_inputs(X, C, seed)
    _, _, mem, off = oracle.partition(X, init, sample, iters, C, r)
    return mem, off


@pytest.mark.parametrize("k", [1, 17, 64])
def test_shard_knn_u8_bit_exact(k):
    X = datagen.clustered_u8(3000, 128, 24, seed=41)
    mem, off = _oracle_shards(X, 5, 2, seed=42)
    gid, gd = ann.shard_knn(T(X), T(mem), T(off), k)
    oid, od = oracle.shard_knn(X, mem, off, k)
    assert np.array_equal(as_u32(gid), oid)
    assert np.array_equal(gd.cpu().numpy().astype(np.float64), od)


def test_shard_knn_u8_duplicates_and_small_shards():
    base = datagen.clustered_u8(300, 32, 4, seed=43)
    X = np.vstack([base, base[:100], base[:50]])  # many exact duplicates -> ties by id
    mem, off = _oracle_shards(X, 6, 2, seed=44)
    gid, gd = ann.shard_knn(T(X), T(mem), T(off), 40)
    oid, od = oracle.shard_knn(X, mem, off, 40)
    assert np.array_equal(as_u32(gid), oid)
    assert np.array_equal(gd.cpu().numpy().astype(np.float64), od)
    # shards smaller than k + 1: trailing padding
    Xs = X[:9]
    members = np.array([0, 1, 2, 3, 4, 5, 6, 7, 8, 2, 5], np.uint32)
    offs = np.array([0, 3, 9, 9, 11], np.int64)  # includes an empty shard
    gid, gd = ann.shard_knn(T(Xs), T(members), T(offs), 8)
    oid, od = oracle.shard_knn(Xs, members, offs, 8)
    assert np.array_equal(as_u32(gid), oid)
    assert np.array_equal(gd.cpu().numpy().astype(np.float64), od)


@pytest.mark.parametrize("k,R", [(128, 64), (240, 128)])
def test_paper_degrees_u8_bit_exact(k, R):
    """The paper's build degrees (Sec. VI-B2: intermediate L = 128, final R = 64;
    Table 6 up to 256 / 128): kNN lists of width k = L, the prune to R and the
    merge, bit-exact against the oracle."""
    X = datagen.clustered_u8(4000, 64, 10, seed=141)
    mem, off = _oracle_shards(X, 3, 2, seed=142)
    gid, gd = ann.shard_knn(T(X), T(mem), T(off), k)
    oid, od = oracle.shard_knn(X, mem, off, k)
    assert np.array_equal(as_u32(gid), oid)
    assert np.array_equal(gd.cpu().numpy().astype(np.float64), od)
    pid, pd = ann.prune(gid, gd, T(mem), T(off), R, N=len(X))
    qid, qd = oracle.prune(oid, od, mem, off, R)
    assert np.array_equal(as_u32(pid), qid)
    g, gdist, deg = ann.merge(pid, pd, T(mem), T(off), len(X))
    og, ogd, odeg = oracle.merge(qid, qd, mem, off, len(X))
    assert np.array_equal(as_u32(g), og)


def test_wide_lists_float_rule():
    """FP32 data with k = 128 (screened list k + 16 = 144) and a BF16 screening list
    of 256 re-ranked exactly: the float rule on every row checked."""
    X = datagen.gaussian_mixture_f32(3000, 48, 6, 2.0, seed=143)
    mem, off = _oracle_shards(X, 3, 2, seed=144)
    gid, gd = ann.shard_knn(T(X), T(mem), T(off), 128)
    rows = np.arange(0, len(mem), 7)
    oid, od = oracle.shard_knn(X, mem, off, 128, rows=rows)
    check_float_lists(X, mem[rows], as_u32(gid)[rows], gd.cpu().numpy()[rows], oid, od)
    gid, gd = ann.shard_knn(T(X), T(mem), T(off), 64, ann.BF16_RERANK, 256)
    oid, od = oracle.shard_knn(X, mem, off, 64, rows=rows)
    check_float_lists(X, mem[rows], as_u32(gid)[rows], gd.cpu().numpy()[rows], oid, od)


@pytest.mark.parametrize("d", [256, 258])
@pytest.mark.parametrize("skip", [True, False])
def test_shard_knn_u8_wide_rows_bit_exact(d, skip):
    """uint8 rows up to d = 258, the widest the integer tiles keep exact: the
    extreme rows (all 255 against all 0: distance 255^2 d, the largest key
    magnitudes) and their duplicates give bit-exact ids and distances, with
    the exact tile skipping on and off."""
    X = datagen.clustered_u8(2600, d, 10, seed=45 + d)
    X[:6] = 255
    X[6:12] = 0
    X[12:18, : d // 2] = 255
    X[12:18, d // 2:] = 0
    X[18:24] = X[100:106]  # duplicates of ordinary rows
    n = X.shape[0]
    # shard 0: the 24 special rows alone (all-255 against all-0 in every list);
    # shard 1: every row; shard 2: the extreme rows beside 400 ordinary ones
    parts = [np.arange(24), np.arange(n), np.concatenate([np.arange(12), np.arange(200, 600)])]
    mem = np.concatenate(parts).astype(np.uint32)
    off = np.cumsum([0] + [len(q) for q in parts]).astype(np.int64)
    ann.tile_prune(skip)
    try:
        gid, gd = ann.shard_knn(T(X), T(mem), T(off), 40)
    finally:
        ann.tile_prune(True)
    oid, od = oracle.shard_knn(X, mem, off, 40)
    assert np.array_equal(as_u32(gid), oid)
    assert np.array_equal(gd.cpu().numpy().astype(np.float64), od)
    assert od[np.isfinite(od)].max() == 255.0 ** 2 * d  # all-255 against all-0


@pytest.mark.parametrize("kind,k", [("f32", 32), ("f32", 8), ("f16", 48), ("bf16", 20)])
def test_shard_knn_float_rule(kind, k):
    if kind == "f32":
        X = datagen.gaussian_mixture_f32(3000, 64, seed=45)
        Xt = T(X)
    elif kind == "f16":
        X = datagen.anisotropic_mixture(2500, 96, 64, 0.25, False, np.float16, seed=46)
        Xt = T(X)
    else:
        X = datagen.gaussian_mixture_f32(2500, 40, seed=47)
        Xt = T(X).to(torch.bfloat16)
        X = Xt.float().cpu().numpy()  # the values the bf16 path sees
    mem, off = _oracle_shards(X, 4, 2, seed=48)
    gid, gd = ann.shard_knn(Xt, T(mem), T(off), k)
    oid, od = oracle.shard_knn(X, mem, off, k)
    check_float_lists(X, mem, gid.cpu().numpy(), gd.cpu().numpy(), oid, od)


# ------------------------------------------------------------------ prune / merge

def _oracle_lists(n=2500, d=64, C=4, r=2, k=32, seed=51):
    X = datagen.clustered_u8(n, d, 16, seed=seed)
    mem, off = _oracle_shards(X, C, r, seed + 1)
    oid, od = oracle.shard_knn(X, mem, off, k)
    return X, mem, off, oid, od.astype(np.float32)


@pytest.mark.parametrize("rule,R", [(ann.PRUNE_RANK, 16), (ann.PRUNE_RANK, 5), (ann.PRUNE_TRUNC, 16),
                                    (ann.PRUNE_RANK, 40)])
def test_prune_bit_exact(rule, R):
    X, mem, off, oid, od = _oracle_lists()
    pid, pd = ann.prune(T(oid), T(od), T(mem), T(off), R, rule)
    qid, qd = oracle.prune(oid, od.astype(np.float64), mem, off, R, rule)
    assert np.array_equal(as_u32(pid), qid)
    assert np.array_equal(pd.cpu().numpy().astype(np.float64), qd)


def test_prune_line_example():
    X = np.array([[0], [1], [3], [7]], np.float32)
    mem = np.arange(4, dtype=np.uint32)
    off = np.array([0, 4], np.int64)
    oid, od = oracle.shard_knn(X, mem, off, 3)
    pid, pd = ann.prune(T(oid), T(od.astype(np.float32)), T(mem), T(off), 2)
    assert as_u32(pid).tolist() == [[1, 2], [0, 2], [1, 3], [2, 1]]


@pytest.mark.parametrize("R", [16, 7])
def test_merge_bit_exact(R):
    X, mem, off, oid, od = _oracle_lists(C=5, r=3)
    qid, qd = oracle.prune(oid, od.astype(np.float64), mem, off, R)
    g, gd, deg = ann.merge(T(qid), T(qd.astype(np.float32)), T(mem), T(off), X.shape[0])
    og, ogd, odeg = oracle.merge(qid, qd, mem, off, X.shape[0])
    assert np.array_equal(as_u32(g), og)
    assert np.array_equal(gd.cpu().numpy().astype(np.float64), ogd)
    assert np.array_equal(as_u32(deg), odeg)


# ------------------------------------------------------------------- query side

def test_knn_query_and_medoid_u8():
    X = datagen.clustered_u8(4000, 128, 16, seed=61)
    Q = datagen.clustered_u8(300, 128, 16, seed=62)
    gid, gd = ann.knn_query(T(X), T(Q), 10)
    oid, od = oracle.bruteforce(X, Q, 10)
    assert np.array_equal(as_u32(gid), oid)
    assert np.array_equal(gd.cpu().numpy().astype(np.float64), od)
    assert int(ann.medoid(T(X)).item()) == oracle.medoid(X)


@pytest.mark.parametrize("kind,d,prec", [("f16", 768, ann.EXACT), ("bf16", 1024, ann.EXACT),
                                         ("f32", 640, ann.F16_RERANK), ("f32", 768, ann.EXACT)])
def test_large_d_streamed_tiles_float_rule(kind, d, prec):
    """128 rows of d >= 640 do not fit shared memory: their K blocks stream
    through the ring beside the B blocks (one launch, several shards)."""
    N = 2500
    if kind == "f16":
        X = datagen.anisotropic_mixture(N, d, 32, 0.25, False, np.float16, seed=151)
        Xt = T(X)
    elif kind == "bf16":
        Xt = T(datagen.gaussian_mixture_f32(N, d, 8, seed=152)).to(torch.bfloat16)
        X = Xt.float().cpu().numpy()
    else:
        X = datagen.powerlaw_gaussian(N, d, 0.8, seed=153)
        Xt = T(X)
    mem, off = _oracle_shards(X, 3, 2, seed=154)
    gid, gd = ann.shard_knn(Xt, T(mem), T(off), 16, precision=prec,
                            rerank_k=64 if prec != ann.EXACT else 0)
    oid, od = oracle.shard_knn(X, mem, off, 16)
    check_float_lists(X, mem, gid.cpu().numpy(), gd.cpu().numpy(), oid, od)


def test_knn_query_large_d_f16():
    X = datagen.anisotropic_mixture(3000, 1024, 16, 0.25, False, np.float16, seed=155)
    Q = datagen.anisotropic_mixture(100, 1024, 16, 0.25, False, np.float16, seed=156)
    gid, gd = ann.knn_query(T(X), T(Q), 10)
    oid, od = oracle.bruteforce(X, Q, 10)
    Xq = np.vstack([X, Q])
    check_float_lists(Xq, np.arange(len(X), len(X) + len(Q)), gid.cpu().numpy(),
                      gd.cpu().numpy(), oid, od)


def test_knn_query_f32_rule():
    X = datagen.gaussian_mixture_f32(3000, 48, seed=63)
    Q = datagen.gaussian_mixture_f32(200, 48, seed=64)
    gid, gd = ann.knn_query(T(X), T(Q), 10)
    oid, od = oracle.bruteforce(X, Q, 10)
    # rows are queries: distances are measured from Q
    Xq = np.vstack([X, Q])
    check_float_lists(Xq, np.arange(len(X), len(X) + len(Q)), gid.cpu().numpy(), gd.cpu().numpy(),
                      oid, od)


@pytest.mark.parametrize("kind", ["u8", "f32"])
def test_search_bit_exact(kind):
    if kind == "u8":
        X = datagen.clustered_u8(3000, 64, 16, seed=71)
        Q = datagen.clustered_u8(150, 64, 16, seed=72)
    else:
        X = datagen.gaussian_mixture_f32(3000, 32, seed=73)
        Q = datagen.gaussian_mixture_f32(150, 32, seed=74)
    mem, off = _oracle_shards(X, 4, 2, seed=75)
    oid, od = oracle.shard_knn(X, mem, off, 24)
    qid, qd = oracle.prune(oid, od, mem, off, 12)
    og, ogd, odeg = oracle.merge(qid, qd, mem, off, X.shape[0])
    entry = oracle.medoid(X)
    for Ls in (10, 32, 64):
        gids, gcnt = ann.search(T(og), T(odeg), T(X), T(Q), entry, Ls, 10)
        rids, rcnt = oracle.search(og, odeg, X, Q, entry, Ls, 10)
        assert np.array_equal(as_u32(gids), rids)
        assert np.array_equal(gcnt.cpu().numpy().astype(np.int64), rcnt)
    gt, _ = oracle.bruteforce(X, Q, 10)
    rec = ann.recall(gids, T(gt), 10)
    assert abs(float(rec.item()) - oracle.recall_at(rids, gt)) < 1e-6


@pytest.mark.parametrize("kind", ["u8", "f32"])
def test_search_eval_through_the_c_abi(kind):
    """ann_search_eval (search from the medoid, then recall@10 against brute-force
    truth): ids and distance counts bit-exact against the oracle's search, recall
    equal to the oracle's recall of its own result."""
    if kind == "u8":
        X = datagen.clustered_u8(2500, 64, 16, seed=271)
        Q = datagen.clustered_u8(120, 64, 16, seed=272)
    else:
        X = datagen.gaussian_mixture_f32(2500, 48, seed=273)
        Q = datagen.gaussian_mixture_f32(120, 48, seed=274)
    mem, off = _oracle_shards(X, 4, 2, seed=275)
    oid, od = oracle.shard_knn(X, mem, off, 24)
    qid, qd = oracle.prune(oid, od, mem, off, 12)
    og, ogd, odeg = oracle.merge(qid, qd, mem, off, X.shape[0])
    entry = oracle.medoid(X)
    gt, _ = oracle.bruteforce(X, Q, 10)
    for Ls in (10, 48):
        gids, rec, gcnt = ann.search_eval(T(og), T(odeg), T(X), T(Q), T(gt), entry, Ls)
        rids, rcnt = oracle.search(og, odeg, X, Q, entry, Ls, 10)
        assert np.array_equal(as_u32(gids), rids)
        assert np.array_equal(gcnt.cpu().numpy().astype(np.int64), rcnt)
        assert abs(float(rec.item()) - oracle.recall_at(rids, gt)) < 1e-6
    with pytest.raises(ann.AnnError):  # recall@10 needs a list of at least 10
        ann.search_eval(T(og), T(odeg), T(X), T(Q), T(gt), entry, 8)


@pytest.mark.parametrize("kind", ["u8", "f32"])
def test_search_from_nearest_entry_bit_exact(kind):
    """Each query starts at its nearest listed entry by (d32, id), picked by brute
    force on the host with the oracle's d32; ids >= N in the list are skipped."""
    if kind == "u8":
        X = datagen.clustered_u8(3000, 64, 16, seed=171)
        Q = datagen.clustered_u8(60, 64, 16, seed=172)
    else:
        X = datagen.gaussian_mixture_f32(3000, 32, seed=173)
        Q = datagen.gaussian_mixture_f32(60, 32, seed=174)
    mem, off = _oracle_shards(X, 4, 2, seed=175)
    oid, od = oracle.shard_knn(X, mem, off, 24)
    qid, qd = oracle.prune(oid, od, mem, off, 12)
    og, ogd, odeg = oracle.merge(qid, qd, mem, off, X.shape[0])
    rng = np.random.default_rng(176)
    entries = np.concatenate([rng.choice(len(X), 40, replace=False),
                              [len(X) + 5]]).astype(np.uint32)
    if kind == "u8":  # a listed id twice: computed twice, counted twice
        entries[3] = entries[7]
    Ls = 32
    gids, gcnt = ann.search_entries(T(og), T(odeg), T(X), T(Q), T(entries), Ls, 10)
    gids, gcnt = as_u32(gids), gcnt.cpu().numpy().astype(np.int64)
    valid = [int(e) for e in entries if e < len(X)]
    for qi in range(len(Q)):
        e = min(valid, key=lambda v: (oracle.d32(Q[qi], X[v]), v))
        rids, rcnt = oracle.search(og, odeg, X, Q[qi:qi + 1], e, Ls, 10)
        assert np.array_equal(gids[qi], rids[0])
        assert gcnt[qi] == rcnt[0] + len(valid)


# ------------------------------------------------------------------- end to end

def test_end_to_end_u8_bit_exact():
    X = datagen.clustered_u8(6000, 128, 32, seed=81)
    C, r, k, R, iters = 4, 2, 32, 16, 5
    sample, init = _part_inputs(X, C, 82)
    out = ann.build_index(T(X), ann.BuildConfig(C=C, r=r, k=k, R=R, iters=iters), T(init), T(sample))
    cent_o, _, mem_o, off_o = oracle.partition(X, init, sample, iters, C, r)
    oid, od = oracle.shard_knn(X, mem_o, off_o, k)
    qid, qd = oracle.prune(oid, od, mem_o, off_o, R)
    og, ogd, odeg = oracle.merge(qid, qd, mem_o, off_o, X.shape[0])
    assert np.array_equal(as_u32(out["members"]), mem_o)
    assert np.array_equal(as_u32(out["knn_id"]), oid)
    assert np.array_equal(as_u32(out["pr_id"]), qid)
    assert np.array_equal(as_u32(out["graph"]), og)
    assert np.array_equal(out["gdist"].cpu().numpy().astype(np.float64), ogd)
    assert np.array_equal(as_u32(out["degree"]), odeg)


def test_end_to_end_gauss10k():
    """The small float workload: N=1e4, d=64, C=4, r=2, k=32, R=16."""
    from paper_2605_10135_gb300 import configs
    w = configs.GAUSS_10K
    X = w.vectors()
    sample, init_rows = w.kmeans_inputs()
    init = X[init_rows].astype(np.float32)
    out = ann.build_index(T(X), ann.BuildConfig(C=w.C, r=w.r, k=w.k, R=w.R), T(init), T(sample))
    cent_o, _, mem_o, off_o = oracle.partition(X, init, sample, 10, w.C, w.r)
    assert np.array_equal(as_u32(out["members"]), mem_o)
    oid, od = oracle.shard_knn(X, mem_o, off_o, w.k)
    check_float_lists(X, mem_o, out["knn_id"].cpu().numpy(), out["knn_d"].cpu().numpy(), oid, od)
    g, deg = as_u32(out["graph"]), as_u32(out["degree"])
    assert np.all(deg <= w.R) and not np.any(g == np.arange(w.N)[:, None])


# ------------------------------------------------------------ precision forms

def _recall10(gid, oid):
    hit = 0
    for g, o in zip(gid[:, :10], oid[:, :10]):
        hit += len(set(g.tolist()) & set(o.tolist()) - {PAD})
    return hit / (10 * len(gid))


_FORM = {ann.BF16_RERANK: OP.BF16, ann.F16_RERANK: OP.F16, ann.FP8_RERANK: OP.E4M3}


def _form_recall_matches_its_definition(X, mem, off, prec, kprime, k, gid, rows):
    """The recall a screening form can reach is fixed by its operand rounding: the
    oracle of the precision forms (operands rounded to the form's type, keys in
    FP64, the kprime smallest screened, exact re-rank) gives each sampled row's
    top 10.  The GPU's top 10 equals it on all but a few rows (keys within FP32
    accumulation rounding of the kprime-th screened one may swap), and its recall
    against the exact lists equals the definition's within 0.01.  Returns
    (GPU recall, the definition's recall) on the sampled rows."""
    _, _, rid, _ = OP.screen_rows(X, mem, off, _FORM[prec], kprime, k, rows)
    oid, _ = oracle.shard_knn(X, mem, off, k, rows=rows)
    g10 = gid[rows][:, :10]
    same = np.mean([set(a.tolist()) == set(b.tolist()) for a, b in zip(g10, rid[:, :10])])
    rec_g, rec_e = _recall10(gid[rows], oid), _recall10(rid, oid)
    assert same >= 0.97, same
    assert abs(rec_g - rec_e) <= 0.01, (rec_g, rec_e)
    return rec_g, rec_e


# BF16 and scaled FP16 keep the exact top 10 on these data (bar 0.995); E4M3's
# 3-bit mantissa loses part of it, and its bar is the recall its definition
# reaches on the same rows (oracle/precision.py), checked on every form.
@pytest.mark.parametrize("prec,bar", [(ann.BF16_RERANK, 0.995), (ann.F16_RERANK, 0.995),
                                      (ann.FP8_RERANK, None)])
def test_precision_forms_rerank_exact_distances_and_recall(prec, bar):
    """BF16 / E4M3 screening tiles, FP32 re-rank of the top 128 (Deep-like unit vectors)."""
    X = datagen.anisotropic_mixture(12000, 96, 64, 0.25, True, np.float32, seed=101)
    mem, off = _oracle_shards(X, 4, 2, seed=102)
    k = 64
    gid, gd = ann.shard_knn(T(X), T(mem), T(off), k, precision=prec, rerank_k=128)
    gid, gd = as_u32(gid), gd.cpu().numpy().astype(np.float64)
    for q in range(0, len(mem), 97):  # every returned distance is the exact FP32 one
        u = mem[q]
        ok = gid[q] != PAD
        true_d = ((X[gid[q][ok]].astype(np.float64) - X[u].astype(np.float64)) ** 2).sum(1)
        assert np.all(np.abs(gd[q][ok] - true_d) <= 1e-5 * true_d + 1e-12)
        key = list(zip(gd[q][ok].tolist(), gid[q][ok].tolist()))
        assert key == sorted(key) and u not in gid[q]
    rows = np.arange(0, len(mem), 37)
    rec, _ = _form_recall_matches_its_definition(X, mem, off, prec, 128, k, gid, rows)
    if bar is not None:
        assert rec >= bar, rec


@pytest.mark.parametrize("prec,bar", [(ann.BF16_RERANK, 0.99), (ann.F16_RERANK, 0.995),
                                      (ann.FP8_RERANK, None)])
def test_precision_forms_with_streamed_tiles(prec, bar):
    """d = 768: the screening tiles stream their A blocks too (E4M3 blocks hold 128
    elements); the re-rank still returns exact FP32 distances, sorted."""
    X = datagen.powerlaw_gaussian(3000, 768, 0.8, seed=105)
    mem, off = _oracle_shards(X, 3, 2, seed=106)
    k = 16
    gid, gd = ann.shard_knn(T(X), T(mem), T(off), k, precision=prec, rerank_k=96)
    gid, gd = as_u32(gid), gd.cpu().numpy().astype(np.float64)
    oid, od = oracle.shard_knn(X, mem, off, k)
    for q in range(0, len(mem), 53):
        u = mem[q]
        ok = gid[q] != PAD
        true_d = ((X[gid[q][ok]].astype(np.float64) - X[u].astype(np.float64)) ** 2).sum(1)
        assert np.all(np.abs(gd[q][ok] - true_d) <= 1e-5 * true_d + 1e-12)
        key = list(zip(gd[q][ok].tolist(), gid[q][ok].tolist()))
        assert key == sorted(key) and u not in gid[q]
    rows = np.arange(0, len(mem), 11)
    rec, _ = _form_recall_matches_its_definition(X, mem, off, prec, 96, k, gid, rows)
    if bar is not None:
        assert rec >= bar, rec


def test_screened_lists_before_the_rerank():
    """ann_shard_knn_screen: BF16 screening of uint8 data is exact (its k' = 128
    list equals the oracle's exact 128 nearest bit for bit); E4M3 screening of
    unit vectors returns the screened set and the screening distances of its
    definition (oracle/precision.py) up to FP32 accumulation rounding."""
    X = datagen.clustered_u8(5000, 64, 12, seed=111)
    mem, off = _oracle_shards(X, 3, 2, seed=112)
    cid, cd = ann.shard_knn_screen(T(X), T(mem), T(off), 32, ann.BF16_RERANK, 128)
    assert cid.shape[1] == 128
    oid, od = oracle.shard_knn(X, mem, off, 128)
    assert np.array_equal(as_u32(cid), oid)
    assert np.array_equal(cd.cpu().numpy().astype(np.float64), od)

    Y = datagen.anisotropic_mixture(8000, 96, 32, 0.25, True, np.float32, seed=113)
    mem, off = _oracle_shards(Y, 3, 2, seed=114)
    cid, cd = ann.shard_knn_screen(T(Y), T(mem), T(off), 32, ann.FP8_RERANK, 128)
    cid, cd = as_u32(cid), cd.cpu().numpy().astype(np.float64)
    rows = np.arange(0, len(mem), 41)
    sid, sdist, _, _ = OP.screen_rows(Y, mem, off, OP.E4M3, 128, 32, rows)
    overlap = np.mean([len(set(a[:100].tolist()) & set(b[:100].tolist())) / 100.0
                       for a, b in zip(cid[rows], sid)])
    assert overlap >= 0.97, overlap
    nrm = (Y.astype(np.float64) ** 2).sum(1)
    for r, p in enumerate(rows):
        ref = dict(zip(sid[r].tolist(), sdist[r].tolist()))
        for g, dg in zip(cid[p].tolist(), cd[p].tolist()):
            if g in ref:  # FP32 sums of 96 exact products, norms of scaled vectors
                assert abs(dg - ref[g]) <= 1e-5 * (nrm[mem[p]] + nrm[g]), (g, dg, ref[g])


@pytest.mark.parametrize("prec", [ann.BF16_RERANK, ann.F16_RERANK])
def test_16bit_precision_forms_are_exact_on_uint8(prec):
    """0..255 and their products are exact in BF16 and in power-of-two-scaled FP16."""
    X = datagen.clustered_u8(4000, 128, 16, seed=103)
    mem, off = _oracle_shards(X, 3, 2, seed=104)
    gid, gd = ann.shard_knn(T(X), T(mem), T(off), 32, precision=prec, rerank_k=64)
    oid, od = oracle.shard_knn(X, mem, off, 32)
    assert np.array_equal(as_u32(gid), oid)
    assert np.array_equal(gd.cpu().numpy().astype(np.float64), od)


@pytest.mark.parametrize("kind", ["u8", "f32"])
def test_autotuner_keeps_the_lists_and_records_a_plan(kind):
    """Tuning runs every candidate plan; the lists must be bit-identical to the
    untuned call, and the decision is used by the next call."""
    if kind == "u8":
        X = datagen.clustered_u8(9000, 128, 32, seed=171)
    else:
        X = datagen.gaussian_mixture_f32(9000, 96, 16, seed=172)
    mem, off = _oracle_shards(X, 3, 2, seed=173)
    k = 24
    ann.autotune(-1)
    ref_id, ref_d = ann.shard_knn(T(X), T(mem), T(off), k)
    ann.autotune(1)
    try:
        got_id, got_d = ann.shard_knn(T(X), T(mem), T(off), k)
    finally:
        ann.autotune(0)
    rows = len(mem)
    plan = ann.autotune_lookup(X.shape[1], T(X).dtype, k, ann.EXACT, 0, rows, 3)
    assert plan is not None and plan["tried"] >= 2 and plan["bn"] in (128, 256)
    assert torch.equal(got_id, ref_id) and torch.equal(got_d, ref_d)
    again_id, again_d = ann.shard_knn(T(X), T(mem), T(off), k)   # uses the tuned plan
    assert torch.equal(again_id, ref_id) and torch.equal(again_d, ref_d)
    ann.autotune(-1)


def test_captured_build_replays_match_eager():
    """The whole build captured as one CUDA graph: replays give the eager result,
    also after new vectors are copied into the captured input."""
    from paper_2605_10135_gb300 import configs
    w = configs.GAUSS_10K
    X = w.vectors()
    sample, init_rows = w.kmeans_inputs()
    init = X[init_rows].astype(np.float32)
    cfg = ann.BuildConfig(C=w.C, r=w.r, k=w.k, R=w.R)
    Xd, init_d, samp_d = T(X), T(init), T(sample)
    eager = ann.build_index(Xd.clone(), cfg, init_d, samp_d)
    cap = ann.CapturedBuild(Xd, cfg, init_d, samp_d)
    out = cap.replay()
    torch.cuda.synchronize()
    for key in ("members", "offsets", "knn_id", "graph", "degree"):
        assert torch.equal(out[key], eager[key]), key
    X2 = w.vectors(seed_offset=5)
    eager2 = ann.build_index(T(X2), cfg, init_d, samp_d)
    cap.X.copy_(T(X2))
    out2 = cap.replay()
    torch.cuda.synchronize()
    assert torch.equal(out2["graph"], eager2["graph"])
    assert cap.kernels > 10


def test_bounded_wait_gives_up_and_the_context_stays_usable():
    """A wait on an mbarrier that nothing completes gives up at its limit (or at
    once when the abort flag is set), records the timeout bit and returns."""
    import time
    ann.device_status()
    ann.wait_selftest(0, 20000)
    assert ann.device_status() & 1
    t0 = time.time()
    ann.wait_selftest(1, 2000000)   # abort flag set: no need to wait 2 s
    assert ann.device_status() & 1
    assert time.time() - t0 < 1.0
    X = datagen.clustered_u8(1500, 32, 8, seed=181)
    mem, off = _oracle_shards(X, 2, 1, seed=182)
    gid, gd = ann.shard_knn(T(X), T(mem), T(off), 8)
    oid, od = oracle.shard_knn(X, mem, off, 8)
    assert np.array_equal(as_u32(gid), oid)
    assert ann.device_status() == 0
