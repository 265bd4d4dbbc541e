"""Grouped tile launch over shards of uneven sizes (the batched form): one launch
over all shards gives the same lists as one launch per shard, and both follow the
oracle (bit for bit for uint8; the float rule for FP32)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2605_10135_gb300 import ann, build, datagen
from tests.parity import as_u32, check_float_lists

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


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


@pytest.mark.parametrize("kind", ["u8", "f32"])
def test_grouped_launch_equals_one_launch_per_shard(kind):
    n = 12000
    if kind == "u8":
        X = datagen.clustered_u8(n, 96, 24, seed=501)
    else:
        X = datagen.powerlaw_gaussian(n, 160, 0.8, seed=502)
    mem, off = datagen.uneven_shards(n, 16, 2, 60, 4000, seed=503)
    sizes = np.diff(off)
    assert sizes.min() < 200 and sizes.max() > 2500  # uneven, with ragged tails
    k = 24
    gi, gd = ann.shard_knn(T(X), T(mem), T(off), k)
    pi, pd = ann.shard_knn_per_shard(T(X), T(mem), off.tolist(), k)
    assert torch.equal(gi, pi) and torch.equal(gd, pd)
    rows = np.random.default_rng(504).choice(len(mem), 300, replace=False)
    oid, od = oracle.shard_knn(X, mem, off, k, rows=rows)
    if kind == "u8":
        assert np.array_equal(as_u32(gi)[rows], oid)
        assert np.array_equal(gd.cpu().numpy()[rows].astype(np.float64), od)
    else:
        check_float_lists(X, mem[rows], as_u32(gi)[rows], gd.cpu().numpy()[rows], oid, od)


def test_build_from_shards_graph_and_capture():
    """The whole batched build (grouped kNN, prune, merge) over a given uneven
    partition: captured replays equal the eager build, and the merged graph
    equals the oracle's merge of the oracle's pruned lists."""
    n = 6000
    X = datagen.clustered_u8(n, 64, 16, seed=511)
    mem, off = datagen.uneven_shards(n, 8, 2, 100, 3000, seed=512)
    cfg = ann.BuildConfig(C=8, r=2, k=16, R=8)
    out = ann.build_from_shards(T(X), T(mem), T(off), cfg)
    cap = ann.CapturedBuild(T(X), cfg, None, None, shards=(T(mem), T(off), off.tolist()))
    rep = cap.replay()
    torch.cuda.synchronize()
    for key in ("knn_id", "knn_d", "graph", "gdist", "degree"):
        assert torch.equal(out[key], rep[key]), key
    oid, od = oracle.shard_knn(X, mem, off, 16)
    qid, qd = oracle.prune(oid, od, mem, off, 8)
    g, gdist, deg = oracle.merge(qid, qd, mem, off, n)
    assert np.array_equal(as_u32(out["graph"]), g)
    assert np.array_equal(out["degree"].cpu().numpy().astype(np.uint32), deg)
