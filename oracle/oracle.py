"""numpy front end of the plain-C oracle (TEST INFRASTRUCTURE ONLY).

Each function marshals numpy arrays into ``ann_oracle.c`` and returns numpy
arrays; the arithmetic lives in the C file.  Only the tests, the smoke check
and the CPU-baseline leg of the benchmark import this module.
"""
from __future__ import annotations

import ctypes as ct
import numpy as np

from . import build as _build

PAD = 0xFFFFFFFF
_DT = {np.dtype(np.float32): 0, np.dtype(np.float16): 1, np.dtype(np.uint8): 3}

_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ct.CDLL(_build.build())
        P, I64, I32, D = ct.c_void_p, ct.c_int64, ct.c_int, ct.c_double
        sig = {
            "or_num_threads": (I32, []),
            "or_d64": (D, [P, I32, I64, P, I32, I64, I32]),
            "or_d32": (ct.c_float, [P, I32, I64, P, I32, I64, I32]),
            "or_kmeans": (None, [P, I64, I32, I32, I32, P, P, I64, I32, P, P]),
            "or_assign": (None, [P, I64, I32, I32, P, I32, I32, I32, P]),
            "or_shards": (None, [P, I64, I32, I32, P, P]),
            "or_selective": (None, [P, I64, I32, I32, P, I32, I32, I32, D, D, I64, I64, P, P]),
            "or_shard_knn_rows": (None, [P, I32, I32, P, P, I32, I32, P, I64, P, P]),
            "or_prune": (None, [P, P, P, P, I32, I32, I32, I32, P, P]),
            "or_merge": (None, [P, P, P, P, I32, I64, I32, P, I64, P, P, P]),
            "or_medoid": (I64, [P, I64, I32, I32]),
            "or_prune_alpha": (None, [P, I32, I32, P, P, P, I64, I32, I32, D, P, P]),
            "or_merge_reverse": (None, [P, P, P, I64, I32, P, P, P]),
            "or_search": (None, [P, P, I32, P, I64, I32, I32, P, I32, I64, I64, I32, I32, P, P]),
            "or_bruteforce": (None, [P, I64, I32, I32, P, I32, I64, I32, P, P]),
        }
        for name, (res, args) in sig.items():
            f = getattr(_lib, name)
            f.restype = res
            f.argtypes = args
    return _lib


def _p(a: np.ndarray | None):
    return None if a is None else a.ctypes.data_as(ct.c_void_p)


def _c(a, dtype=None):
    return np.ascontiguousarray(a if dtype is None else np.asarray(a, dtype=dtype))


def dtype_code(x: np.ndarray) -> int:
    return _DT[x.dtype]


def num_threads() -> int:
    return lib().or_num_threads()


def d64(x: np.ndarray, y: np.ndarray) -> float:
    """Squared Euclidean distance of two vectors, FP64."""
    x, y = _c(x), _c(y)
    return lib().or_d64(_p(x), dtype_code(x), 0, _p(y), dtype_code(y), 0, x.shape[-1])


def d32(x: np.ndarray, y: np.ndarray) -> float:
    """Squared Euclidean distance, FP32, terms summed in index order, unfused."""
    x, y = _c(x), _c(y)
    return lib().or_d32(_p(x), dtype_code(x), 0, _p(y), dtype_code(y), 0, x.shape[-1])


def kmeans(X: np.ndarray, init: np.ndarray, sample_idx: np.ndarray, iters: int):
    """Lloyd k-means on the sample rows; returns (centroids f32 [C, d], labels [S])."""
    X = _c(X)
    init = _c(init, np.float32)
    sample_idx = _c(sample_idx, np.uint32)
    C, d = init.shape
    cent = np.empty((C, d), np.float32)
    lab = np.empty(len(sample_idx), np.int32)
    lib().or_kmeans(_p(X), X.shape[0], d, dtype_code(X), C, _p(init), _p(sample_idx),
                    len(sample_idx), iters, _p(cent), _p(lab))
    return cent, lab


def assign(X: np.ndarray, cent: np.ndarray, r: int, use_d64: bool = False) -> np.ndarray:
    """The r nearest centroids of every vector, [N, r] uint32."""
    X = _c(X)
    cent = _c(cent, np.float32)
    out = np.empty((X.shape[0], r), np.uint32)
    lib().or_assign(_p(X), X.shape[0], X.shape[1], dtype_code(X), _p(cent), cent.shape[0], r,
                    int(use_d64), _p(out))
    return out


def shards(assign_: np.ndarray, C: int):
    """Member lists sorted by id per shard: (members [N*r] uint32, offsets [C+1] int64)."""
    a = _c(assign_, np.uint32)
    N, r = a.shape
    members = np.empty(N * r, np.uint32)
    offsets = np.empty(C + 1, np.int64)
    lib().or_shards(_p(a), N, r, C, _p(members), _p(offsets))
    return members, offsets


def selective(X, cent, omega, M=None, eps=float("inf"), tau0=1.0, block=None, cap=0):
    """Blockwise-adaptive assignment with selective replication (Sec. V).

    Returns (assign [N, omega] uint32 with PAD for unused slots, stats [2] int64 =
    (replicas, overflowed originals))."""
    X = _c(X)
    cent = _c(cent, np.float32)
    C = cent.shape[0]
    N = X.shape[0]
    M = C if M is None else M
    block = max(N, 1) if block is None else block
    out = np.empty((N, omega), np.uint32)
    stats = np.zeros(2, np.int64)
    lib().or_selective(_p(X), N, X.shape[1], dtype_code(X), _p(cent), C, omega, M, float(eps),
                       float(tau0), int(block), int(cap), _p(out), _p(stats))
    return out, stats


def partition(X, init, sample_idx, iters, C, r):
    cent, _ = kmeans(X, init, sample_idx, iters)
    a = assign(X, cent, r)
    members, offsets = shards(a, C)
    return cent, a, members, offsets


def shard_knn(X, members, offsets, k, rows=None):
    """Exact kNN inside each shard by (d64, id); rows = member positions (all if None)."""
    X = _c(X)
    members = _c(members, np.uint32)
    offsets = _c(offsets, np.int64)
    C = len(offsets) - 1
    if rows is None:
        n = int(offsets[-1])
        rp = None
    else:
        rp = _c(rows, np.int64)
        n = len(rp)
    ids = np.empty((n, k), np.uint32)
    ds = np.empty((n, k), np.float64)
    lib().or_shard_knn_rows(_p(X), X.shape[1], dtype_code(X), _p(members), _p(offsets), C, k,
                            _p(rp), n, _p(ids), _p(ds))
    return ids, ds


def prune(knn_id, knn_d, members, offsets, R, rule=0):
    """Prune every shard list from k to R entries (rule 0 rank-detour, 1 truncation)."""
    knn_id = _c(knn_id, np.uint32)
    knn_d = _c(knn_d, np.float64)
    members = _c(members, np.uint32)
    offsets = _c(offsets, np.int64)
    rows, k = knn_id.shape
    C = len(offsets) - 1
    pid = np.empty((rows, R), np.uint32)
    pd = np.empty((rows, R), np.float64)
    lib().or_prune(_p(knn_id), _p(knn_d), _p(members), _p(offsets), C, k, R, rule, _p(pid), _p(pd))
    return pid, pd


def merge(pr_id, pr_d, members, offsets, N, gids=None):
    """Dedup-then-reprune union of each vector's shard lists: (graph, gdist, degree)."""
    pr_id = _c(pr_id, np.uint32)
    pr_d = _c(pr_d, np.float64)
    members = _c(members, np.uint32)
    offsets = _c(offsets, np.int64)
    R = pr_id.shape[1]
    C = len(offsets) - 1
    if gids is None:
        gp, ng = None, N
    else:
        gp = _c(gids, np.int64)
        ng = len(gp)
    graph = np.empty((ng, R), np.uint32)
    gd = np.empty((ng, R), np.float64)
    deg = np.empty(ng, np.uint32)
    lib().or_merge(_p(pr_id), _p(pr_d), _p(members), _p(offsets), C, N, R, _p(gp), ng,
                   _p(graph), _p(gd), _p(deg))
    return graph, gd, deg


def prune_alpha(X, knn_id, knn_d, R, alpha=1.2):
    """Occlusion prune of every list from k to R (kept entries in list order)."""
    X = _c(X)
    knn_id = _c(knn_id, np.uint32)
    knn_d = _c(knn_d, np.float64)
    rows, k = knn_id.shape
    pid = np.empty((rows, R), np.uint32)
    pd = np.empty((rows, R), np.float64)
    lib().or_prune_alpha(_p(X), X.shape[1], dtype_code(X), _p(knn_id), _p(knn_d), None, rows, k,
                         R, float(alpha), _p(pid), _p(pd))
    return pid, pd


def merge_reverse(graph, gdist, degree):
    """Merged graph with reverse edges: (graph, gdist, degree)."""
    graph = _c(graph, np.uint32)
    gdist = _c(gdist, np.float64)
    degree = _c(degree, np.uint32)
    N, R = graph.shape
    og = np.empty((N, R), np.uint32)
    od = np.empty((N, R), np.float64)
    odeg = np.empty(N, np.uint32)
    lib().or_merge_reverse(_p(graph), _p(gdist), _p(degree), N, R, _p(og), _p(od), _p(odeg))
    return og, od, odeg


def medoid(X) -> int:
    X = _c(X)
    return int(lib().or_medoid(_p(X), X.shape[0], X.shape[1], dtype_code(X)))


def search(graph, degree, X, Q, entry, Ls, topk=10):
    """Best-first beam search of each query; returns (ids [nq, topk], distance counts [nq])."""
    graph = _c(graph, np.uint32)
    degree = _c(degree, np.uint32)
    X, Q = _c(X), _c(Q)
    nq = Q.shape[0]
    out = np.empty((nq, topk), np.uint32)
    cnt = np.empty(nq, np.int64)
    lib().or_search(_p(graph), _p(degree), graph.shape[1], _p(X), X.shape[0], X.shape[1],
                    dtype_code(X), _p(Q), dtype_code(Q), nq, entry, Ls, topk, _p(out), _p(cnt))
    return out, cnt


def bruteforce(X, Q, k):
    """Exact top-k of each query over all vectors by (d64, id)."""
    X, Q = _c(X), _c(Q)
    nq = Q.shape[0]
    ids = np.empty((nq, k), np.uint32)
    ds = np.empty((nq, k), np.float64)
    lib().or_bruteforce(_p(X), X.shape[0], X.shape[1], dtype_code(X), _p(Q), dtype_code(Q), nq,
                        k, _p(ids), _p(ds))
    return ids, ds


def recall_at(found: np.ndarray, truth: np.ndarray, k: int = 10) -> float:
    """Mean over rows of |first k found  intersect  first k truth| / k."""
    hit = 0
    for f, t in zip(found[:, :k], truth[:, :k]):
        hit += len(set(f.tolist()) & set(t.tolist()) - {PAD})
    return hit / (k * len(found))
