"""Seeded synthetic inputs for the DBL reachability index.

Shared by the CPU oracle, the tests and the benchmark.  Holds no part of the
index's arithmetic: only graph, insertion-stream and query-stream generation
(R-MAT, splitmix64, Fisher-Yates; see ``rmat.c``).

The workload recipes stand in for the paper's SNAP datasets (Section 6,
Table 2), which are not used here:

* ``tiny``   : scale 14, n = 16,384, m = 80,000, seed 1, 10k insertions,
               100k mixed queries (exact uniform descendants).
* ``social`` : n = 4,847,571, m = 68,993,773 (LJ's size in Table 2), seed 2,
               1M insertions, 10M mixed queries (random-walk descendants).
* ``large``  : n = 2^24, m = 2^28, seed 3.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIBDIR = os.path.join(_HERE, "_lib")
_LIB = os.path.join(_LIBDIR, "libdblgen.so")
_lock = threading.Lock()
_lib = None

RMAT_A, RMAT_B, RMAT_C = 0.57, 0.19, 0.19


def build(force: bool = False) -> str:
    """Compile ``rmat.c`` into ``_lib/libdblgen.so`` (gcc, OpenMP)."""
    src = os.path.join(_HERE, "rmat.c")
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(src):
        return _LIB
    os.makedirs(_LIBDIR, exist_ok=True)
    tmp = _LIB + f".{os.getpid()}.tmp"
    subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                           src, "-o", tmp, "-lm"])
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            P = ctypes.c_void_p
            i32, i64, u64, dbl = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
            lib.dblgen_rmat_csr.argtypes = [i32, i64, dbl, dbl, dbl, u64, P, P]
            lib.dblgen_rmat_csr.restype = ctypes.c_int
            lib.dblgen_insertions.argtypes = [i32, P, P, i64, u64, P, P]
            lib.dblgen_insertions.restype = ctypes.c_int
            lib.dblgen_queries.argtypes = [i32, P, P, i64, P, P, i64, u64, ctypes.c_int, P, P]
            lib.dblgen_queries.restype = ctypes.c_int
            lib.dblgen_loguniform_batches.argtypes = [i64, i64, i64, u64, P, i64]
            lib.dblgen_loguniform_batches.restype = i64
            lib.dblgen_permutation.argtypes = [i32, u64, P]
            lib.dblgen_permutation.restype = ctypes.c_int
            lib.dblgen_splitmix64_at.argtypes = [u64, u64]
            lib.dblgen_splitmix64_at.restype = u64
            lib.dblgen_stream_key.argtypes = [u64, u64]
            lib.dblgen_stream_key.restype = u64
            _lib = lib
    return _lib


def _p(a: np.ndarray | None):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def splitmix64_at(key: int, i: int) -> int:
    """i-th output of splitmix64 started from state ``key``."""
    return int(_load().dblgen_splitmix64_at(key, i))


def permutation(n: int, seed: int) -> np.ndarray:
    out = np.empty(n, dtype=np.int32)
    rc = _load().dblgen_permutation(n, seed, _p(out))
    if rc:
        raise ValueError(f"dblgen_permutation failed ({rc})")
    return out


def rmat_csr(n: int, m: int, seed: int, a: float = RMAT_A, b: float = RMAT_B,
             c: float = RMAT_C) -> tuple[np.ndarray, np.ndarray]:
    """Directed R-MAT graph: (row_ptr int32[n+1], col int32[m]), rows sorted,
    exactly m distinct edges, no self-loops, ids permuted."""
    row_ptr = np.empty(n + 1, dtype=np.int32)
    col = np.empty(max(m, 1), dtype=np.int32)
    rc = _load().dblgen_rmat_csr(n, m, a, b, c, seed, _p(row_ptr), _p(col))
    if rc:
        raise ValueError(f"dblgen_rmat_csr failed ({rc})")
    return row_ptr, col[:m]


def insertions(row_ptr: np.ndarray, col: np.ndarray, count: int, seed: int):
    """``count`` new distinct edges (src, dst), u != v, not already in the graph."""
    n = row_ptr.shape[0] - 1
    src = np.empty(count, dtype=np.int32)
    dst = np.empty(count, dtype=np.int32)
    rc = _load().dblgen_insertions(n, _p(row_ptr), _p(col), count, seed, _p(src), _p(dst))
    if rc:
        raise ValueError(f"dblgen_insertions failed ({rc})")
    return src, dst


def queries(row_ptr: np.ndarray, col: np.ndarray, q: int, seed: int, exact: bool,
            extra_src: np.ndarray | None = None, extra_dst: np.ndarray | None = None):
    """Mixed query stream: even indices uniform pairs, odd indices (u, descendant
    of u) on the graph plus the extra edges."""
    n = row_ptr.shape[0] - 1
    qu = np.empty(q, dtype=np.int32)
    qv = np.empty(q, dtype=np.int32)
    ne = 0 if extra_src is None else int(extra_src.shape[0])
    if ne:
        extra_src = np.ascontiguousarray(extra_src, dtype=np.int32)
        extra_dst = np.ascontiguousarray(extra_dst, dtype=np.int32)
    rc = _load().dblgen_queries(n, _p(row_ptr), _p(col), ne, _p(extra_src) if ne else None,
                                _p(extra_dst) if ne else None, q, seed, int(exact),
                                _p(qu), _p(qv))
    if rc:
        raise ValueError(f"dblgen_queries failed ({rc})")
    return qu, qv


def loguniform_batches(total: int, lo: int, hi: int, seed: int) -> np.ndarray:
    """Batch sizes floor(exp(U[ln lo, ln(hi+1)))) summing to ``total``."""
    cap = total // max(lo, 1) + 16
    out = np.empty(cap, dtype=np.int64)
    nb = _load().dblgen_loguniform_batches(total, lo, hi, seed, _p(out), cap)
    if nb < 0:
        raise ValueError("dblgen_loguniform_batches: capacity")
    return out[:nb].copy()


def uniform_pairs(n: int, q: int, seed: int) -> tuple[np.ndarray, np.ndarray]:
    """q independent uniform pairs (numpy Generator keyed by seed)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return (rng.integers(0, n, q, dtype=np.int64).astype(np.int32),
            rng.integers(0, n, q, dtype=np.int64).astype(np.int32))


def community_dag(n: int, m: int, communities: int, alpha: float, cross: float, seed: int):
    """A graph of `communities` R-MAT communities of power-law sizes
    (size of community c proportional to (c + 1)^-alpha, at least 64
    vertices), each with edges in proportion to its size, plus a share
    `cross` of the m edges between communities, always from a community to
    a later one (so the communities' strongly connected components never
    merge).  Ids are relabelled by a seeded permutation.  Returns
    (row_ptr int32[n+1], col int32[m']) with m' <= m distinct edges, no
    self-loops, rows sorted."""
    w = np.array([(c + 1.0) ** -alpha for c in range(communities)])
    sizes = np.maximum(64, np.floor(w / w.sum() * n)).astype(np.int64)
    sizes[0] += n - sizes.sum()
    off = np.concatenate([[0], np.cumsum(sizes)])
    inner = int(m * (1.0 - cross))
    srcs, dsts = [], []
    for c in range(communities):
        mc = max(1, int(inner * sizes[c] / n))
        mc = min(mc, int(sizes[c]) * (int(sizes[c]) - 1) // 4)
        rp, col = rmat_csr(int(sizes[c]), mc, seed * 1000 + c)
        srcs.append(np.repeat(np.arange(sizes[c], dtype=np.int64), np.diff(rp)) + off[c])
        dsts.append(col.astype(np.int64) + off[c])
    rng = np.random.Generator(np.random.PCG64(seed))
    mx = m - sum(len(x) for x in srcs)
    p = sizes / sizes.sum()
    a = rng.choice(communities, size=2 * mx, p=p)
    b = rng.choice(communities, size=2 * mx, p=p)
    keep = a != b
    a, b = np.minimum(a[keep], b[keep]), np.maximum(a[keep], b[keep])  # from the earlier community
    cs = off[a] + rng.integers(0, sizes[a])
    cd = off[b] + rng.integers(0, sizes[b])
    srcs.append(cs[:mx])
    dsts.append(cd[:mx])
    src, dst = np.concatenate(srcs), np.concatenate(dsts)
    perm = permutation(n, seed + 1).astype(np.int64)
    src, dst = perm[src], perm[dst]
    key = np.unique(src * n + dst)
    src, dst = (key // n), (key % n)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(row_ptr, src + 1, 1)
    return np.cumsum(row_ptr).astype(np.int32), dst.astype(np.int32)


# --------------------------------------------------------------------------
# workload recipes
# --------------------------------------------------------------------------
WORKLOADS = {
    # name: (n, m, seed, insertions, queries, exact descendants)
    "tiny": (16384, 80_000, 1, 10_000, 100_000, True),
    "social": (4_847_571, 68_993_773, 2, 1_000_000, 10_000_000, False),
    "large": (1 << 24, 1 << 28, 3, 1_000_000, 10_000_000, False),
}


def _cache_path(name: str, part: str) -> str | None:
    d = os.environ.get("DBL_INPUT_CACHE")
    if not d:
        return None
    os.makedirs(d, exist_ok=True)
    return os.path.join(d, f"{name}_{part}.npy")


def _cached(name, part, fn):
    p = _cache_path(name, part)
    if p and os.path.exists(p):
        return np.load(p)
    arr = fn()
    if p:
        np.save(p, arr)
    return arr


def workload(name: str, n_insert: int | None = None, n_query: int | None = None,
             with_queries: bool = True) -> dict:
    """Generate (or load from $DBL_INPUT_CACHE) one of the named workloads.

    Returns a dict with n, m, row_ptr, col, ins_src, ins_dst, q_u, q_v.  Queries
    are drawn on the graph after all insertions."""
    n, m, seed, ni, nq, exact = WORKLOADS[name]
    ni = ni if n_insert is None else n_insert
    nq = nq if n_query is None else n_query
    tag = f"{name}"
    g = _cached(tag, "graph", lambda: np.concatenate(rmat_csr(n, m, seed)))
    row_ptr, col = g[: n + 1].copy(), g[n + 1:].copy()
    ins = _cached(f"{tag}_i{ni}", "ins",
                  lambda: np.stack(insertions(row_ptr, col, ni, seed + 100)))
    out = dict(name=name, n=n, m=m, seed=seed, row_ptr=row_ptr, col=col,
               ins_src=ins[0].copy(), ins_dst=ins[1].copy())
    if with_queries:
        qs = _cached(f"{tag}_i{ni}_q{nq}", "qry",
                     lambda: np.stack(queries(row_ptr, col, nq, seed + 200, exact,
                                              ins[0], ins[1])))
        out["q_u"], out["q_v"] = qs[0].copy(), qs[1].copy()
    return out
