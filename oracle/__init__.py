"""CPU oracle for the DBL reachability index (arXiv 2101.09441).

TEST INFRASTRUCTURE ONLY: a plain, slow, obviously sequential statement of
what the index computes (``dbl_oracle.c``, plain C), used to check the CUDA
library element by element.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the benchmark's CPU-baseline leg may import it.  It shares no code with the
CUDA library, which never calls it.

Each function cites the passage it follows:

* ``degree_landmarks``  -- Section 4.1, landmark heuristic M(u)=|Pre(u)|*|Suc(u)|.
* ``zero_degree_leaves`` -- Definition 2 (BL label) and the hashing paragraph
  of Section 4.1; h is Fibonacci hashing because the paper leaves it open.
* ``OracleIndex.build`` -- Algorithm 1 and the BL construction paragraph.
* ``OracleIndex.insert_edges`` -- Algorithm 3, its DL_out mirror and the BL
  update of Section 5, one edge at a time.
* ``OracleIndex.query`` -- Algorithm 2 (label tests, Theorems 1-2, pruned BFS).

Pins (``tests/test_oracle_*.py``): brute-force transitive closure by boolean
matrix squaring, the worked example of Figures 1-2, the Lemma 1/2 and Theorem
1/2 invariants, and incremental insertion against a rebuild.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIBDIR = os.path.join(_HERE, "_lib")
_LIB = os.path.join(_LIBDIR, "liborc.so")
_lock = threading.Lock()
_lib = None

# decided-by codes (Algorithm 2 order)
UNDECIDED, SELF, DL, BL, THM1, THM2, BFS_POS, BFS_NEG = range(8)
CODE_NAMES = ["undecided", "self", "dl", "bl", "thm1", "thm2", "bfs_pos", "bfs_neg"]


def build(force: bool = False) -> str:
    """Compile ``dbl_oracle.c`` into ``_lib/liborc.so`` (gcc, OpenMP)."""
    src = os.path.join(_HERE, "dbl_oracle.c")
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(src):
        return _LIB
    os.makedirs(_LIBDIR, exist_ok=True)
    tmp = _LIB + f".{os.getpid()}.tmp"
    subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=gnu11",
                           src, "-o", tmp])
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            P = ctypes.c_void_p
            i32, i64 = ctypes.c_int32, ctypes.c_int64
            lib.orc_create.argtypes = [i32, P, P, i32, i32]
            lib.orc_create.restype = P
            lib.orc_destroy.argtypes = [P]
            lib.orc_destroy.restype = None
            lib.orc_degree_landmarks.argtypes = [P, P]
            lib.orc_zero_degree_leaves.argtypes = [P, P, P]
            lib.orc_rank_landmarks.argtypes = [P, ctypes.c_int, P]
            lib.orc_add_vertices.argtypes = [P, i32]
            lib.orc_threshold_leaves.argtypes = [P, i64, P, P]
            lib.orc_leaf_hash.argtypes = [i32, i32]
            lib.orc_leaf_hash.restype = i32
            lib.orc_build.argtypes = [P, P, P, P, ctypes.c_int]
            lib.orc_insert_edge.argtypes = [P, i32, i32]
            lib.orc_insert_edges.argtypes = [P, P, P, i64]
            lib.orc_query.argtypes = [P, P, P, i64, P, P, P, ctypes.c_int]
            lib.orc_labels.argtypes = [P, P, P, P, P]
            lib.orc_labels.restype = None
            lib.orc_words_dl.argtypes = [P]
            lib.orc_words_dl.restype = i32
            lib.orc_words_bl.argtypes = [P]
            lib.orc_words_bl.restype = i32
            lib.orc_num_edges.argtypes = [P]
            lib.orc_num_edges.restype = i64
            lib.orc_csr.argtypes = [P, P, P]
            lib.orc_csr.restype = None
            lib.orc_insert_stats.argtypes = [P, P]
            lib.orc_insert_stats.restype = None
            lib.orc_mark.argtypes = [P]
            lib.orc_rewind.argtypes = [P]
            _lib = lib
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def leaf_hash(v: int, kprime: int) -> int:
    """Bucket of leaf v: floor(frac(v*phi)*k'), Fibonacci hashing for k'=2^b."""
    return int(_load().orc_leaf_hash(v, kprime))


class OracleIndex:
    """Sequential DBL index on the CPU (see module docstring)."""

    def __init__(self, row_ptr, col, k: int, kprime: int):
        lib = _load()
        self.row_ptr = _i32(row_ptr)
        self.col = _i32(col)
        self.n = int(self.row_ptr.shape[0] - 1)
        self.k, self.kprime = int(k), int(kprime)
        self._h = lib.orc_create(self.n, _p(self.row_ptr), _p(self.col), self.k, self.kprime)
        if not self._h:
            raise ValueError("orc_create failed")
        self.wd = lib.orc_words_dl(self._h)
        self.wb = lib.orc_words_bl(self._h)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and _lib is not None:
            _lib.orc_destroy(h)
            self._h = None

    # selection (Section 4.1, Definition 2)
    def degree_landmarks(self) -> np.ndarray:
        out = np.empty(self.k, dtype=np.int32)
        _load().orc_degree_landmarks(self._h, _p(out))
        return out

    def zero_degree_leaves(self):
        bucket = np.empty(self.n, dtype=np.int32)
        role = np.empty(self.n, dtype=np.uint8)
        _load().orc_zero_degree_leaves(self._h, _p(bucket), _p(role))
        return bucket, role

    # Section 6, "Label Node Selection" (Table 3 rankings, the M(u) <= r leaf rule)
    RULES = {"M": 0, "A": 1, "B": 2, "C": 3}

    def rank_landmarks(self, rule: str = "M") -> np.ndarray:
        """Top-k by M = |Pre|*|Suc| or Table 3's A = max, B = min, C = sum; ties by id."""
        out = np.empty(self.k, dtype=np.int32)
        if _load().orc_rank_landmarks(self._h, self.RULES[rule], _p(out)):
            raise ValueError(f"orc_rank_landmarks failed for rule {rule}")
        return out

    def threshold_leaves(self, r: int):
        """Leaves with M(v) <= r (roles: Definition 2 when M(v) = 0, both otherwise)."""
        bucket = np.empty(self.n, dtype=np.int32)
        role = np.empty(self.n, dtype=np.uint8)
        if _load().orc_threshold_leaves(self._h, int(r), _p(bucket), _p(role)):
            raise ValueError("orc_threshold_leaves: r must be >= 0")
        return bucket, role

    # Algorithm 1
    def build(self, landmarks=None, leaf_bucket=None, leaf_role=None, nthreads: int = 1):
        if landmarks is None:
            landmarks = self.degree_landmarks()
        if leaf_bucket is None:
            leaf_bucket, leaf_role = self.zero_degree_leaves()
        self.landmarks = _i32(landmarks)
        self.leaf_bucket = _i32(leaf_bucket)
        self.leaf_role = np.ascontiguousarray(leaf_role, dtype=np.uint8)
        if self.landmarks.shape[0] != self.k or self.leaf_bucket.shape[0] != self.n:
            raise ValueError("landmarks / leaf arrays have the wrong length")
        rc = _load().orc_build(self._h, _p(self.landmarks), _p(self.leaf_bucket),
                               _p(self.leaf_role), int(nthreads))
        if rc:
            raise ValueError(f"orc_build failed ({rc})")
        return self

    # vertex insertion (Section 1): isolated vertices with empty labels
    def add_vertices(self, count: int) -> int:
        first = self.n
        rc = _load().orc_add_vertices(self._h, int(count))
        if rc:
            raise ValueError(f"orc_add_vertices failed ({rc})")
        self.n += int(count)
        if getattr(self, "leaf_bucket", None) is not None:
            self.leaf_bucket = np.concatenate([self.leaf_bucket, np.full(count, -1, np.int32)])
            self.leaf_role = np.concatenate([self.leaf_role, np.zeros(count, np.uint8)])
        return first

    # Algorithm 3 (+ mirrors), one edge at a time
    def insert_edges(self, src, dst):
        src, dst = _i32(src), _i32(dst)
        rc = _load().orc_insert_edges(self._h, _p(src), _p(dst), int(src.shape[0]))
        if rc:
            raise ValueError(f"orc_insert_edges failed ({rc})")

    def insert_stats(self):
        out = np.zeros(3, dtype=np.uint64)
        _load().orc_insert_stats(self._h, _p(out))
        return dict(skipped=int(out[0]), applied=int(out[1]), visits=int(out[2]))

    # Algorithm 2
    def query(self, u, v, nthreads: int = 1):
        u, v = _i32(u), _i32(v)
        q = int(u.shape[0])
        ans = np.empty(q, dtype=np.uint8)
        code = np.empty(q, dtype=np.uint8)
        stats = np.zeros(10, dtype=np.uint64)
        rc = _load().orc_query(self._h, _p(u), _p(v), q, _p(ans), _p(code), _p(stats), int(nthreads))
        if rc:
            raise ValueError(f"orc_query failed ({rc})")
        self.last_query_stats = stats
        return ans, code

    def mark(self):
        """Remember the current labels and graph (one mark per process)."""
        if _load().orc_mark(self._h):
            raise MemoryError("orc_mark")

    def rewind(self):
        """Return to the state saved by mark()."""
        if _load().orc_rewind(self._h):
            raise ValueError("orc_rewind: no mark for this index")

    def labels(self):
        """(dl_in, dl_out, bl_in, bl_out) as uint64 [n, words]."""
        dl_in = np.empty((self.n, self.wd), dtype=np.uint64)
        dl_out = np.empty((self.n, self.wd), dtype=np.uint64)
        bl_in = np.empty((self.n, self.wb), dtype=np.uint64)
        bl_out = np.empty((self.n, self.wb), dtype=np.uint64)
        _load().orc_labels(self._h, _p(dl_in), _p(dl_out), _p(bl_in), _p(bl_out))
        return dl_in, dl_out, bl_in, bl_out

    def csr(self):
        """Current graph (base + inserted edges) as (row_ptr int64, col int32)."""
        m = int(_load().orc_num_edges(self._h))
        row_ptr = np.empty(self.n + 1, dtype=np.int64)
        col = np.empty(max(m, 1), dtype=np.int32)
        _load().orc_csr(self._h, _p(row_ptr), _p(col))
        return row_ptr, col[:m]
