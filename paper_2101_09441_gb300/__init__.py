"""GB300-native DBL reachability index (arXiv 2101.09441).

Python binding of ``libdbl.so`` (C ABI in ``include/dbl.h``): argument
marshalling only.  Every step of the index runs in the library's CUDA
kernels; PyTorch provides device memory (through the library's allocator
callbacks) and streams.  There is no CPU fallback: importing works without a
GPU, but every index operation needs the built library and a CUDA device and
raises otherwise.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libdbl.so")

DBL_OK, DBL_ERR_INVALID, DBL_ERR_OOM, DBL_ERR_CUDA, DBL_ERR_TIMEOUT, DBL_ERR_CAPACITY, DBL_ERR_BUSY, \
    DBL_ERR_POISONED, DBL_ERR_CANCELLED, DBL_ERR_IO = range(10)
STATUS_NAMES = ["ok", "invalid", "oom", "cuda", "timeout", "capacity", "busy", "poisoned", "cancelled", "io"]
CODE_UNDECIDED, CODE_SELF, CODE_DL, CODE_BL, CODE_THM1, CODE_THM2, CODE_BFS_POS, CODE_BFS_NEG = range(8)
FLAG_ASYNC, FLAG_PERSISTENT, FLAG_TIMING, FLAG_FINE_L2, FLAG_DEFER = 1, 2, 4, 8, 16
# landmark rankings of dbl_options.landmark_rule: M = |Pre|*|Suc| (Section 4.1), and Table 3's
# A = max, B = min, C = sum of the two degrees
LANDMARK_RULES = {"M": 0, "A": 1, "B": 2, "C": 3}

KERNEL_NAMES = ["propagate", "query_label", "search_expand", "search_other", "insert_append", "insert_seed",
                "build_prep", "other"]

EXPORTS = ["dbl_default_options", "dbl_build", "dbl_insert_edges", "dbl_query", "dbl_query_host",
           "dbl_insert_edges_host", "dbl_labels", "dbl_selection", "dbl_add_vertices", "dbl_snapshot", "dbl_restore", "dbl_sync",
           "dbl_stats", "dbl_phase_trace", "dbl_timings", "dbl_info", "dbl_last_error", "dbl_destroy", "dbl_insert_edges_noalloc",
           "dbl_features", "dbl_coverage", "dbl_select_by_score", "dbl_mlp_create", "dbl_mlp_destroy",
           "dbl_mlp_params", "dbl_mlp_forward", "dbl_mlp_gradients", "dbl_mlp_train_step", "dbl_mlp_sync", "dbl_mlp_last_error",
           "dbl_qctx_create", "dbl_qctx_destroy", "dbl_query_ctx", "dbl_qctx_last_error", "dbl_server_default_options",
           "dbl_server_create", "dbl_server_submit", "dbl_server_wait", "dbl_server_drain", "dbl_server_report",
           "dbl_server_reset_stats", "dbl_server_destroy", "dbl_autotune", "dbl_set_schedule", "dbl_barrier_probe",
           "dbl_server_cancel", "dbl_select_spread", "dbl_select_uncovered", "dbl_save", "dbl_load"]
MLP_PARAMS = 18817


class _ServerOptions(ctypes.Structure):
    _fields_ = [("slots", ctypes.c_int32), ("max_batch", ctypes.c_int64), ("max_pending", ctypes.c_int64),
                ("mem_fraction", ctypes.c_double), ("max_memory", ctypes.c_int64)]


class DblError(RuntimeError):
    def __init__(self, status: int, msg: str):
        self.status = status
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else status}: {msg}")


_ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
_FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)


class _Options(ctypes.Structure):
    _fields_ = [("alloc", _ALLOC_FN), ("free", _FREE_FN), ("ctx", ctypes.c_void_p),
                ("edge_capacity", ctypes.c_int64), ("flags", ctypes.c_int32), ("bfs_words", ctypes.c_int32),
                ("team", ctypes.c_int32), ("query_unroll", ctypes.c_int32), ("search_first_log2", ctypes.c_int32),
                ("landmark_rule", ctypes.c_int32), ("leaf_r", ctypes.c_int64), ("vertex_capacity", ctypes.c_int64),
                ("initial_slots", ctypes.c_int32), ("build_split", ctypes.c_int32), ("build_order", ctypes.c_int32),
                ("search_table_log2", ctypes.c_int32)]


class _Graph(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("m", ctypes.c_int64), ("row_ptr", ctypes.c_void_p),
                ("col", ctypes.c_void_p)]


_lib = None
_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile the CUDA library in-tree (nvcc, sm_103a)."""
    from . import native_build
    return native_build.build(force=force)


def lib():
    """The loaded ``libdbl.so``; raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2101_09441_gb300.build()")
            L = ctypes.CDLL(LIB_PATH)
            P, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
            L.dbl_default_options.argtypes = [P]
            L.dbl_default_options.restype = None
            L.dbl_build.argtypes = [P, P, i32, P, P, i32, P, P, P]
            L.dbl_insert_edges.argtypes = [P, P, P, i64, P]
            L.dbl_query.argtypes = [P, P, P, i64, P, P, P]
            L.dbl_query_host.argtypes = [P, P, P, i64, P, P, P]
            L.dbl_insert_edges_host.argtypes = [P, P, P, i64, P]
            L.dbl_insert_edges_noalloc.argtypes = [P, P, P, i64, P]
            L.dbl_labels.argtypes = [P, P, P, P, P, P]
            L.dbl_selection.argtypes = [P, P, P, P, P]
            L.dbl_add_vertices.argtypes = [P, i64, P, P]
            L.dbl_snapshot.argtypes = [P, ctypes.c_int, P]
            L.dbl_restore.argtypes = [P, ctypes.c_int, P]
            L.dbl_sync.argtypes = [P, P]
            L.dbl_stats.argtypes = [P, P, P]
            L.dbl_phase_trace.argtypes = [P, P, P]
            L.dbl_info.argtypes = [P, P]
            L.dbl_timings.argtypes = [P, P, P, P]
            L.dbl_last_error.argtypes = [P]
            L.dbl_last_error.restype = ctypes.c_char_p
            L.dbl_destroy.argtypes = [P, P]
            L.dbl_destroy.restype = None
            f32 = ctypes.c_float
            L.dbl_autotune.argtypes = [P, P, P, i64, P, P, i64, P, i32, P, P]
            L.dbl_set_schedule.argtypes = [P, i32, i32, i32]
            L.dbl_qctx_create.argtypes = [P, P, P]
            L.dbl_qctx_destroy.argtypes = [P, P]
            L.dbl_qctx_destroy.restype = None
            L.dbl_query_ctx.argtypes = [P, P, P, P, i64, P, P, P]
            L.dbl_qctx_last_error.argtypes = [P]
            L.dbl_qctx_last_error.restype = ctypes.c_char_p
            L.dbl_server_default_options.argtypes = [P]
            L.dbl_server_default_options.restype = None
            L.dbl_server_create.argtypes = [P, P, P]
            L.dbl_server_submit.argtypes = [P, i32, P, P, i64, P, P]
            L.dbl_server_wait.argtypes = [P, ctypes.c_uint64, P]
            L.dbl_server_cancel.argtypes = [P, ctypes.c_uint64]
            L.dbl_barrier_probe.argtypes = [P, i64, i32, P]
            L.dbl_server_drain.argtypes = [P]
            L.dbl_server_report.argtypes = [P, P]
            L.dbl_server_reset_stats.argtypes = [P]
            L.dbl_server_destroy.argtypes = [P]
            L.dbl_server_destroy.restype = None
            L.dbl_features.argtypes = [P, P, P]
            L.dbl_coverage.argtypes = [P, P, P, P, i64, i32, P, P, P, P]
            L.dbl_select_by_score.argtypes = [P, P, i32, P, P]
            L.dbl_select_spread.argtypes = [P, P, i32, P, P]
            L.dbl_select_uncovered.argtypes = [P, P, i32, i32, i32, P, P]
            L.dbl_save.argtypes = [P, ctypes.c_char_p, P]
            L.dbl_load.argtypes = [ctypes.c_char_p, P, P, P]
            L.dbl_mlp_create.argtypes = [P, P, P]
            L.dbl_mlp_destroy.argtypes = [P, P]
            L.dbl_mlp_destroy.restype = None
            L.dbl_mlp_params.argtypes = [P, P, P]
            L.dbl_mlp_forward.argtypes = [P, P, P, i64, P, P]
            L.dbl_mlp_gradients.argtypes = [P, P, P, P, i64, P, P, P]
            L.dbl_mlp_train_step.argtypes = [P, P, P, P, i64, f32, f32, P, P]
            L.dbl_mlp_sync.argtypes = [P, P]
            L.dbl_mlp_last_error.argtypes = [P]
            L.dbl_mlp_last_error.restype = ctypes.c_char_p
            for name in EXPORTS:
                fn = getattr(L, name)
                if fn.restype is ctypes.c_int:  # default restype: dbl_status
                    fn.restype = ctypes.c_int
            _lib = L
    return _lib


def _ptr(t) -> int:
    return 0 if t is None else int(t.data_ptr())


def _stream_handle(stream) -> int:
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream)


class DBLIndex:
    """A DBL index resident on one GPU (see ``include/dbl.h``).

    All tensor arguments are CUDA tensors (int32 ids, uint8 answers) on the
    index's device; they are used on ``stream`` (default: the current one).
    """

    def __init__(self, row_ptr, col, k: int = 64, kprime: int = 64, landmarks=None, leaf_buckets=None,
                 leaf_roles=None, edge_capacity: int = 0, flags: int = 0, team: int = 0, stream=None,
                 torch_allocator: bool = True, query_unroll: int = 0, search_first_log2: int = 0,
                 landmark_rule: str = "M", leaf_r: int = 0, vertex_capacity: int = 0, initial_slots: int = 0,
                 build_split: int = 0, build_order: int = 0, search_table_log2: int = 0):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("DBLIndex needs a CUDA device")
        L = lib()
        self._stream = stream
        self.device = row_ptr.device
        self.row_ptr = row_ptr.to(torch.int32).contiguous()
        self.col = col.to(torch.int32).contiguous()
        self.n = int(self.row_ptr.numel() - 1)
        self.m = int(self.col.numel())
        self.k, self.kprime = int(k), int(kprime)
        opt = self._options(edge_capacity=edge_capacity, flags=flags, team=team, query_unroll=query_unroll,
                            search_first_log2=search_first_log2, landmark_rule=LANDMARK_RULES[landmark_rule],
                            leaf_r=leaf_r, vertex_capacity=vertex_capacity, initial_slots=initial_slots,
                            build_split=build_split, build_order=build_order, search_table_log2=search_table_log2,
                            torch_allocator=torch_allocator)
        self._opt = opt
        g = _Graph(self.n, self.m, _ptr(self.row_ptr), _ptr(self.col))
        self._keep = [t.to(torch.int32).contiguous() if t is not None and t.dtype != torch.uint8 else t
                      for t in (landmarks, leaf_buckets, leaf_roles)]
        lm, lb, lr = self._keep
        h = ctypes.c_void_p()
        st = L.dbl_build(ctypes.byref(g), _ptr(lm), self.k, _ptr(lb), _ptr(lr), self.kprime, ctypes.byref(opt),
                         _stream_handle(stream), ctypes.byref(h))
        if st != DBL_OK:
            raise DblError(st, L.dbl_last_error(None).decode())
        self._h = h

    def _options(self, torch_allocator: bool = True, **fields) -> _Options:
        """dbl_options with the given fields, and (torch_allocator) device
        memory from PyTorch's caching allocator through the callbacks."""
        import torch
        opt = _Options()
        lib().dbl_default_options(ctypes.byref(opt))
        for name, value in fields.items():
            setattr(opt, name, int(value))
        self._refuse = [0, 0]  # allocations to let through, then to refuse (fail_allocations)
        if torch_allocator:
            dev = self.device.index if self.device.index is not None else torch.cuda.current_device()
            refuse = self._refuse

            def _alloc(nbytes, strm, ctx):
                if refuse[1] > 0:
                    if refuse[0] > 0:
                        refuse[0] -= 1
                    else:
                        refuse[1] -= 1
                        return None
                try:
                    return torch.cuda.caching_allocator_alloc(int(nbytes), dev, stream=int(strm or 0))
                except Exception:
                    return None

            def _free(p, nbytes, strm, ctx):
                try:
                    torch.cuda.caching_allocator_delete(int(p))
                except Exception:
                    pass

            self._cb = (_ALLOC_FN(_alloc), _FREE_FN(_free))
            opt.alloc, opt.free = self._cb
        self._opt = opt
        return opt

    def save(self, path: str, stream=None):
        """dbl_save: write the index (graph, choices, labels, inserted edges) to a file."""
        self._check(lib().dbl_save(self._h, os.fsencode(path), self._s(stream)))

    @classmethod
    def load(cls, path: str, device=None, flags: int = 0, team: int = 0, stream=None, torch_allocator: bool = True,
             query_unroll: int = 0, search_first_log2: int = 0, search_table_log2: int = 0) -> "DBLIndex":
        """dbl_load: an index read from a file written by save(), on `device`
        (default: the current CUDA device)."""
        import torch
        self = cls.__new__(cls)
        self._stream = stream
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.row_ptr = self.col = None
        self._keep = []
        opt = self._options(flags=flags, team=team, query_unroll=query_unroll, search_first_log2=search_first_log2,
                            search_table_log2=search_table_log2, torch_allocator=torch_allocator)
        h = ctypes.c_void_p()
        st = lib().dbl_load(os.fsencode(path), ctypes.byref(opt), _stream_handle(stream), ctypes.byref(h))
        if st != DBL_OK:
            raise DblError(st, lib().dbl_last_error(None).decode())
        self._h = h
        info = self.info()
        self.n, self.m, self.k, self.kprime = info["n"], info["m"], info["k"], info["kprime"]
        return self

    def barrier_probe(self, spin_limit: int = 1 << 20, absent_block: int = -1, stream=None):
        """dbl_barrier_probe: one cooperative launch on the index's grid barrier
        in which `absent_block` (-1: none) never arrives and the other blocks
        give up after `spin_limit` polls (then DBL_ERR_TIMEOUT, index poisoned)."""
        self._check(lib().dbl_barrier_probe(self._h, int(spin_limit), int(absent_block), self._s(stream)))

    def fail_allocations(self, count: int = 1, after: int = 0):
        """Make the allocator callback return NULL for `count` device
        allocations the library asks for, after letting the next `after`
        through (host-side fault injection: the library must report
        DBL_ERR_OOM and leave the index unchanged)."""
        self._refuse[0], self._refuse[1] = int(after), int(count)

    # ------------------------------------------------------------------
    def _check(self, st):
        if st != DBL_OK:
            raise DblError(st, lib().dbl_last_error(self._h).decode())

    def _s(self, stream):
        return _stream_handle(stream if stream is not None else self._stream)

    def close(self):
        h = getattr(self, "_h", None)
        if h and _lib is not None:
            _lib.dbl_destroy(h, self._s(None))
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------------
    @staticmethod
    def _pair(a, b):
        """Two equally long int32 device vectors."""
        import torch
        a = a.to(torch.int32).contiguous()
        b = b.to(torch.int32).contiguous()
        if a.numel() != b.numel():
            raise ValueError(f"paired id arrays differ in length ({a.numel()} vs {b.numel()})")
        return a, b

    def insert_edges(self, src, dst, stream=None):
        src, dst = self._pair(src, dst)
        self._check(lib().dbl_insert_edges(self._h, _ptr(src), _ptr(dst), int(src.numel()), self._s(stream)))

    def insert_edges_noalloc(self, src, dst, stream=None):
        """dbl_insert_edges_noalloc: the same insertion without allocating device
        memory (scratch in a fixed library array; at most 2^20 edges per call)."""
        src, dst = self._pair(src, dst)
        self._check(lib().dbl_insert_edges_noalloc(self._h, _ptr(src), _ptr(dst), int(src.numel()),
                                                   self._s(stream)))

    def query(self, u, v, with_code: bool = True, out=None, stream=None):
        """Answer q(u[i], v[i]); returns (ans uint8, code uint8 or None)."""
        import torch
        u, v = self._pair(u, v)
        q = int(u.numel())
        if out is None:
            ans = torch.empty(q, dtype=torch.uint8, device=u.device)
            code = torch.empty(q, dtype=torch.uint8, device=u.device) if with_code else None
        else:
            ans, code = out
        self._check(lib().dbl_query(self._h, _ptr(u), _ptr(v), q, _ptr(ans), _ptr(code), self._s(stream)))
        return ans, code

    def query_host(self, u: np.ndarray, v: np.ndarray, with_code: bool = False, out=None, stream=None):
        """Host-buffer form: numpy in, numpy out (transfers inside the call)."""
        u = np.ascontiguousarray(u, dtype=np.int32)
        v = np.ascontiguousarray(v, dtype=np.int32)
        if u.shape != v.shape:
            raise ValueError("u and v differ in length")
        q = int(u.shape[0])
        if out is None:
            ans = np.empty(q, dtype=np.uint8)
            code = np.empty(q, dtype=np.uint8) if with_code else None
        else:
            ans, code = out
        self._check(lib().dbl_query_host(self._h, u.ctypes.data, v.ctypes.data, q, ans.ctypes.data,
                                         code.ctypes.data if code is not None else None, self._s(stream)))
        return ans, code

    def insert_edges_host(self, src: np.ndarray, dst: np.ndarray, stream=None):
        src = np.ascontiguousarray(src, dtype=np.int32)
        dst = np.ascontiguousarray(dst, dtype=np.int32)
        if src.shape != dst.shape:
            raise ValueError("src and dst differ in length")
        self._check(lib().dbl_insert_edges_host(self._h, src.ctypes.data, dst.ctypes.data, int(src.shape[0]),
                                                self._s(stream)))

    def labels(self, stream=None):
        """(dl_in, dl_out, bl_in, bl_out) as int64 tensors [n, words] (uint64 bit patterns)."""
        import torch
        wd, wb = (self.k + 63) // 64, (self.kprime + 63) // 64
        out = [torch.empty((self.n, w), dtype=torch.int64, device=self.device) for w in (wd, wd, wb, wb)]
        self._check(lib().dbl_labels(self._h, *[_ptr(t) for t in out], self._s(stream)))
        return tuple(out)

    def selection(self, stream=None):
        import torch
        lm = torch.empty(self.k, dtype=torch.int32, device=self.device)
        lb = torch.empty(self.n, dtype=torch.int32, device=self.device)
        lr = torch.empty(self.n, dtype=torch.uint8, device=self.device)
        self._check(lib().dbl_selection(self._h, _ptr(lm), _ptr(lb), _ptr(lr), self._s(stream)))
        return lm, lb, lr

    def snapshot(self, slot: int = 0, stream=None):
        self._check(lib().dbl_snapshot(self._h, slot, self._s(stream)))

    def restore(self, slot: int = 0, stream=None):
        self._check(lib().dbl_restore(self._h, slot, self._s(stream)))
        self.n = self.info()["n"]  # the snapshot's vertex count

    def add_vertices(self, count: int, stream=None) -> int:
        """dbl_add_vertices: `count` isolated vertices with empty labels; returns the first new id."""
        first = ctypes.c_int32(0)
        self._check(lib().dbl_add_vertices(self._h, int(count), ctypes.byref(first), self._s(stream)))
        self.n = self.info()["n"]
        return int(first.value)

    def sync(self, stream=None):
        self._check(lib().dbl_sync(self._h, self._s(stream)))

    def stats(self, stream=None) -> np.ndarray:
        out = np.zeros(16, dtype=np.uint64)
        self._check(lib().dbl_stats(self._h, out.ctypes.data, self._s(stream)))
        return out

    def phase_trace(self, stream=None) -> list:
        """Nanoseconds since the start of the last persistent launch at each of its
        phase marks (start, every grid barrier, end); needs FLAG_TIMING."""
        out = np.zeros(64, dtype=np.int64)
        self._check(lib().dbl_phase_trace(self._h, out.ctypes.data, self._s(stream)))
        return [int(x) for x in out[1:1 + int(out[0])]]

    def timings(self, stream=None) -> dict:
        """Per kernel class: (ms, launches) since the last call (needs FLAG_TIMING)."""
        ms = np.zeros(8, dtype=np.float64)
        cnt = np.zeros(8, dtype=np.uint64)
        self._check(lib().dbl_timings(self._h, ms.ctypes.data, cnt.ctypes.data, self._s(stream)))
        return {name: (float(ms[i]), int(cnt[i])) for i, name in enumerate(KERNEL_NAMES)}

    def info(self) -> dict:
        out = np.zeros(16, dtype=np.int64)
        self._check(lib().dbl_info(self._h, out.ctypes.data))
        return dict(n=int(out[0]), k=int(out[1]), kprime=int(out[2]), edges_stored=int(out[3]),
                    edge_capacity=int(out[4]), m=int(out[5]), record_bytes=int(out[6]), flags=int(out[7]),
                    launches=int(out[8]), half_words=int(out[9]), vertex_capacity=int(out[10]))

    def autotune(self, src, dst, u, v, trials: int = 2, cache: str | None = None, stream=None) -> dict:
        """dbl_autotune on a sample insertion batch and query batch; keeps the
        fastest frontier schedule.  With `cache` (a JSON path), a result stored
        for this graph's (n, m, k, kprime) is applied instead of re-measuring."""
        import json
        import torch
        key = f"{self.n}:{self.m}:{self.k}:{self.kprime}"
        if cache and os.path.exists(cache):
            table = json.load(open(cache))
            if key in table:
                r = table[key]
                self._apply_schedule(int(r["team"]), bool(r["persistent"]), int(r.get("query_unroll", 0)))
                return dict(r, cached=True)
        src, dst = self._pair(src, dst)
        u, v = self._pair(u, v)
        ans = torch.empty(u.numel(), dtype=torch.uint8, device=u.device)
        rep = np.zeros(16, dtype=np.float64)
        self._check(lib().dbl_autotune(self._h, _ptr(src), _ptr(dst), int(src.numel()), _ptr(u), _ptr(v),
                                       int(u.numel()), _ptr(ans), int(trials), rep.ctypes.data, self._s(stream)))
        teams = (1, 4, 8, 16, 32)
        out = {"team": int(rep[10]), "persistent": bool(rep[11]), "best_ms": float(rep[12]),
               "level_ms": {t: float(rep[i]) for i, t in enumerate(teams)},
               "persistent_ms": {t: float(rep[5 + i]) for i, t in enumerate(teams)}}
        if u.numel():
            qms = {qpt: float(rep[13 + i]) for i, qpt in enumerate((1, 2, 4))}
            out["query_unroll_ms"] = qms
            out["query_unroll"] = min(qms, key=qms.get)
        if cache:
            table = json.load(open(cache)) if os.path.exists(cache) else {}
            table[key] = out
            json.dump(table, open(cache, "w"), indent=1)
        return out

    def _apply_schedule(self, team: int, persistent: bool, query_unroll: int = 0):
        self._check(lib().dbl_set_schedule(self._h, int(team), int(persistent), int(query_unroll)))

    def set_schedule(self, team: int, persistent: bool, query_unroll: int = 0):
        """dbl_set_schedule: team width (1, 4, 8, 16, 32), persistent or
        level-by-level frontier loops, label-test pairs per lane group (1, 2, 4; 0 keeps)."""
        self._apply_schedule(team, persistent, query_unroll)

    # ------------------------------------------------------------------ learned scorer
    def features(self, stream=None):
        """dbl_features: bf16 [n, 16] (log1p-scaled per-vertex counts)."""
        import torch
        out = torch.empty((self.n, 16), dtype=torch.bfloat16, device=self.device)
        self._check(lib().dbl_features(self._h, _ptr(out), self._s(stream)))
        return out

    def coverage(self, u, v, reach=None, base_slots: int = 0, stream=None):
        """dbl_coverage: (count int32 [n], target float32 [n], pairs kept)."""
        import torch
        u, v = self._pair(u, v)
        if reach is not None:
            reach = reach.to(torch.uint8).contiguous()
        count = torch.empty(self.n, dtype=torch.int32, device=self.device)
        target = torch.empty(self.n, dtype=torch.float32, device=self.device)
        kept = ctypes.c_int64(0)
        self._check(lib().dbl_coverage(self._h, _ptr(u), _ptr(v), _ptr(reach), int(u.numel()), int(base_slots),
                                       _ptr(count), _ptr(target), ctypes.byref(kept), self._s(stream)))
        return count, target, int(kept.value)

    def select_by_score(self, scores, k: int, stream=None):
        """dbl_select_by_score: the k best-scored vertices (ties by id), int32 [k]."""
        import torch
        scores = scores.to(torch.float32).contiguous()
        out = torch.empty(int(k), dtype=torch.int32, device=self.device)
        self._check(lib().dbl_select_by_score(self._h, _ptr(scores), int(k), _ptr(out), self._s(stream)))
        return out

    def select_uncovered(self, scores, k: int, covered_slots: int, spread: bool = False, stream=None):
        """dbl_select_uncovered: k vertices by score (spread: excluding the
        neighbours of earlier picks), none in the strongly connected component
        of one of the first covered_slots landmarks; int32 [k] (-1 for slots
        left empty)."""
        import torch
        scores = scores.to(torch.float32).contiguous()
        out = torch.empty(int(k), dtype=torch.int32, device=self.device)
        self._check(lib().dbl_select_uncovered(self._h, _ptr(scores), int(k), int(covered_slots), int(bool(spread)),
                                               _ptr(out), self._s(stream)))
        return out

    def select_spread(self, scores, k: int, stream=None):
        """dbl_select_spread: k vertices by score, each excluding its in- and
        out-neighbours from later picks; int32 [k] (-1 for slots left empty)."""
        import torch
        scores = scores.to(torch.float32).contiguous()
        out = torch.empty(int(k), dtype=torch.int32, device=self.device)
        self._check(lib().dbl_select_spread(self._h, _ptr(scores), int(k), _ptr(out), self._s(stream)))
        return out


class QueryContext:
    """dbl_qctx: scratch for one query batch in flight; batches on different
    contexts may run concurrently (different streams / threads)."""

    def __init__(self, ix: "DBLIndex", stream=None):
        self.ix = ix
        h = ctypes.c_void_p()
        st = lib().dbl_qctx_create(ix._h, ctypes.byref(h), _stream_handle(stream))
        if st != DBL_OK:
            raise DblError(st, lib().dbl_last_error(ix._h).decode())
        self._h = h

    def query(self, u, v, with_code: bool = True, stream=None):
        import torch
        u, v = DBLIndex._pair(u, v)
        q = int(u.numel())
        ans = torch.empty(q, dtype=torch.uint8, device=u.device)
        code = torch.empty(q, dtype=torch.uint8, device=u.device) if with_code else None
        st = lib().dbl_query_ctx(self.ix._h, self._h, _ptr(u), _ptr(v), q, _ptr(ans), _ptr(code),
                                 _stream_handle(stream))
        if st != DBL_OK:
            raise DblError(st, lib().dbl_qctx_last_error(self._h).decode())
        return ans, code

    def close(self, stream=None):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.dbl_qctx_destroy(self._h, _stream_handle(stream))
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """dbl_server: continuous-batching request loop over one index (host
    buffers in, host buffers out).  Keep the arrays of a request alive until
    wait() returns for its ticket."""

    def __init__(self, ix: "DBLIndex", slots: int = 4, max_batch: int = 1 << 18, max_pending: int = 1 << 16,
                 mem_fraction: float = 0.5, max_memory: int = 0):
        self.ix = ix
        o = _ServerOptions()
        lib().dbl_server_default_options(ctypes.byref(o))
        o.slots, o.max_batch, o.max_pending, o.mem_fraction = int(slots), int(max_batch), int(max_pending), \
            float(mem_fraction)
        o.max_memory = int(max_memory)
        h = ctypes.c_void_p()
        st = lib().dbl_server_create(ix._h, ctypes.byref(o), ctypes.byref(h))
        if st != DBL_OK:
            raise DblError(st, lib().dbl_last_error(ix._h).decode())
        self._h = h
        self._keep = {}

    def submit(self, kind: int, a: np.ndarray, b: np.ndarray, ans: np.ndarray | None = None) -> int:
        """kind 0: query pairs (answers into ans, uint8); kind 1: insert edges."""
        a = np.ascontiguousarray(a, dtype=np.int32)
        b = np.ascontiguousarray(b, dtype=np.int32)
        if a.shape != b.shape:
            raise ValueError("a and b differ in length")
        if kind == 0 and ans is None:
            ans = np.empty(a.shape[0], dtype=np.uint8)
        t = ctypes.c_uint64(0)
        st = lib().dbl_server_submit(self._h, int(kind), a.ctypes.data, b.ctypes.data, int(a.shape[0]),
                                     ans.ctypes.data if ans is not None else None, ctypes.byref(t))
        if st != DBL_OK:
            raise DblError(st, "server submit")
        self._keep[t.value] = (a, b, ans)
        return int(t.value)

    def wait(self, ticket: int):
        """(answers or None, latency seconds)."""
        lat = ctypes.c_double(0)
        st = lib().dbl_server_wait(self._h, ctypes.c_uint64(ticket), ctypes.byref(lat))
        a, b, ans = self._keep.pop(ticket)
        if st != DBL_OK:
            raise DblError(st, "server request failed")
        return ans, float(lat.value)

    def cancel(self, ticket: int) -> bool:
        """dbl_server_cancel: True if the request was dropped before any slot
        took it (wait() then raises DBL_ERR_CANCELLED), False if too late."""
        st = lib().dbl_server_cancel(self._h, ctypes.c_uint64(ticket))
        if st == DBL_ERR_BUSY:
            return False
        if st != DBL_OK:
            raise DblError(st, "server cancel")
        return True

    def drain(self):
        lib().dbl_server_drain(self._h)

    def report(self) -> dict:
        out = np.zeros(16, dtype=np.float64)
        lib().dbl_server_report(self._h, out.ctypes.data)
        keys = ["query_p50_s", "query_p99_s", "insert_p50_s", "insert_p99_s", "pairs", "edges", "query_requests",
                "insert_requests", "slots", "elapsed_s", "device_batches", "batched_requests", "epochs", "cancelled",
                "slots_admitted", "bytes_per_slot"]
        return {k: float(out[i]) for i, k in enumerate(keys)}

    def reset_stats(self):
        lib().dbl_server_reset_stats(self._h)

    def close(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.dbl_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class MLP:
    """The 16-128-128-1 landmark scorer (dbl_mlp_*): bf16 tensor-core kernels,
    fp32 master weights.  Parameters are a flat float vector in the order
    W1 [16,128], b1, W2 [128,128], b2, w3 [128], b3."""

    def __init__(self, params: np.ndarray, stream=None):
        params = np.ascontiguousarray(params, dtype=np.float32)
        if params.shape != (MLP_PARAMS,):
            raise ValueError(f"expected {MLP_PARAMS} parameters")
        self._stream = stream
        h = ctypes.c_void_p()
        st = lib().dbl_mlp_create(params.ctypes.data, ctypes.byref(h), _stream_handle(stream))
        if st != DBL_OK:
            raise DblError(st, "dbl_mlp_create")
        self._h = h

    def _check(self, st):
        if st != DBL_OK:
            raise DblError(st, lib().dbl_mlp_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.dbl_mlp_destroy(self._h, _stream_handle(self._stream))
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @staticmethod
    def init_params(seed: int) -> np.ndarray:
        """He-normal weights, zero biases (numpy Generator keyed by seed)."""
        rng = np.random.Generator(np.random.PCG64(seed))
        p = np.zeros(MLP_PARAMS, dtype=np.float32)
        p[0:2048] = rng.normal(0, np.sqrt(2 / 16) / 4, 2048)   # features are log-counts up to ~20
        p[2176:2176 + 16384] = rng.normal(0, np.sqrt(2 / 128), 16384)
        p[18688:18816] = rng.normal(0, np.sqrt(1 / 128), 128)
        return p

    def params(self) -> np.ndarray:
        out = np.empty(MLP_PARAMS, dtype=np.float32)
        self._check(lib().dbl_mlp_params(self._h, out.ctypes.data, _stream_handle(self._stream)))
        return out

    def forward(self, X, rows_idx=None, stream=None, out=None, sync=True):
        """Scores of the rows (float32 [rows]); with sync=False the call only
        queues the kernel (errors then surface at the next sync())."""
        import torch
        R = int(rows_idx.numel()) if rows_idx is not None else int(X.shape[0])
        y = out if out is not None else torch.empty(R, dtype=torch.float32, device=X.device)
        self._check(lib().dbl_mlp_forward(self._h, _ptr(X), _ptr(rows_idx), R, _ptr(y),
                                          _stream_handle(stream or self._stream)))
        if sync:
            self.sync(stream)
        return y

    def gradients(self, X, target, rows_idx=None, stream=None):
        import torch
        R = int(rows_idx.numel()) if rows_idx is not None else int(X.shape[0])
        g = torch.empty(MLP_PARAMS, dtype=torch.float32, device=X.device)
        loss = torch.empty(1, dtype=torch.float32, device=X.device)
        self._check(lib().dbl_mlp_gradients(self._h, _ptr(X), _ptr(target), _ptr(rows_idx), R, _ptr(g), _ptr(loss),
                                            _stream_handle(stream or self._stream)))
        self.sync(stream)
        return g, loss

    def sync(self, stream=None):
        """dbl_mlp_sync: wait for the stream and raise if a tensor-core kernel
        gave up a bounded wait."""
        self._check(lib().dbl_mlp_sync(self._h, _stream_handle(stream or self._stream)))

    def train_step(self, X, target, rows_idx=None, lr: float = 0.05, momentum: float = 0.9, loss=None,
                   stream=None):
        R = int(rows_idx.numel()) if rows_idx is not None else int(X.shape[0])
        self._check(lib().dbl_mlp_train_step(self._h, _ptr(X), _ptr(target), _ptr(rows_idx), R, float(lr),
                                             float(momentum), _ptr(loss), _stream_handle(stream or self._stream)))
