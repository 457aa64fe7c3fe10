"""GPU label propagation (GVE-LPA, arXiv 2312.08140) for GB300: Python binding.

A thin ctypes layer over liblpa.so whose functions carry the names of the C ABI
in include/lpa.h and only marshal arguments: every step of the computation runs
in the library's CUDA kernels.  PyTorch provides device memory and streams.
Importing works without a GPU; calling any lpa_* function needs the built
library (``__graft_entry__.build()``) and raises if it is missing -- there is no
CPU fallback.

Pointer arguments accept a torch tensor (its data_ptr), a numpy array (host
pointer), a raw integer address, or None.  Stream arguments accept None (torch's
current stream when CUDA is available, else the legacy default stream), a
torch.cuda.Stream, or a raw cudaStream_t integer.
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liblpa.so")

LPA_OK = 0
LPA_ERR_INVALID_ARG = 1
LPA_ERR_INVALID_GRAPH = 2
LPA_ERR_OUT_OF_MEMORY = 3
LPA_ERR_CUDA = 4
LPA_ERR_TIMEOUT = 5
LPA_ERR_BUSY = 6
LPA_ERR_NOT_FOUND = 7
LPA_ERR_NOT_READY = 8

LPA_MODE_SYNC = 0
LPA_MODE_ASYNC = 1
LPA_MODE_SYNC_FULL = 2
MODES = {"sync": LPA_MODE_SYNC, "async": LPA_MODE_ASYNC, "sync_full": LPA_MODE_SYNC_FULL}

LPA_HOST_PTRS = 0
LPA_DEVICE_PTRS = 1
LPA_BORROW = 2
LPA_REORDER_DEGREE = 4
LPA_REORDER_SHUFFLE = 8
LPA_KEEP_ORDER = 16
LPA_NONSTRICT = 0x100
LPA_PRUNE_OTHER = 0x200

LPA_MAX_RECORDED_ITERS = 64
LPA_BINS = 5
_H = LPA_MAX_RECORDED_ITERS
_B = LPA_BINS


class LpaRunInfo(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int32), ("exit_reason", ctypes.c_int32),
                ("changed", ctypes.c_int64 * _H), ("active", ctypes.c_int64 * _H),
                ("scanned", ctypes.c_int64 * _H), ("edges_touched", ctypes.c_int64)]

    def as_dict(self):
        it = min(self.iterations, _H)
        return {"iterations": self.iterations, "exit_reason": self.exit_reason,
                "changed": list(self.changed[:it]), "active": list(self.active[:it]),
                "scanned": list(self.scanned[:it]), "edges_touched": self.edges_touched}


class LpaGraphProps(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("nnz", ctypes.c_int64), ("num_graphs", ctypes.c_int32),
                ("weighted", ctypes.c_int32), ("exact", ctypes.c_int32), ("weight_bytes", ctypes.c_int32),
                ("max_degree", ctypes.c_int64), ("device_bytes", ctypes.c_int64),
                ("sweeps_total", ctypes.c_int64), ("scanned_total", ctypes.c_int64),
                ("launches_total", ctypes.c_int64), ("rows_distinct", ctypes.c_int32),
                ("storage_order", ctypes.c_int32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class LpaConfig(ctypes.Structure):
    _fields_ = [("small_max", ctypes.c_int32), ("warp_max", ctypes.c_int32),
                ("mid_max", ctypes.c_int32), ("large_max", ctypes.c_int32),
                ("dense_permille", ctypes.c_int32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class LpaProfile(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int32), ("reserved", ctypes.c_int32), ("init_ms", ctypes.c_float),
                ("finish_ms", ctypes.c_float * _H), ("sweep_ms", (ctypes.c_float * _B) * _H),
                ("bin_vertices", (ctypes.c_int64 * _B) * _H), ("bin_entries", (ctypes.c_int64 * _B) * _H),
                ("bin_changed", (ctypes.c_int64 * _B) * _H), ("bin_changed_entries", (ctypes.c_int64 * _B) * _H)]

    def as_dict(self):
        it = min(self.iterations, _H)
        return {"iterations": self.iterations, "init_ms": self.init_ms,
                "finish_ms": list(self.finish_ms[:it]),
                "sweep_ms": [list(self.sweep_ms[t]) for t in range(it)],
                "bin_vertices": [list(self.bin_vertices[t]) for t in range(it)],
                "bin_entries": [list(self.bin_entries[t]) for t in range(it)],
                "bin_changed": [list(self.bin_changed[t]) for t in range(it)],
                "bin_changed_entries": [list(self.bin_changed_entries[t]) for t in range(it)]}


class LpaAutotuneInfo(ctypes.Structure):
    _fields_ = [("cached", ctypes.c_int32), ("candidates", ctypes.c_int32), ("search_ms", ctypes.c_float),
                ("default_ms", ctypes.c_float), ("chosen_ms", ctypes.c_float), ("sample_graphs", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_ if f != "reserved"}


class LpaServeConfig(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_int64), ("arena_vertices", ctypes.c_int64),
                ("arena_entries", ctypes.c_int64), ("max_slots", ctypes.c_int32), ("mode", ctypes.c_int32),
                ("tolerance", ctypes.c_double), ("max_iters", ctypes.c_int32),
                ("solo_min_entries", ctypes.c_int64)]


class LpaServeStats(ctypes.Structure):
    _fields_ = [("cycles", ctypes.c_int64), ("active", ctypes.c_int32), ("pending", ctypes.c_int32),
                ("arena_bytes", ctypes.c_int64), ("solo_bytes", ctypes.c_int64)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class LpaError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{_STATUS.get(status, status)}: {message}")
        self.status = status
        self.message = message


_STATUS = {0: "ok", 1: "invalid argument", 2: "invalid graph", 3: "out of memory", 4: "CUDA error",
           5: "timeout", 6: "busy", 7: "not found", 8: "not ready"}

_lib = None
_lock = threading.Lock()
_V = ctypes.c_void_p
_I64 = ctypes.c_int64
_I32 = ctypes.c_int32
_U32 = ctypes.c_uint32
_D = ctypes.c_double
_P = ctypes.POINTER

_SIGS = {
    "lpa_version": ([], ctypes.c_char_p),
    "lpa_status_string": ([ctypes.c_int], ctypes.c_char_p),
    "lpa_last_error": ([], ctypes.c_char_p),
    "lpa_graph_create": ([_I64, _I64, _V, _V, _V, _U32, _V, _P(_V)], ctypes.c_int),
    "lpa_graph_destroy": ([_V], ctypes.c_int),
    "lpa_release_cached_memory": ([], ctypes.c_int),
    "lpa_graph_props_get": ([_V, _P(LpaGraphProps)], ctypes.c_int),
    "lpa_graph_get_config": ([_V, _P(LpaConfig)], ctypes.c_int),
    "lpa_graph_set_config": ([_V, _P(LpaConfig)], ctypes.c_int),
    "lpa_graph_debug_stall": ([_V, ctypes.c_int32], ctypes.c_int),
    "lpa_tolerance_threshold": ([_D, _I64, _P(_I64)], ctypes.c_int),
    "lpa_run": ([_V, ctypes.c_int, _D, _I32, _V, _V, _P(LpaRunInfo)], ctypes.c_int),
    "lpa_run_profiled": ([_V, ctypes.c_int, _D, _I32, _V, _V, _P(LpaRunInfo), _P(LpaProfile)], ctypes.c_int),
    "lpa_modularity": ([_V, _V, _P(ctypes.c_double), _V], ctypes.c_int),
    "lpa_modularity_noalloc": ([_I64, _I64, _V, _V, _V, _V, _P(ctypes.c_double), _V], ctypes.c_int),
    "lpa_autotune": ([_V, ctypes.c_int, _D, _I32, _I32, _V, _P(LpaConfig), _P(LpaAutotuneInfo)], ctypes.c_int),
    "lpa_autotune_cache_clear": ([], ctypes.c_int),
    "lpa_batch_autotune": ([_V, ctypes.c_int, _D, _I32, _I32, _I32, _V, _P(LpaConfig), _P(LpaAutotuneInfo)],
                           ctypes.c_int),
    "lpa_batch_get_config": ([_V, _P(LpaConfig)], ctypes.c_int),
    "lpa_batch_set_config": ([_V, _P(LpaConfig)], ctypes.c_int),
    "lpa_batch_create": ([_I32, _V, _V, _V, _V, _V, _U32, _V, _P(_V)], ctypes.c_int),
    "lpa_batch_destroy": ([_V], ctypes.c_int),
    "lpa_batch_props_get": ([_V, _P(LpaGraphProps)], ctypes.c_int),
    "lpa_batch_run": ([_V, ctypes.c_int, _D, _I32, _V, _V, _P(LpaRunInfo)], ctypes.c_int),
    "lpa_batch_modularity": ([_V, _I32, _V, _P(ctypes.c_double), _V], ctypes.c_int),
    "lpa_serve_create": ([_P(LpaServeConfig), _P(_V)], ctypes.c_int),
    "lpa_serve_submit": ([_V, _I64, _I64, _V, _V, _V, _P(ctypes.c_uint64)], ctypes.c_int),
    "lpa_serve_poll": ([_V, _P(ctypes.c_uint64), _I32, _P(_I32)], ctypes.c_int),
    "lpa_serve_fetch": ([_V, ctypes.c_uint64, _V, _P(LpaRunInfo)], ctypes.c_int),
    "lpa_serve_release": ([_V, ctypes.c_uint64], ctypes.c_int),
    "lpa_serve_stats": ([_V, _P(LpaServeStats)], ctypes.c_int),
    "lpa_serve_destroy": ([_V], ctypes.c_int),
}


def exported_symbols():
    """Names of the C entry points this binding expects liblpa.so to export."""
    return sorted(_SIGS)


def load(path: str = LIB_PATH):
    """Load liblpa.so (raises RuntimeError if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(path):
                raise RuntimeError(f"{path} is missing: build it with __graft_entry__.build() "
                                   "(there is no CPU fallback)")
            lib = ctypes.CDLL(path)
            for name, (args, res) in _SIGS.items():
                fn = getattr(lib, name)
                fn.argtypes = args
                fn.restype = res
            _lib = lib
    return _lib


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if hasattr(x, "ctypes"):
        return x.ctypes.data
    raise TypeError(f"cannot pass {type(x)} as a pointer")


def _stream(s):
    if s is None:
        try:
            import torch
            if torch.cuda.is_available() and torch.cuda.is_initialized():
                return torch.cuda.current_stream().cuda_stream
        except Exception:
            pass
        return None
    if isinstance(s, int):
        return s
    return s.cuda_stream


def _check(st):
    if st != LPA_OK:
        msg = load().lpa_last_error().decode()
        raise LpaError(st, msg)


def lpa_version() -> str:
    return load().lpa_version().decode()


def lpa_status_string(st: int) -> str:
    return load().lpa_status_string(st).decode()


def lpa_last_error() -> str:
    return load().lpa_last_error().decode()


def lpa_tolerance_threshold(tolerance, n) -> int:
    """floor(tolerance * n) as the runs compute it: the largest dN that meets
    the tolerance test of Algorithm 1 on an n-vertex graph (no GPU needed)."""
    out = _I64()
    _check(load().lpa_tolerance_threshold(float(tolerance), int(n), ctypes.byref(out)))
    return out.value


def lpa_graph_create(n, nnz, offsets, indices, weights=None, flags=LPA_HOST_PTRS, stream=None):
    h = _V()
    _check(load().lpa_graph_create(n, nnz, _ptr(offsets), _ptr(indices), _ptr(weights), flags,
                                   _stream(stream), ctypes.byref(h)))
    return h.value


def lpa_graph_destroy(g):
    _check(load().lpa_graph_destroy(g))


def lpa_release_cached_memory():
    _check(load().lpa_release_cached_memory())


def lpa_graph_props_get(g) -> dict:
    p = LpaGraphProps()
    _check(load().lpa_graph_props_get(g, ctypes.byref(p)))
    return p.as_dict()


def lpa_graph_get_config(g) -> LpaConfig:
    c = LpaConfig()
    _check(load().lpa_graph_get_config(g, ctypes.byref(c)))
    return c


def lpa_graph_debug_stall(g, block_threads):
    """Test hook: the first block of the next row kernel of `block_threads`
    threads to produce a tile skips that tile's index copy, once (its waits
    give up: LPA_ERR_TIMEOUT)."""
    _check(load().lpa_graph_debug_stall(g, block_threads))


def lpa_graph_set_config(g, cfg: LpaConfig):
    _check(load().lpa_graph_set_config(g, ctypes.byref(cfg)))


_MODE_FLAGS = {"nonstrict": LPA_NONSTRICT, "prune_other": LPA_PRUNE_OTHER}


def _mode(m):
    """"sync", "async", "sync_full", each optionally with "+" suffixes
    "nonstrict" (LPA_NONSTRICT) and "prune_other" (LPA_PRUNE_OTHER), or an
    int."""
    if isinstance(m, str):
        base, *flags = m.split("+")
        if base not in MODES or any(f not in _MODE_FLAGS for f in flags):
            raise ValueError(f"unknown mode {m!r}")
        v = MODES[base]
        for f in flags:
            v |= _MODE_FLAGS[f]
        return v
    return int(m)


def lpa_run(g, mode, tolerance, max_iters, labels_out, stream=None, info=True):
    """Returns an LpaRunInfo when info is True (the call then waits), else None."""
    ri = LpaRunInfo() if info else None
    _check(load().lpa_run(g, _mode(mode), tolerance, max_iters, _ptr(labels_out), _stream(stream),
                          ctypes.byref(ri) if info else None))
    return ri


def lpa_run_profiled(g, mode, tolerance, max_iters, labels_out, stream=None):
    ri, prof = LpaRunInfo(), LpaProfile()
    _check(load().lpa_run_profiled(g, _mode(mode), tolerance, max_iters, _ptr(labels_out), _stream(stream),
                                   ctypes.byref(ri), ctypes.byref(prof)))
    return ri, prof


def lpa_modularity(g, labels, stream=None) -> float:
    q = ctypes.c_double()
    _check(load().lpa_modularity(g, _ptr(labels), ctypes.byref(q), _stream(stream)))
    return q.value


def lpa_modularity_noalloc(n, nnz, offsets, indices, weights, labels, stream=None) -> float:
    """Modularity from caller-owned device CSR and labels; the library allocates
    nothing for it (for callers that may not allocate device memory)."""
    q = ctypes.c_double()
    _check(load().lpa_modularity_noalloc(n, nnz, _ptr(offsets), _ptr(indices), _ptr(weights), _ptr(labels),
                                         ctypes.byref(q), _stream(stream)))
    return q.value


def lpa_autotune(g, mode, tolerance, max_iters, trials=2, stream=None):
    """Returns (LpaConfig chosen, dict of LpaAutotuneInfo)."""
    c, inf = LpaConfig(), LpaAutotuneInfo()
    _check(load().lpa_autotune(g, _mode(mode), tolerance, max_iters, trials, _stream(stream), ctypes.byref(c),
                               ctypes.byref(inf)))
    return c, inf.as_dict()


def lpa_batch_autotune(b, mode, tolerance, max_iters, trials=2, sample_permille=125, stream=None):
    """Returns (LpaConfig chosen, dict of LpaAutotuneInfo)."""
    c, inf = LpaConfig(), LpaAutotuneInfo()
    _check(load().lpa_batch_autotune(b, _mode(mode), tolerance, max_iters, trials, sample_permille,
                                     _stream(stream), ctypes.byref(c), ctypes.byref(inf)))
    return c, inf.as_dict()


def lpa_autotune_cache_clear():
    _check(load().lpa_autotune_cache_clear())


def lpa_batch_get_config(b) -> LpaConfig:
    c = LpaConfig()
    _check(load().lpa_batch_get_config(b, ctypes.byref(c)))
    return c


def lpa_batch_set_config(b, cfg: LpaConfig):
    _check(load().lpa_batch_set_config(b, ctypes.byref(cfg)))


def lpa_batch_create(G, graph_vtx_off, graph_edge_off, offsets, indices, weights=None, flags=LPA_HOST_PTRS,
                     stream=None):
    h = _V()
    _check(load().lpa_batch_create(G, _ptr(graph_vtx_off), _ptr(graph_edge_off), _ptr(offsets), _ptr(indices),
                                   _ptr(weights), flags, _stream(stream), ctypes.byref(h)))
    return h.value


def lpa_batch_destroy(b):
    _check(load().lpa_batch_destroy(b))


def lpa_batch_props_get(b) -> dict:
    p = LpaGraphProps()
    _check(load().lpa_batch_props_get(b, ctypes.byref(p)))
    return p.as_dict()


def lpa_batch_run(b, G, mode, tolerance, max_iters, labels_out, stream=None, info=True):
    """Returns a list of G LpaRunInfo when info is True (the call then waits)."""
    infos = (LpaRunInfo * G)() if info else None
    _check(load().lpa_batch_run(b, _mode(mode), tolerance, max_iters, _ptr(labels_out), _stream(stream),
                                infos))
    return list(infos) if info else None


def lpa_batch_modularity(b, g, labels, stream=None) -> float:
    q = ctypes.c_double()
    _check(load().lpa_batch_modularity(b, g, _ptr(labels), ctypes.byref(q), _stream(stream)))
    return q.value


def lpa_serve_create(hbm_budget_bytes, arena_vertices, arena_entries, max_slots=64, mode="sync",
                     tolerance=0.05, max_iters=20, solo_min_entries=0):
    cfg = LpaServeConfig(hbm_budget_bytes, arena_vertices, arena_entries, max_slots, _mode(mode), tolerance,
                         max_iters, solo_min_entries)
    h = _V()
    _check(load().lpa_serve_create(ctypes.byref(cfg), ctypes.byref(h)))
    return h.value


def lpa_serve_submit(s, n, nnz, offsets, indices, weights=None) -> int:
    """Host arrays in; returns the ticket.  Raises LpaError with status
    LPA_ERR_BUSY when the request does not fit now."""
    t = ctypes.c_uint64()
    _check(load().lpa_serve_submit(s, n, nnz, _ptr(offsets), _ptr(indices), _ptr(weights), ctypes.byref(t)))
    return t.value


def lpa_serve_poll(s, cap=1024):
    buf = (ctypes.c_uint64 * max(cap, 1))()
    k = _I32()
    _check(load().lpa_serve_poll(s, buf, cap, ctypes.byref(k)))
    return list(buf[:k.value])


def lpa_serve_fetch(s, ticket, n):
    """Returns (labels numpy int32[n], LpaRunInfo)."""
    import numpy as np
    lab = np.empty(max(n, 1), dtype=np.int32)
    ri = LpaRunInfo()
    _check(load().lpa_serve_fetch(s, ticket, lab.ctypes.data, ctypes.byref(ri)))
    return lab[:n], ri


def lpa_serve_release(s, ticket):
    _check(load().lpa_serve_release(s, ticket))


def lpa_serve_stats(s) -> dict:
    st = LpaServeStats()
    _check(load().lpa_serve_stats(s, ctypes.byref(st)))
    return st.as_dict()


def lpa_serve_destroy(s):
    _check(load().lpa_serve_destroy(s))


class Graph:
    """Owning wrapper: a graph handle built from host (numpy) or device (torch) CSR."""

    def __init__(self, off, idx, w=None, stream=None):
        n = int(off.shape[0]) - 1
        nnz = int(idx.shape[0])
        dev = hasattr(off, "is_cuda") and off.is_cuda
        self.n, self.nnz = n, nnz
        self.handle = lpa_graph_create(n, nnz, off, idx, w, LPA_DEVICE_PTRS if dev else LPA_HOST_PTRS, stream)

    def run(self, mode="sync", tolerance=0.05, max_iters=20, labels_out=None, stream=None, info=True):
        import torch
        if labels_out is None:
            labels_out = torch.empty(max(self.n, 1), dtype=torch.int32, device="cuda")
        ri = lpa_run(self.handle, mode, tolerance, max_iters, labels_out, stream, info)
        return labels_out[:self.n], (ri.as_dict() if ri is not None else None)

    def modularity(self, labels, stream=None) -> float:
        return lpa_modularity(self.handle, labels, stream)

    def props(self) -> dict:
        return lpa_graph_props_get(self.handle)

    def close(self):
        if self.handle:
            lpa_graph_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
