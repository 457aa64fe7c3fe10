"""CPU oracle for GVE-LPA (arXiv 2312.08140): test infrastructure only.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` import this package.  The CUDA library never calls it and the two
share no code.  The arithmetic lives in ``lpa_oracle.c`` (plain single-threaded
C, fp64 sums); this module compiles it with gcc and marshals numpy arrays.

Functions and the passages they follow:
  pick(...)            Eq. 2 (Section 3.3) with the strict smallest-id tie-break
                       (Section 4.1.5); scanCommunities of Algorithm 1.
  lpa_sync(...)        Jacobi reading of Algorithm 1 (all vertices read the
                       previous sweep's labels); tolerance and cap of Sections
                       4.1.2-4.1.3.
  lpa_async(...)       Algorithm 1 with one thread in ascending vertex order,
                       vertex pruning (Section 4.1.4).
  lpa_async_ex(...)    the same with options, among them the pruning rule of
                       FLPA (Section 2), and the vertices scanned per sweep.
  modularity(...)      Eq. 1 (Section 3.2), community form, fp64.
  converged(...)       the tolerance test dN / N <= tau of Algorithm 1
                       (Section 4.1.3), decided exactly.
  count_labels_outside_component / count_not_local_max: output checkers.

Parity status: pick, lpa_sync, lpa_async and modularity are pinned by the
hand-worked cases, closed forms, brute-force enumeration and library checks in
``tests/test_oracle_pins.py``.  The labels of the GPU's asynchronous mode are
order-dependent, so only invariants and modularity bounds compare them.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lpa_oracle.c")
_LIB = os.path.join(_HERE, "liblpa_oracle.so")
_lock = threading.Lock()
_lib = None

_i64 = ctypes.c_int64
_ptr = ctypes.c_void_p


def build(force: bool = False) -> str:
    """Compile lpa_oracle.c into liblpa_oracle.so next to it (gcc -O2)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _bind(lib):
    for name in ("oracle_lpa_sync", "oracle_lpa_async", "oracle_lpa_async_order", "oracle_lpa_sync_nonstrict",
                 "oracle_lpa_async_nonstrict", "oracle_lpa_async_ex", "oracle_sync_sweep",
                 "oracle_count_labels_outside_component", "oracle_count_not_local_max", "oracle_converged"):
        getattr(lib, name).restype = _i64
    lib.oracle_pick.restype = ctypes.c_int32
    lib.oracle_pick_nonstrict.restype = ctypes.c_int32
    lib.oracle_modularity.restype = ctypes.c_int
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _bind(ctypes.CDLL(build()))
    return _lib


def load_variant(so_path):
    """Bind another build of lpa_oracle.c (the tests compile deliberately broken
    copies to show that the pins catch them).  Returns an object exposing the
    same functions as this module."""
    lib = _bind(ctypes.CDLL(os.path.abspath(so_path)))

    class _Variant:
        pass

    v = _Variant()
    for name in ("pick", "sync_sweep", "lpa_sync", "lpa_async", "lpa_async_ex", "modularity",
                 "count_labels_outside_component", "count_not_local_max", "converged"):
        fn = globals()[name]
        setattr(v, name, (lambda f: (lambda *a, **k: f(*a, _lib_override=lib, **k)))(fn))
    return v


def _csr(off, idx, w):
    off = np.ascontiguousarray(off, dtype=np.int64)
    idx = np.ascontiguousarray(idx, dtype=np.int32)
    w = None if w is None else np.ascontiguousarray(w, dtype=np.float32)
    n = off.shape[0] - 1
    return n, off, idx, w


def _p(a):
    return None if a is None else a.ctypes.data_as(_ptr)


def _check(ret, what):
    if ret < 0:
        raise ValueError(f"oracle {what} rejected its input (code {ret})")
    return ret


def converged(dN, n, tau, _lib_override=None) -> bool:
    """The tolerance test of Algorithm 1 (Section 4.1.3), dN / N <= tau,
    decided exactly for the binary64 value of tau."""
    lib = _lib_override or _load()
    return bool(_check(lib.oracle_converged(_i64(int(dN)), _i64(int(n)), ctypes.c_double(float(tau))), "converged"))


def pick(off, idx, w, C, i, sweep=None, _lib_override=None) -> int:
    """Eq. 2 for vertex i given labels C; sweep=t (>= 1) selects the non-strict
    tie-break of sweep t, None the strict one."""
    n, off, idx, w = _csr(off, idx, w)
    C = np.ascontiguousarray(C, dtype=np.int32)
    lib = _lib_override or _load()
    if sweep is None:
        return _check(lib.oracle_pick(_i64(n), _p(off), _p(idx), _p(w), _p(C), _i64(i)), "pick")
    return _check(lib.oracle_pick_nonstrict(_i64(n), _p(off), _p(idx), _p(w), _p(C), _i64(i), _i64(sweep)), "pick")


def sync_sweep(off, idx, w, C_in, _lib_override=None):
    """One Jacobi sweep; returns (C_out, dN)."""
    n, off, idx, w = _csr(off, idx, w)
    C_in = np.ascontiguousarray(C_in, dtype=np.int32)
    C_out = np.empty(n, dtype=np.int32)
    dN = _check((_lib_override or _load()).oracle_sync_sweep(_i64(n), _p(off), _p(idx), _p(w), _p(C_in), _p(C_out)),
                "sync_sweep")
    return C_out, dN


def _run(fn, off, idx, w, tau, max_iters):
    n, off, idx, w = _csr(off, idx, w)
    C = np.empty(n, dtype=np.int32)
    hist = np.zeros(max(max_iters, 1), dtype=np.int64)
    it = _check(fn(_i64(n), _p(off), _p(idx), _p(w), ctypes.c_double(float(tau)), _i64(max_iters),
                   _p(C), _p(hist)), "lpa")
    return C, int(it), hist[:it].copy()


def lpa_sync(off, idx, w=None, tau=0.05, max_iters=20, nonstrict=False, _lib_override=None):
    """Synchronous LPA (strict or non-strict tie-break); returns (labels,
    iterations, changed-per-sweep)."""
    lib = _lib_override or _load()
    return _run(lib.oracle_lpa_sync_nonstrict if nonstrict else lib.oracle_lpa_sync, off, idx, w, tau, max_iters)


def lpa_async(off, idx, w=None, tau=0.05, max_iters=20, order=None, nonstrict=False, _lib_override=None):
    """Algorithm 1, one thread; the vertex loop visits `order` (a permutation of
    0..n-1; default ascending) in every sweep; strict or non-strict tie-break.
    Returns (labels, iterations, changed)."""
    lib = _lib_override or _load()
    if order is None and not nonstrict:
        return _run(lib.oracle_lpa_async, off, idx, w, tau, max_iters)
    order = None if order is None else np.ascontiguousarray(order, dtype=np.int64)
    f = lib.oracle_lpa_async_nonstrict if nonstrict else lib.oracle_lpa_async_order
    fn = lambda n, o, i, ww, t, m, C, h: f(n, o, i, ww, t, m, _p(order), C, h)
    return _run(fn, off, idx, w, tau, max_iters)


def lpa_async_ex(off, idx, w=None, tau=0.05, max_iters=20, order=None, nonstrict=False, prune_other=False,
                 _lib_override=None):
    """Algorithm 1, one thread, with options: `prune_other` applies the FLPA
    pruning rule (Section 2: a vertex whose label changes to c marks only the
    neighbours whose label is not c).  Returns (labels, iterations, changed,
    active), active = vertices scanned per sweep."""
    lib = _lib_override or _load()
    n, off, idx, w = _csr(off, idx, w)
    C = np.empty(n, dtype=np.int32)
    hist = np.zeros(max(max_iters, 1), dtype=np.int64)
    act = np.zeros(max(max_iters, 1), dtype=np.int64)
    order = None if order is None else np.ascontiguousarray(order, dtype=np.int64)
    it = _check(lib.oracle_lpa_async_ex(_i64(n), _p(off), _p(idx), _p(w), ctypes.c_double(float(tau)),
                                        _i64(max_iters), _p(order), ctypes.c_int(int(nonstrict)),
                                        ctypes.c_int(int(prune_other)), _p(C), _p(hist), _p(act)), "lpa")
    return C, int(it), hist[:it].copy(), act[:it].copy()


def modularity(off, idx, w, C, _lib_override=None) -> float:
    n, off, idx, w = _csr(off, idx, w)
    C = np.ascontiguousarray(C, dtype=np.int32)
    q = ctypes.c_double(0.0)
    _check((_lib_override or _load()).oracle_modularity(_i64(n), _p(off), _p(idx), _p(w), _p(C), ctypes.byref(q)),
           "modularity")
    return q.value


def count_labels_outside_component(off, idx, C, _lib_override=None) -> int:
    n, off, idx, _ = _csr(off, idx, None)
    C = np.ascontiguousarray(C, dtype=np.int32)
    return _check((_lib_override or _load()).oracle_count_labels_outside_component(_i64(n), _p(off), _p(idx), _p(C)),
                  "component check")


def count_not_local_max(off, idx, w, C, _lib_override=None) -> int:
    n, off, idx, w = _csr(off, idx, w)
    C = np.ascontiguousarray(C, dtype=np.int32)
    return _check((_lib_override or _load()).oracle_count_not_local_max(_i64(n), _p(off), _p(idx), _p(w), _p(C)),
                  "local-max check")
