"""Multi-core CPU label propagation in the paper's own design (Section 4.1:
OpenMP dynamic chunks of 2048 vertices, per-thread collision-free tables,
8-bit flags with vertex pruning), compiled from gve_lpa_omp.c.  A comparison
point for the GPU library, reported by bench.py; not the oracle and not on
the GPU path."""
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gve_lpa_omp.c")
_LIB = os.path.join(_HERE, "libgve_lpa_omp.so")
_lib = None


def build(force=False):
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O3", "-std=gnu11", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        lib.cpu_lpa_run.restype = ctypes.c_int64
        lib.cpu_lpa_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def threads():
    return int(_load().cpu_lpa_threads())


def run(off, idx, w=None, mode="async", tau=0.05, max_iters=20, n_threads=0):
    """Returns (labels, iterations, changed-per-sweep)."""
    off = np.ascontiguousarray(off, dtype=np.int64)
    idx = np.ascontiguousarray(idx, dtype=np.int32)
    w = None if w is None else np.ascontiguousarray(w, dtype=np.float32)
    n = off.shape[0] - 1
    C = np.empty(max(n, 1), dtype=np.int32)
    hist = np.zeros(max(max_iters, 1), dtype=np.int64)
    p = lambda a: None if a is None else a.ctypes.data_as(ctypes.c_void_p)
    it = _load().cpu_lpa_run(ctypes.c_int64(n), p(off), p(idx), p(w), ctypes.c_int(0 if mode == "sync" else 1),
                             ctypes.c_double(tau), ctypes.c_int64(max_iters), ctypes.c_int(n_threads), p(C), p(hist))
    if it < 0:
        raise MemoryError("cpu_lpa_run: allocation failed")
    return C[:n], int(it), hist[:it].copy()
