"""Seeded synthetic graphs shaped like the paper's workloads (Table 1 classes).

This module only draws edges and lays them out as symmetric CSR; it holds no
part of label propagation.  Both the CUDA path (through the tests and
``bench.py``) and the CPU oracle consume its output, so neither side ever
generates its own inputs.

Every graph is undirected and stored with both directions of each edge
(the paper adds reverse edges and uses unit weights, Table 1 caption), rows
sorted ascending, ``int64`` offsets, ``int32`` indices and either no weight
array (unit weights) or ``float32`` integer weights that are symmetric by
construction.

Workload recipes (sizes are the defaults):
  planted_partition  10 blocks x 1000 vertices, pair probabilities 14/999
                     inside a block and 2/9000 across (Poisson(14) intra and
                     Poisson(2) inter neighbours per vertex), unit weights.
  rmat               R-MAT scale s, edge factor f, (a,b,c,d) = (.57,.19,.19,.05),
                     symmetrised, optionally de-duplicated and without
                     self-loops; stands in for the web and social graphs.
  road_grid          rows x cols 4-neighbour lattice, 10% of edges dropped,
                     0.1% shortcuts, integer weights 1..8; stands in for the
                     road and k-mer graphs (mean degree ~3.6).
  batched_sbm        the batched planted-partition distribution: n
                     log-uniform in [100, 200000], 2..64 blocks, mean degree
                     uniform in [4, 64] with 80% of it inside blocks, integer
                     weights 1..4, seed 1000 + g for graph g.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gen.c")
_LIB = os.path.join(_HERE, "liblpa_inputs.so")
_lock = threading.Lock()
_lib = None
_P = ctypes.c_void_p
_i64 = ctypes.c_int64


def build(force: bool = False) -> str:
    """Compile gen.c (gcc -O2 -fopenmp) into liblpa_inputs.so beside it."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-fopenmp", "-fPIC", "-shared",
                               "-ffp-contract=off", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.gen_grid_count.restype = _i64
            lib.csr_dedup.restype = _i64
            _lib = lib
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(_P)


@dataclass
class Graph:
    """Symmetric CSR: off int64[n+1], idx int32[nnz], w float32[nnz] or None (unit)."""
    off: np.ndarray
    idx: np.ndarray
    w: np.ndarray | None
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.off.shape[0] - 1)

    @property
    def nnz(self) -> int:
        return int(self.off[-1])

    def degrees(self) -> np.ndarray:
        return np.diff(self.off)


def from_edges(n, src, dst, *, symmetrise=True, dedup=True, drop_self=True, wmax=0, wseed=0,
               meta=None) -> Graph:
    """Edge list -> symmetric CSR with sorted rows.  wmax > 0 gives integer weights
    uniform in 1..wmax hashed from the unordered vertex pair (symmetric)."""
    lib = _load()
    src = np.ascontiguousarray(src, dtype=np.int32)
    dst = np.ascontiguousarray(dst, dtype=np.int32)
    m = src.shape[0]
    deg = np.zeros(n, dtype=np.int64)
    lib.csr_degrees(_i64(n), _i64(m), _p(src), _p(dst), ctypes.c_int32(int(symmetrise)),
                    ctypes.c_int32(int(drop_self)), _p(deg))
    off = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(deg, out=off[1:])
    idx = np.empty(int(off[-1]), dtype=np.int32)
    lib.csr_fill_sorted(_i64(n), _i64(m), _p(src), _p(dst), ctypes.c_int32(int(symmetrise)),
                        ctypes.c_int32(int(drop_self)), _p(off), _p(deg), _p(idx))
    if dedup:
        nnz = lib.csr_dedup(_i64(n), _p(off), _p(idx), _p(deg))
        idx = idx[:nnz]
    w = None
    if wmax > 0:
        w = np.empty(idx.shape[0], dtype=np.float32)
        lib.csr_pair_weights(_i64(n), _p(off), _p(idx), ctypes.c_int32(wmax), ctypes.c_uint64(wseed),
                             _p(w))
    return Graph(off, idx, w, dict(meta or {}))


def from_undirected_pairs(n, pairs, weights=None) -> Graph:
    """Small helper for hand-built graphs: pairs [(u, v), ...] (each undirected
    edge once; u == v adds a self-loop entry once), optional per-pair weights."""
    rows = [[] for _ in range(n)]
    for k, (u, v) in enumerate(pairs):
        wt = 1.0 if weights is None else float(weights[k])
        rows[u].append((v, wt))
        if u != v:
            rows[v].append((u, wt))
    off = np.zeros(n + 1, dtype=np.int64)
    idx, w = [], []
    for i in range(n):
        for v, wt in sorted(rows[i]):
            idx.append(v)
            w.append(wt)
        off[i + 1] = len(idx)
    return Graph(off, np.asarray(idx, dtype=np.int32),
                 None if weights is None else np.asarray(w, dtype=np.float32), {"kind": "hand"})


def sbm(n, block_sizes, p_in, p_out, seed, wmax=0) -> Graph:
    lib = _load()
    bstart = np.zeros(len(block_sizes) + 1, dtype=np.int64)
    np.cumsum(np.asarray(block_sizes, dtype=np.int64), out=bstart[1:])
    assert bstart[-1] == n
    rowcnt = np.empty(n, dtype=np.int64)
    args = (_i64(n), ctypes.c_int32(len(block_sizes)), _p(bstart), ctypes.c_double(p_in),
            ctypes.c_double(p_out), ctypes.c_uint64(seed))
    lib.gen_sbm_count(*args, _p(rowcnt))
    rowstart = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(rowcnt, out=rowstart[1:])
    m = int(rowstart[-1])
    src = np.empty(m, dtype=np.int32)
    dst = np.empty(m, dtype=np.int32)
    lib.gen_sbm_fill(*args, _p(rowstart), _p(src), _p(dst))
    meta = {"kind": "sbm", "n": n, "blocks": len(block_sizes), "p_in": p_in, "p_out": p_out,
            "seed": seed, "wmax": wmax}
    return from_edges(n, src, dst, symmetrise=True, dedup=False, drop_self=True, wmax=wmax,
                      wseed=seed, meta=meta)


def equal_blocks(n, nb):
    base, extra = divmod(n, nb)
    return [base + (1 if k < extra else 0) for k in range(nb)]


def planted_partition(n=10_000, blocks=10, intra=14.0, inter=2.0, seed=1) -> Graph:
    """Config of 10 blocks x 1000: Poisson(intra) intra- and Poisson(inter) inter-block degree."""
    nb_size = n // blocks
    p_in = intra / (nb_size - 1)
    p_out = inter / (n - nb_size)
    g = sbm(n, equal_blocks(n, blocks), p_in, p_out, seed)
    g.meta.update(kind="planted_partition")
    return g


def rmat(scale, edge_factor=16, a=0.57, b=0.19, c=0.19, seed=1, dedup=True, drop_self=True,
         wmax=0) -> Graph:
    lib = _load()
    n = 1 << scale
    m = edge_factor * n
    src = np.empty(m, dtype=np.int32)
    dst = np.empty(m, dtype=np.int32)
    lib.gen_rmat_edges(ctypes.c_int32(scale), _i64(m), ctypes.c_double(a), ctypes.c_double(b),
                       ctypes.c_double(c), ctypes.c_uint64(seed), _p(src), _p(dst))
    meta = {"kind": "rmat", "scale": scale, "edge_factor": edge_factor, "abcd": [a, b, c, 1 - a - b - c],
            "seed": seed, "dedup": dedup, "drop_self": drop_self}
    g = from_edges(n, src, dst, symmetrise=True, dedup=dedup, drop_self=drop_self, wmax=wmax,
                   wseed=seed, meta=meta)
    del src, dst
    return g


def road_grid(rows=4096, cols=4096, drop=0.10, shortcut=0.001, wmax=8, seed=1) -> Graph:
    lib = _load()
    keep = 1.0 - drop
    kept = lib.gen_grid_count(_i64(rows), _i64(cols), ctypes.c_double(keep), ctypes.c_uint64(seed))
    n_short = int(round(shortcut * kept))
    src = np.empty(kept + n_short, dtype=np.int32)
    dst = np.empty(kept + n_short, dtype=np.int32)
    lib.gen_grid_fill(_i64(rows), _i64(cols), ctypes.c_double(keep), ctypes.c_uint64(seed),
                      _i64(n_short), _p(src), _p(dst))
    meta = {"kind": "road_grid", "rows": rows, "cols": cols, "drop": drop, "shortcut": shortcut,
            "wmax": wmax, "seed": seed}
    return from_edges(rows * cols, src, dst, symmetrise=True, dedup=True, drop_self=True,
                      wmax=wmax, wseed=seed, meta=meta)


def batched_sbm_params(g, n_min=100, n_max=200_000, seed_base=1000):
    """Per-graph draw of the batched distribution: (n, blocks, mean degree)."""
    rng = np.random.default_rng(seed_base + g)
    n = int(round(math.exp(rng.uniform(math.log(n_min), math.log(n_max)))))
    nb = min(int(rng.integers(2, 65)), n)
    d = float(rng.uniform(4.0, 64.0))
    return n, nb, d


def batched_sbm_graph(g, n_min=100, n_max=200_000, seed_base=1000, wmax=4) -> Graph:
    n, nb, d = batched_sbm_params(g, n_min, n_max, seed_base)
    sizes = equal_blocks(n, nb)
    nbs = n / nb
    p_in = min(1.0, 0.8 * d / max(nbs - 1.0, 1.0))
    p_out = min(1.0, 0.2 * d / max(n - nbs, 1.0))
    gr = sbm(n, sizes, p_in, p_out, seed_base + g, wmax=wmax)
    gr.meta.update(kind="batched_sbm", index=g, mean_degree=d)
    return gr


def pack(graphs):
    """Pack graphs back to back: returns (vtx_off int64[G+1], edge_off int64[G+1],
    off int64[N+1] global, idx int32 global ids, w float32 or None)."""
    G = len(graphs)
    vtx_off = np.zeros(G + 1, dtype=np.int64)
    edge_off = np.zeros(G + 1, dtype=np.int64)
    for k, gr in enumerate(graphs):
        vtx_off[k + 1] = vtx_off[k] + gr.n
        edge_off[k + 1] = edge_off[k] + gr.nnz
    N, E = int(vtx_off[-1]), int(edge_off[-1])
    off = np.zeros(N + 1, dtype=np.int64)
    idx = np.empty(E, dtype=np.int32)
    weighted = any(gr.w is not None for gr in graphs)
    w = np.empty(E, dtype=np.float32) if weighted else None
    for k, gr in enumerate(graphs):
        v0, e0 = int(vtx_off[k]), int(edge_off[k])
        off[v0 + 1:v0 + gr.n + 1] = gr.off[1:] + e0
        idx[e0:e0 + gr.nnz] = gr.idx + v0
        if weighted:
            w[e0:e0 + gr.nnz] = 1.0 if gr.w is None else gr.w
    return vtx_off, edge_off, off, idx, w


def random_small(n, p, seed, wmax=0, self_loops=0.0, multi=False) -> Graph:
    """Tiny random undirected graph for brute-force checks (numpy only)."""
    rng = np.random.default_rng(seed)
    pairs = []
    for u in range(n):
        if self_loops and rng.random() < self_loops:
            pairs.append((u, u))
        for v in range(u + 1, n):
            if rng.random() < p:
                pairs.append((u, v))
                if multi and rng.random() < 0.2:
                    pairs.append((u, v))
    weights = None if wmax <= 0 else rng.integers(1, wmax + 1, size=len(pairs)).astype(np.float32)
    g = from_undirected_pairs(n, pairs, weights)
    g.meta.update(kind="random_small", seed=seed, p=p)
    return g


def row_range_sample(g, v0, min_entries):
    """A bounded sample of a large graph for timing CPU code on its rows: the
    rows [v0, v1) of g, v1 the first row boundary at least min_entries entries
    past off[v0] (or the end), as a graph of their own.  Its vertices are the
    sampled vertices and every neighbour of theirs, numbered in increasing
    order of their ids in g; only the sampled rows keep their entries (the
    neighbours' rows are empty).  Returns (graph, v1, ids) with ids[k] the id
    in g of vertex k."""
    n = g.n
    v0 = int(min(max(v0, 0), max(n - 1, 0)))
    e0 = int(g.off[v0])
    v1 = int(np.searchsorted(g.off, e0 + int(min_entries), side="left"))
    v1 = min(max(v1, v0 + 1), n)
    e1 = int(g.off[v1])
    nb = g.idx[e0:e1]
    ids = np.union1d(np.arange(v0, v1, dtype=np.int64), nb.astype(np.int64))
    deg = np.zeros(ids.size, dtype=np.int64)
    deg[np.searchsorted(ids, np.arange(v0, v1, dtype=np.int64))] = np.diff(g.off[v0:v1 + 1])
    off = np.zeros(ids.size + 1, dtype=np.int64)
    np.cumsum(deg, out=off[1:])
    idx = np.searchsorted(ids, nb.astype(np.int64)).astype(np.int32)
    w = None if g.w is None else np.ascontiguousarray(g.w[e0:e1])
    meta = dict(g.meta, sample_rows=(v0, v1), sample_entries=e1 - e0)
    return Graph(off, idx, w, meta), v1, ids
