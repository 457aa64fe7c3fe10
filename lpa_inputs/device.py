"""Seeded synthetic inputs built on the GPU with plain torch operations.

The two largest workloads -- R-MAT scale 27 with edge factor 14 (~3.7e9
directed entries) and the batch of 4,096 planted-partition graphs (~1e8
vertices, ~3.7e9 entries) -- would take minutes and tens of GB of host memory
with the host generators, so they are drawn here, on the device, from the same
recipes (R-MAT: Chakrabarti, Zhan & Faloutsos, SDM 2004; planted partition:
equal blocks, a fixed share of each graph's edges inside blocks) with torch's
seeded CUDA generator.  The random streams differ from the host generators',
so these graphs are not the host ones edge for edge.

Edges are drawn in chunks; each chunk's symmetric (u, v) keys are sorted and
split into buckets by the range of u, each bucket is deduplicated on its own
(every sort stays below 2^31 elements), and the buckets, in order, give the
rows of the CSR with sorted neighbours.

Nothing here computes any part of label propagation: only edges, CSR
structure and integer weights.  Every returned tensor lives on the device;
callers copy to the host what they hand to the oracle.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

CHUNK = 1 << 28                 # edges drawn per step


@dataclass
class DeviceCSR:
    """Symmetric CSR on the device: off int64[n+1], idx int32[nnz], w float32 or None."""
    n: int
    off: "object"
    idx: "object"
    w: "object" = None

    @property
    def nnz(self) -> int:
        return int(self.idx.shape[0])


def _build_csr(torch, n, chunks, nbuckets, device, finish=None):
    """chunks yields (src, dst) int64 device tensors, one direction per edge.
    Both directions are kept, self-loops dropped, duplicates removed.
    finish(u, v) -> (idx_part int32, w_part float32 or None) maps a bucket's
    sorted unique (u, v) to stored entries (default: idx = v, no weights).
    Returns (off int64[n+1], idx int32[E], w float32[E] or None)."""
    width = max(1, -(-n // nbuckets))
    bounds = torch.arange(1, nbuckets, device=device, dtype=torch.int64) * width * n
    parts = [[] for _ in range(nbuckets)]
    for src, dst in chunks:
        keep = src != dst
        keys = torch.cat([(src * n + dst)[keep], (dst * n + src)[keep]])
        del src, dst, keep
        keys, _ = torch.sort(keys)
        cut = torch.searchsorted(keys, bounds).tolist()
        lo = 0
        for b, hi in enumerate(cut + [int(keys.shape[0])]):
            if hi > lo:
                parts[b].append(keys[lo:hi].clone())
            lo = hi
        del keys
    counts = torch.zeros(n, dtype=torch.int64, device=device)
    done = []
    for b in range(nbuckets):
        if not parts[b]:
            continue
        k = torch.unique(torch.cat(parts[b]), sorted=True)
        parts[b] = None
        u = torch.div(k, n, rounding_mode="floor")
        counts += torch.bincount(u, minlength=n)
        done.append(k)
    off = torch.zeros(n + 1, dtype=torch.int64, device=device)
    torch.cumsum(counts, 0, out=off[1:])
    del counts
    E = int(off[-1])
    idx = torch.empty(E, dtype=torch.int32, device=device)
    w = None
    pos = 0
    for j, k in enumerate(done):
        u = torch.div(k, n, rounding_mode="floor")
        v = k - u * n
        done[j] = None
        if finish is None:
            ip, wp = v.to(torch.int32), None
        else:
            ip, wp = finish(u, v)
        idx[pos:pos + k.shape[0]] = ip
        if wp is not None:
            if w is None:
                w = torch.empty(E, dtype=torch.float32, device=device)
            w[pos:pos + k.shape[0]] = wp
        pos += int(k.shape[0])
        del u, v, k, ip, wp
    return off, idx, w


def rmat_device(scale, edge_factor=14, a=0.57, b=0.19, c=0.19, seed=1, device="cuda", nbuckets=64):
    """R-MAT graph: edge_factor * 2^scale directed draws, each choosing one of the
    four quadrants per level with probabilities (a, b, c, 1-a-b-c), then
    symmetrised, self-loops dropped and duplicates removed; unit weights."""
    import torch
    n = 1 << scale
    m = edge_factor * n
    gen = torch.Generator(device=device)
    gen.manual_seed(seed)

    def chunks():
        for s0 in range(0, m, CHUNK):
            k = min(CHUNK, m - s0)
            src = torch.zeros(k, dtype=torch.int64, device=device)
            dst = torch.zeros(k, dtype=torch.int64, device=device)
            for level in range(scale):
                r = torch.rand(k, generator=gen, device=device)
                bit = 1 << (scale - 1 - level)
                src += (r >= a + b).to(torch.int64) * bit                          # quadrants c, d
                dst += (((r >= a) & (r < a + b)) | (r >= a + b + c)).to(torch.int64) * bit   # b, d
                del r
            yield src, dst

    off, idx, _ = _build_csr(torch, n, chunks(), nbuckets, device)
    return DeviceCSR(n, off, idx, None)


def _pair_weights(torch, u, v, wmax, seed):
    """Integer weights uniform in 1..wmax from a hash of the unordered pair, so
    w(u, v) == w(v, u)."""
    lo = torch.minimum(u, v)
    hi = torch.maximum(u, v)
    h = lo * 0x9E3779B1 + hi * 0x85EBCA77 + seed * 0xC2B2AE3D
    h = h ^ (h >> 29)
    h = h * 0x27D4EB2F
    h = h ^ (h >> 31)
    return (torch.remainder(h, wmax) + 1).to(torch.float32)


def batched_params(G=4096, n_min=100, n_max=200_000, seed_base=1000):
    """Per-graph (n, blocks, mean degree): n log-uniform in [n_min, n_max], blocks
    uniform in [2, 64], mean degree uniform in [4, 64] (numpy, seed_base + g)."""
    params = []
    for g in range(G):
        rng = np.random.default_rng(seed_base + g)
        n = int(round(math.exp(rng.uniform(math.log(n_min), math.log(n_max)))))
        nb = min(int(rng.integers(2, 65)), n)
        d = float(rng.uniform(4.0, 64.0))
        params.append((n, nb, d))
    return params


def batched_planted_partition_device(G=4096, n_min=100, n_max=200_000, seed_base=1000, wmax=4,
                                     intra=0.8, device="cuda", nbuckets=16):
    """G planted-partition graphs packed back to back.  Graph g has the
    parameters of batched_params; its vertices are split into equal blocks and
    it gets round(n d / 2) undirected edge draws, a share `intra` of them
    between two vertices of one block and the rest between blocks, endpoints
    uniform; then symmetrised, self-loops dropped, duplicates removed, integer
    weights 1..wmax.

    Returns (vtx_off int64[G+1] host, edge_off int64[G+1] host, off int64[N+1]
    device (global positions), idx int32[E] device (graph-local ids),
    w float32[E] device, params)."""
    import torch
    params = batched_params(G, n_min, n_max, seed_base)
    ns = np.array([p[0] for p in params], dtype=np.int64)
    nbs = np.array([p[1] for p in params], dtype=np.int64)
    ms = np.array([int(round(p[0] * p[2] / 2.0)) for p in params], dtype=np.int64)
    vtx_off = np.zeros(G + 1, dtype=np.int64)
    np.cumsum(ns, out=vtx_off[1:])
    N = int(vtx_off[-1])
    gen = torch.Generator(device=device)
    gen.manual_seed(seed_base)
    dev = lambda a: torch.from_numpy(a).to(device)
    ns_d, nbs_d, vo_d = dev(ns), dev(nbs), dev(vtx_off)
    edge_graph_off = np.zeros(G + 1, dtype=np.int64)
    np.cumsum(ms, out=edge_graph_off[1:])
    ego_d = dev(edge_graph_off)
    M = int(edge_graph_off[-1])

    def chunks():
        for s0 in range(0, M, CHUNK):
            k = min(CHUNK, M - s0)
            e = torch.arange(s0, s0 + k, device=device, dtype=torch.int64)
            gid = torch.searchsorted(ego_d, e, right=True) - 1          # graph of each draw
            del e
            n_e = ns_d[gid]
            nb_e = nbs_d[gid]
            base = torch.div(n_e, nb_e, rounding_mode="floor")
            extra = n_e - base * nb_e                                   # the first `extra` blocks hold base + 1
            u = torch.minimum((torch.rand(k, generator=gen, device=device, dtype=torch.float64) * n_e).long(),
                              n_e - 1)
            cut = extra * (base + 1)
            blk = torch.where(u < cut, torch.div(u, base + 1, rounding_mode="floor"),
                              extra + torch.div(u - cut, torch.clamp(base, min=1), rounding_mode="floor"))
            first = blk < extra
            bstart = torch.where(first, blk * (base + 1), cut + (blk - extra) * base)
            bsize = torch.where(first, base + 1, base)
            del blk, first, cut, base, extra, nb_e
            r = torch.rand(k, generator=gen, device=device, dtype=torch.float64)
            inside = torch.rand(k, generator=gen, device=device) < intra
            v_in = bstart + torch.minimum((r * bsize).long(), bsize - 1)
            outside = torch.clamp(n_e - bsize, min=1)
            o = torch.minimum((r * outside).long(), outside - 1)
            v_out = torch.where(o < bstart, o, o + bsize)
            v = torch.where(inside | (n_e == bsize), v_in, v_out)
            del r, inside, v_in, v_out, o, outside, bstart, bsize, n_e
            v0 = vo_d[gid]
            del gid
            yield u + v0, v + v0

    def finish(u, v):
        g = torch.searchsorted(vo_d, u, right=True) - 1
        return (v - vo_d[g]).to(torch.int32), _pair_weights(torch, u, v, wmax, seed_base)

    off, idx, w = _build_csr(torch, N, chunks(), nbuckets, device, finish)
    edge_off = off[vo_d].cpu().numpy().astype(np.int64)
    return vtx_off, edge_off, off, idx, w, params


def graph_slice_to_host(vtx_off, edge_off, off, idx, w, g):
    """Graph g of a packed batch as host arrays (local offsets and ids)."""
    v0, v1 = int(vtx_off[g]), int(vtx_off[g + 1])
    e0, e1 = int(edge_off[g]), int(edge_off[g + 1])
    o = (off[v0:v1 + 1] - e0).cpu().numpy().astype(np.int64)
    i = idx[e0:e1].cpu().numpy().astype(np.int32)
    ww = None if w is None else w[e0:e1].cpu().numpy().astype(np.float32)
    return o, i, ww
