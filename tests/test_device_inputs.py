"""The generators of the two largest workloads (lpa_inputs.device), run with
torch on the CPU at small sizes.  They must give symmetric CSR with sorted,
distinct rows and no self-loops (batch weights symmetric integers 1..4, ids
local to each graph), the same graph for any bucket count, and the recipe they
state:

* R-MAT: the number of entries and the quadrant shares of the host generator
  (the same recipe drawn from another random stream), within sampling noise;
* planted-partition batch: per graph, the number of distinct pairs that
  round(n d / 2) uniform draws (80% inside a block) leave once self-loops and
  duplicates are dropped, from the occupancy formula -- k draws spread evenly
  over P pairs leave P (1 - exp(-k / P)) distinct ones in expectation -- and
  the share of entries inside blocks that follows from it.

A generator that drew the quadrants with other probabilities, kept
duplicates or self-loops, sent the 20% of draws between blocks into a block,
or mixed up graph-local and global ids fails one of these."""
import math

import numpy as np
import pytest

import lpa_inputs as L
from test_inputs import _check_symmetric

torch = pytest.importorskip("torch")
from lpa_inputs.device import (batched_params, batched_planted_partition_device,  # noqa: E402
                               graph_slice_to_host, rmat_device)


def _host(g):
    return L.Graph(g.off.numpy().astype(np.int64), g.idx.numpy().astype(np.int32), None, {})


def _quadrant_shares(off, idx, n):
    src = np.repeat(np.arange(n), np.diff(off))
    lo_s, lo_d = src < n // 2, idx < n // 2
    return np.mean(lo_s & lo_d), np.mean(~lo_s & ~lo_d)


def test_device_rmat_is_the_host_recipe():
    scale, ef = 11, 14
    n = 1 << scale
    for seed in (1, 2):
        g = rmat_device(scale, ef, seed=seed, device="cpu", nbuckets=4)
        hg = _host(g)
        _check_symmetric(hg)
        assert g.n == n and hg.w is None
        h = L.rmat(scale, ef, seed=seed)
        # the same recipe from another random stream: ~4e4 entries, so the
        # counts and shares agree to about 1% (the bounds are several sigma)
        assert abs(g.nnz / h.nnz - 1.0) < 0.03, (g.nnz, h.nnz)
        ll, hh = _quadrant_shares(hg.off, hg.idx, n)
        hll, hhh = _quadrant_shares(h.off, h.idx, n)
        assert abs(ll - hll) < 0.01 and abs(hh - hhh) < 0.01, (ll, hll, hh, hhh)
        deg, hdeg = np.diff(hg.off), np.diff(h.off)
        assert abs(np.mean(deg == 0) - np.mean(hdeg == 0)) < 0.03
        assert 0.85 < deg.max() / hdeg.max() < 1.15
    # the buckets only split the sort: one bucket gives the same graph
    a = rmat_device(scale, ef, seed=1, device="cpu", nbuckets=4)
    b = rmat_device(scale, ef, seed=1, device="cpu", nbuckets=1)
    assert torch.equal(a.off, b.off) and torch.equal(a.idx, b.idx)
    c = rmat_device(scale, ef, seed=2, device="cpu", nbuckets=4)
    assert not torch.equal(a.idx[:1000], c.idx[:1000])


def _expected_entries(n, nb, d, intra=0.8):
    """Expected stored entries and inside-block share of one graph of the
    batch recipe: M = round(n d / 2) draws, u uniform, v uniform in u's block
    with probability `intra` (self-loops dropped) else uniform outside it.
    Inside block b (size s): M intra (s - 1) / n non-self draws over
    s (s - 1) / 2 pairs.  Between blocks: M (1 - intra) draws, each pair hit
    with probability about 2 / (n (n - n / nb)) (blocks differ by at most one
    vertex)."""
    M = int(round(n * d / 2.0))
    sizes = L.equal_blocks(n, nb)
    inside = 0.0
    for s in sizes:
        P = s * (s - 1) / 2.0
        if P > 0:
            inside += P * (1.0 - math.exp(-M * intra * (s - 1) / n / P))
    Q = (n * n - sum(s * s for s in sizes)) / 2.0
    between = Q * (1.0 - math.exp(-M * (1.0 - intra) * 2.0 / (n * (n - n / nb))))
    return 2.0 * (inside + between), inside / (inside + between)


def _inside_share(off, idx, n, nb):
    blk = np.repeat(np.arange(nb), L.equal_blocks(n, nb))
    src = np.repeat(np.arange(n), np.diff(off))
    return float(np.mean(blk[src] == blk[idx]))


@pytest.mark.parametrize("n_min,n_max,G,tol", [(2000, 20000, 8, 0.02), (100, 3000, 6, 0.08)])
def test_device_batch_is_its_stated_recipe(n_min, n_max, G, tol):
    vo, eo, off, idx, w, params = batched_planted_partition_device(G=G, n_min=n_min, n_max=n_max,
                                                                   device="cpu", nbuckets=3)
    assert params == batched_params(G, n_min, n_max)
    # the per-graph draws are the host batch's (same seeds, same rule)
    assert params == [L.batched_sbm_params(k, n_min, n_max) for k in range(G)]
    assert vo[0] == 0 and np.array_equal(np.diff(vo), [p[0] for p in params])
    assert np.array_equal(eo, off[torch.from_numpy(vo)].numpy()) and eo[-1] == idx.shape[0]
    for k in range(G):
        n, nb, d = params[k]
        o, i, ww = graph_slice_to_host(vo, eo, off, idx, w, k)
        g = L.Graph(o, i, ww, {})
        _check_symmetric(g)                       # local ids, weights symmetric
        assert set(np.unique(ww).tolist()) <= {1.0, 2.0, 3.0, 4.0}
        e, share = _expected_entries(n, nb, d)
        assert abs(len(i) / e - 1.0) < tol, (k, len(i), e)
        assert abs(_inside_share(o, i, n, nb) - share) < tol, (k, share)
    # one bucket gives the same batch
    _, _, off1, idx1, w1, _ = batched_planted_partition_device(G=G, n_min=n_min, n_max=n_max,
                                                               device="cpu", nbuckets=1)
    assert torch.equal(off, off1) and torch.equal(idx, idx1) and torch.equal(w, w1)
