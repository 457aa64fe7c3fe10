"""The seeded generators give symmetric, sorted CSR of the advertised shape and
the advertised distributions (R-MAT quadrant rates, grid drop and shortcut rates)."""
import numpy as np
import pytest

import lpa_inputs as L


def _check_symmetric(g, allow_self=False, allow_dup=False):
    n = g.n
    assert g.off[0] == 0 and np.all(np.diff(g.off) >= 0) and g.off[-1] == g.idx.shape[0]
    assert g.idx.min(initial=0) >= 0 and g.idx.max(initial=0) < max(n, 1)
    src = np.repeat(np.arange(n, dtype=np.int64), np.diff(g.off))
    dst = g.idx.astype(np.int64)
    if not allow_self:
        assert not np.any(src == dst)
    fwd = src * n + dst
    rev = dst * n + src
    order_f = np.argsort(fwd, kind="stable")
    order_r = np.argsort(rev, kind="stable")
    assert np.array_equal(fwd[order_f], rev[order_r])
    if g.w is not None:
        assert np.array_equal(g.w[order_f], g.w[order_r])
    # rows sorted ascending (and strictly when duplicates are removed)
    d = np.diff(dst)
    same_row = np.diff(src) == 0
    assert np.all(d[same_row] >= 0)
    if not allow_dup:
        assert np.all(d[same_row] > 0)


def test_planted_partition_shape():
    g = L.planted_partition()
    _check_symmetric(g)
    assert g.n == 10_000 and g.w is None
    mean_deg = g.nnz / g.n
    assert 15.0 < mean_deg < 17.0
    blk = np.repeat(np.arange(g.n) // 1000, np.diff(g.off))
    intra = np.mean(blk == g.idx // 1000)
    assert abs(intra - 14 / 16) < 0.01
    g2 = L.planted_partition()
    assert np.array_equal(g.off, g2.off) and np.array_equal(g.idx, g2.idx)


def test_rmat_shape_and_determinism():
    g = L.rmat(12, 16, seed=1)
    _check_symmetric(g)
    assert g.n == 4096
    deg = np.diff(g.off)
    assert deg.max() > 20 * deg.mean()        # heavy tail
    g2 = L.rmat(12, 16, seed=1)
    assert np.array_equal(g.idx, g2.idx)
    g3 = L.rmat(12, 16, seed=2)
    assert not np.array_equal(g.idx[:1000], g3.idx[:1000])
    raw = L.rmat(10, 8, seed=1, dedup=False, drop_self=False)
    _check_symmetric(raw, allow_self=True, allow_dup=True)
    assert raw.nnz == 2 * 8 * 1024


def test_road_grid_shape():
    g = L.road_grid(64, 64, seed=1)
    _check_symmetric(g)
    assert g.n == 4096
    assert 3.3 < g.nnz / g.n < 3.8
    assert g.w is not None and g.w.min() >= 1 and g.w.max() <= 8 and np.all(g.w == np.round(g.w))


def test_batched_params_and_pack():
    ps = [L.batched_sbm_params(g) for g in range(200)]
    ns = np.array([p[0] for p in ps])
    assert ns.min() >= 100 and ns.max() <= 200_000
    assert all(2 <= p[1] <= 64 and 4.0 <= p[2] <= 64.0 for p in ps)
    graphs = [L.batched_sbm_graph(g, n_max=3000) for g in range(5)]
    for gr in graphs:
        _check_symmetric(gr)
        assert gr.w.min() >= 1 and gr.w.max() <= 4
    vo, eo, off, idx, w = L.pack(graphs)
    assert vo[-1] == sum(gr.n for gr in graphs) and off[-1] == eo[-1]
    for k, gr in enumerate(graphs):
        assert np.array_equal(idx[eo[k]:eo[k + 1]] - vo[k], gr.idx)


def test_rmat_quadrant_probabilities():
    """Each recursion level of R-MAT picks quadrant (row bit, column bit) =
    (0,0), (0,1), (1,0), (1,1) with a, b, c, d; the raw symmetrised entries
    show those rates at every bit level (the mirrored half swaps b and c)."""
    scale = 14
    raw = L.rmat(scale, 16, seed=3, dedup=False, drop_self=False)
    src = np.repeat(np.arange(raw.n, dtype=np.int64), np.diff(raw.off))
    dst = raw.idx.astype(np.int64)
    a, b, c, d = 0.57, 0.19, 0.19, 0.05
    for level in (scale - 1, scale // 2, 0):
        rs, cs = (src >> level) & 1, (dst >> level) & 1
        got = [np.mean((rs == r) & (cs == q)) for r, q in ((0, 0), (0, 1), (1, 0), (1, 1))]
        want = [a, (b + c) / 2, (b + c) / 2, d]
        assert np.allclose(got, want, atol=0.01), (level, got)


def test_road_grid_drop_and_shortcut_rates():
    """About 90% of the 4-neighbour lattice edges are kept, and 0.1% of that
    count is added as shortcuts (non-lattice pairs)."""
    rows, cols = 256, 256
    g = L.road_grid(rows, cols, seed=4)
    src = np.repeat(np.arange(g.n, dtype=np.int64), np.diff(g.off))
    dst = g.idx.astype(np.int64)
    up = src < dst
    s, t = src[up], dst[up]
    lattice = ((t - s == 1) & (s // cols == t // cols)) | (t - s == cols)
    n_lattice = rows * (cols - 1) + cols * (rows - 1)
    kept = int(lattice.sum())
    assert abs(kept / n_lattice - 0.90) < 0.01
    shortcuts = int((~lattice).sum())
    assert abs(shortcuts - 0.001 * kept) <= max(5, 0.2 * 0.001 * kept)


def test_row_range_sample_keeps_the_rows_in_order():
    """The sample holds exactly rows [v0, v1) with their neighbours relabelled
    in increasing order of their ids (so comparisons of ids, and with them the
    smallest-id tie-break, are unchanged), and at least the asked-for entries."""
    g = L.rmat(12, 16, seed=3)
    v0 = 700
    s, v1, ids = L.row_range_sample(g, v0, 5000)
    assert s.nnz == g.off[v1] - g.off[v0] >= 5000 and g.off[v1 - 1] - g.off[v0] < 5000
    assert np.all(np.diff(ids) > 0)
    for v in (v0, (v0 + v1) // 2, v1 - 1):
        k = int(np.searchsorted(ids, v))
        assert ids[k] == v
        assert np.array_equal(ids[s.idx[s.off[k]:s.off[k + 1]]], g.idx[g.off[v]:g.off[v + 1]])
    sampled = np.isin(ids, np.arange(v0, v1))
    assert np.all(np.diff(s.off)[~sampled] == 0)
