"""GPU label propagation vs the CPU oracle, through the C ABI.

Synchronous modes (LPA_MODE_SYNC, LPA_MODE_SYNC_FULL) must reproduce the
oracle's labels, sweep count and per-sweep changed counts exactly: every graph
here has integer weights, so every per-label sum is exact in any order.  The
asynchronous mode is order-dependent (Section 4.1), so it is held to
invariants: labels stay inside the vertex's connected component, the GPU's
modularity of its labels equals the oracle's, and that modularity is not below
the floor of tests/async_bounds.py (serial runs of Algorithm 1 in several
vertex orders); vertices off their local argmax are reported.
"""
import json
import os

from async_bounds import assert_async_quality, assert_local_max_bound, gpu_runs, serial_qs

import numpy as np
import pytest

import lpa_inputs as L
import oracle as O

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lpa():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    import paper_2312_08140_gb300 as m
    m.load()
    return m


def run_gpu(lpa, g, mode, tau=0.05, iters=20, cfg=None):
    import torch
    h = lpa.lpa_graph_create(g.n, g.nnz, g.off, g.idx, g.w)
    try:
        if cfg is not None:
            lpa.lpa_graph_set_config(h, lpa.LpaConfig(*cfg))
        out = torch.full((max(g.n, 1),), -7, dtype=torch.int32, device="cuda")
        info = lpa.lpa_run(h, mode, tau, iters, out)
        return out[:g.n].cpu().numpy(), info.as_dict(), h
    except Exception:
        lpa.lpa_graph_destroy(h)
        raise


def assert_sync_parity(lpa, g, tau=0.05, iters=20, cfg=None, modes=("sync", "sync_full")):
    ref, it, changed = O.lpa_sync(g.off, g.idx, g.w, tau, iters)
    for mode in modes:
        got, info, h = run_gpu(lpa, g, mode, tau, iters, cfg)
        lpa.lpa_graph_destroy(h)
        assert info["iterations"] == it, (mode, info["iterations"], it)
        assert info["changed"] == changed.tolist()[:64], mode
        mism = np.flatnonzero(got != ref)
        assert mism.size == 0, f"{mode}: {mism.size} labels differ, first at {mism[:5]}"
    return ref, it


def _golden():
    with open(os.path.join(ROOT, "tests", "golden", "hand_worked.json")) as f:
        return json.load(f)["cases"]


def _case_graph(case):
    if "clique" in case:
        k = case["clique"]
        return L.from_undirected_pairs(case["n"], [(u, v) for u in range(k) for v in range(u + 1, k)])
    return L.from_undirected_pairs(case["n"], [tuple(p) for p in case["pairs"]], case.get("weights"))


@pytest.mark.parametrize("case", [c for c in _golden() if c["mode"] == "sync"], ids=lambda c: c["name"])
def test_hand_worked_sync(lpa, case):
    g = _case_graph(case)
    for mode in ("sync", "sync_full"):
        got, info, h = run_gpu(lpa, g, mode, case.get("tau", 0.05), case.get("max_iters", 20))
        lpa.lpa_graph_destroy(h)
        assert got.tolist() == case["labels"]
        assert info["iterations"] == case["iterations"]
        assert info["changed"] == case["changed"]


def test_random_small_graphs_sync(lpa):
    rng = np.random.default_rng(11)
    for t in range(120):
        n = int(rng.integers(1, 60))
        g = L.random_small(n, float(rng.uniform(0.02, 0.6)), seed=70000 + t, wmax=int(rng.integers(0, 5)),
                           self_loops=0.1, multi=bool(t % 3 == 0))
        assert_sync_parity(lpa, g, tau=float(rng.choice([0.0, 0.05, 0.2])), iters=int(rng.integers(1, 25)))


def test_planted_partition_sync(lpa):
    g = L.planted_partition()
    ref, it = assert_sync_parity(lpa, g)
    assert it >= 3


@pytest.mark.parametrize("cfg", [None, (4, 64, 512, 1024, 0), (8, 256, 2048, 4096, 1001),
                                 (1, 33, 100, 200, 200)])
def test_rmat_bins_and_spill_sync(lpa, cfg):
    """R-MAT scale 16 has vertices in all five degree bins, and rows above
    4096 entries, whose inserts into the last bin's 8192-slot table are
    bounded (they would go to the overflow path if they failed)."""
    g = L.rmat(16, 16, seed=3)
    assert int(np.diff(g.off).max()) > 4096
    assert_sync_parity(lpa, g, cfg=cfg)


def test_profiled_path_matches_oracle(lpa):
    """lpa_run_profiled launches every sweep kernel from the host (the path
    the benchmark's roofline pass and ncu see) instead of the device loop; on
    R-MAT scale 16 (all five degree bins, rows above 4096 entries) its
    synchronous labels, sweep count and per-sweep changed counts
    are the oracle's, and its asynchronous labels stay inside components."""
    import torch
    g = L.rmat(16, 16, seed=3)
    ref, it, changed = O.lpa_sync(g.off, g.idx, g.w, 0.05, 20)
    h = lpa.lpa_graph_create(g.n, g.nnz, g.off, g.idx, g.w)
    try:
        out = torch.full((g.n,), -7, dtype=torch.int32, device="cuda")
        for mode in ("sync", "sync_full"):
            ri, prof = lpa.lpa_run_profiled(h, mode, 0.05, 20, out)
            got = out.cpu().numpy()
            mism = np.flatnonzero(got != ref)
            assert mism.size == 0, f"{mode}: {mism.size} labels differ, first at {mism[:5]}"
            assert ri.iterations == it and prof.iterations == it, (mode, ri.iterations, prof.iterations, it)
            assert list(ri.changed[:it]) == changed.tolist(), mode
        ri, prof = lpa.lpa_run_profiled(h, "async", 0.05, 20, out)
        got = out.cpu().numpy()
        assert np.all((got >= 0) & (got < g.n))
        assert O.count_labels_outside_component(g.off, g.idx, got) == 0
        assert prof.iterations == ri.iterations
    finally:
        lpa.lpa_graph_destroy(h)


def test_rmat_raw_duplicates_selfloops_sync(lpa):
    g = L.rmat(12, 8, seed=5, dedup=False, drop_self=False)
    assert_sync_parity(lpa, g)


def _props_rows_distinct(lpa, g):
    h = lpa.lpa_graph_create(g.n, g.nnz, g.off, g.idx, g.w)
    try:
        return lpa.lpa_graph_props_get(h)["rows_distinct"]
    finally:
        lpa.lpa_graph_destroy(h)


def test_first_sweep_of_repeat_free_rows(lpa):
    """A single graph whose rows list each neighbour once, in increasing order,
    runs its first synchronous sweep without label reads or hash tables (every
    label still equals its vertex id, so each label's sum is one entry's
    weight).  The detection must hold exactly: rows out of order, or with a
    neighbour listed twice (adjacent, so the only descent is an equal pair),
    keep the general path.  Every variant matches the oracle in all degree
    bins, strict and non-strict."""
    g = L.rmat(14, 16, seed=6, drop_self=False, wmax=8)         # sorted rows, self-loops kept
    assert int(np.diff(g.off).max()) > 2048                     # reaches the last bin
    assert _props_rows_distinct(lpa, g) == 1

    # one row (the longest) reversed: distinct but not increasing
    v = int(np.argmax(np.diff(g.off)))
    idx_r, w_r = g.idx.copy(), g.w.copy()
    s0, e0 = int(g.off[v]), int(g.off[v + 1])
    idx_r[s0:e0] = idx_r[s0:e0][::-1]
    w_r[s0:e0] = w_r[s0:e0][::-1]
    g_rev = L.Graph(g.off, idx_r, w_r, {})
    assert _props_rows_distinct(lpa, g_rev) == 0

    # every row of degree >= 2 lists its lightest neighbour twice, side by side
    rows_i, rows_w = [], []
    deg = np.diff(g.off)
    for u in range(g.n):
        a, b = int(g.off[u]), int(g.off[u + 1])
        ri, rw = g.idx[a:b], g.w[a:b]
        if b - a >= 2:
            k = int(np.argmin(rw))
            ri = np.insert(ri, k, ri[k])
            rw = np.insert(rw, k, rw[k])
        rows_i.append(ri)
        rows_w.append(rw)
    off_d = np.zeros(g.n + 1, dtype=np.int64)
    np.cumsum(deg + (deg >= 2), out=off_d[1:])
    g_dup = L.Graph(off_d, np.concatenate(rows_i).astype(np.int32), np.concatenate(rows_w).astype(np.float32), {})
    assert _props_rows_distinct(lpa, g_dup) == 0

    for gr in (g, g_rev, g_dup):
        assert_sync_parity(lpa, gr)
        ref, it, ch = O.lpa_sync(gr.off, gr.idx, gr.w, nonstrict=True)
        got, info, h = run_gpu(lpa, gr, "sync+nonstrict")
        lpa.lpa_graph_destroy(h)
        assert info["iterations"] == it and np.array_equal(got, ref)
    # the duplicated entries change the first sweep's picks somewhere, so the
    # two graphs are told apart by the oracle too
    assert not np.array_equal(O.sync_sweep(g.off, g.idx, g.w, np.arange(g.n, dtype=np.int32))[0],
                              O.sync_sweep(g_dup.off, g_dup.idx, g_dup.w, np.arange(g.n, dtype=np.int32))[0])


def test_weighted_grid_sync(lpa):
    g = L.road_grid(200, 173, seed=2)       # ragged: n is not a multiple of any tile
    assert_sync_parity(lpa, g, iters=7)


def test_weighted_sbm_sync(lpa):
    g = L.batched_sbm_graph(3, n_max=20000)
    assert_sync_parity(lpa, g)


def test_edge_cases(lpa):
    import torch
    # N == 0
    h = lpa.lpa_graph_create(0, 0, np.zeros(1, np.int64), np.zeros(0, np.int32))
    info = lpa.lpa_run(h, "sync", 0.05, 20, None)
    assert info.iterations == 0 and info.exit_reason == 2
    lpa.lpa_graph_destroy(h)
    # no entries: one sweep, nothing changes, labels = ids
    g = L.Graph(np.zeros(6, np.int64), np.zeros(0, np.int32), None)
    for mode in ("sync", "async", "sync_full"):
        got, info, h = run_gpu(lpa, g, mode)
        lpa.lpa_graph_destroy(h)
        assert got.tolist() == list(range(5)) and info["iterations"] == 1 and info["changed"] == [0]
    # max_iters == 0: labels stay ids
    g = L.planted_partition(n=500, blocks=5, seed=2)
    got, info, h = run_gpu(lpa, g, "async", 0.05, 0)
    lpa.lpa_graph_destroy(h)
    assert np.array_equal(got, np.arange(g.n)) and info["iterations"] == 0 and info["exit_reason"] == 2
    # tolerance 1: exactly one sweep
    assert_sync_parity(lpa, g, tau=1.0)
    # cap reached
    ref, it = assert_sync_parity(lpa, L.from_undirected_pairs(2, [(0, 1)]), iters=5)
    assert it == 5


def test_invalid_graphs_rejected(lpa):
    off = np.array([0, 2, 3, 4], np.int64)
    idx = np.array([1, 2, 0, 0], np.int32)
    bad = [
        (np.array([0, 2, 1, 4], np.int64), idx, None),          # decreasing offsets
        (np.array([0, 2, 3, 5], np.int64), idx, None),          # offsets[n] != nnz
        (off, np.array([1, 3, 0, 0], np.int32), None),          # index out of range
        (off, np.array([1, -1, 0, 0], np.int32), None),         # negative index
        (off, idx, np.array([1, -2, 1, 1], np.float32)),        # negative weight
        (off, idx, np.array([1, np.nan, 1, 1], np.float32)),    # NaN weight
        (off, idx, np.array([1, np.inf, 1, 1], np.float32)),    # inf weight
    ]
    for o, i, w in bad:
        with pytest.raises(lpa.LpaError) as e:
            lpa.lpa_graph_create(3, 4, o, i, w)
        assert e.value.status in (lpa.LPA_ERR_INVALID_GRAPH, lpa.LPA_ERR_INVALID_ARG)
    with pytest.raises(lpa.LpaError):
        lpa.lpa_graph_create(-1, 0, off, idx)
    h = lpa.lpa_graph_create(3, 4, off, idx)
    import torch
    out = torch.empty(3, dtype=torch.int32, device="cuda")
    for args in (("sync", -0.1, 20), ("sync", 1.5, 20), ("sync", 0.05, -1), (7, 0.05, 20)):
        with pytest.raises(lpa.LpaError):
            lpa.lpa_run(h, args[0], args[1], args[2], out)
    lpa.lpa_graph_destroy(h)


def test_non_integer_weights_flagged_inexact(lpa):
    g = L.road_grid(64, 64, seed=4)
    w = g.w * 0.37
    h = lpa.lpa_graph_create(g.n, g.nnz, g.off, g.idx, w)
    assert lpa.lpa_graph_props_get(h)["exact"] == 0
    lpa.lpa_graph_destroy(h)
    h = lpa.lpa_graph_create(g.n, g.nnz, g.off, g.idx, g.w)
    p = lpa.lpa_graph_props_get(h)
    assert p["exact"] == 1 and p["weighted"] == 1 and p["weight_bytes"] == 1    # integers <= 255: one byte
    lpa.lpa_graph_destroy(h)


def test_integer_weight_widths(lpa):
    """Integer weights are stored in one byte when all are <= 255 and in four
    otherwise; both give the oracle's labels exactly, as do non-integer ones."""
    base = L.road_grid(90, 70, seed=9)
    rng = np.random.default_rng(4)
    # symmetric weights: the same value on (i, j) and (j, i)
    src = np.repeat(np.arange(base.n), np.diff(base.off))
    key = np.minimum(src, base.idx).astype(np.int64) * base.n + np.maximum(src, base.idx)
    for wmax, width in ((255, 1), (256, 4), (100000, 4)):
        vals = rng.integers(1, wmax + 1, size=key.size)
        _, inv = np.unique(key, return_inverse=True)
        w = vals[inv].astype(np.float32)
        w[inv == inv[np.argmax(vals[inv])]] = wmax             # the largest weight occurs
        g = L.Graph(base.off, base.idx, w, {})
        h = lpa.lpa_graph_create(g.n, g.nnz, g.off, g.idx, g.w)
        assert lpa.lpa_graph_props_get(h)["weight_bytes"] == width
        lpa.lpa_graph_destroy(h)
        assert_sync_parity(lpa, g)


def test_weighted_degree_thresholds_and_max_degree(lpa):
    """Creation records the largest degree and whether every per-label sum is
    exact: integer weights whose row sums reach 2^31 are not (32-bit sums could
    overflow), and borrowed integer weights (kept as fp32) are not once a row
    sum reaches 2^24.  A row whose degree x largest weight reaches 2^24 but
    whose sum does not stays exact."""
    import torch
    # star 0 - {1, 2}, plus an edge 3 - 4
    off = np.array([0, 2, 3, 4, 5, 6], np.int64)
    idx = np.array([1, 2, 0, 0, 4, 3], np.int32)
    cases = [
        (np.array([1.5e9, 1.5e9, 1.5e9, 1.5e9, 1, 1], np.float32), 0, 0),     # row 0 sums to 3e9 >= 2^31
        (np.array([1.5e9, 1, 1.5e9, 1, 1, 1], np.float32), 0, 1),             # largest row sum 1.5e9 + 1
        (np.array([2 ** 23, 2 ** 23, 2 ** 23, 2 ** 23, 1, 1], np.float32), True, 0),   # 2^24
        (np.array([2 ** 23, 2 ** 23 - 1, 2 ** 23, 2 ** 23 - 1, 1, 1], np.float32), True, 1),
    ]
    for w, borrow, exact in cases:
        if borrow:
            t_off, t_idx, t_w = (torch.from_numpy(a).cuda() for a in (off, idx, w))
            h = lpa.lpa_graph_create(5, 6, t_off, t_idx, t_w, lpa.LPA_DEVICE_PTRS | lpa.LPA_BORROW)
        else:
            h = lpa.lpa_graph_create(5, 6, off, idx, w)
        p = lpa.lpa_graph_props_get(h)
        lpa.lpa_graph_destroy(h)
        assert p["exact"] == exact, (w, borrow)
        assert p["max_degree"] == 2
    g = L.rmat(14, 16, seed=5)
    h = lpa.lpa_graph_create(g.n, g.nnz, g.off, g.idx, g.w)
    assert lpa.lpa_graph_props_get(h)["max_degree"] == int(np.diff(g.off).max())
    lpa.lpa_graph_destroy(h)


def test_async_small_sbm_graphs(lpa):
    """Small graphs fit in one wave of the GPU; the asynchronous mode must
    still visit each warp's or thread's vertices in order (Algorithm 1) rather
    than all at once, or its quality falls to that of the synchronous mode
    (on the 509-vertex graph here: 0.63 against the serial 0.76)."""
    for gi in range(50, 70):
        check_async(lpa, L.batched_sbm_graph(gi, n_max=5000))


def hub_graph(leaves, repeat=False):
    """A hub joined to `leaves` vertices that are paired into triangles with it
    (every leaf pair also linked), so the hub's row holds `leaves` distinct
    labels in the first sweep: more than the last bin's shared table holds.
    With `repeat` the hub-leaf 1 edge is listed twice (adjacent entries in
    both rows), so the graph is not repeat-free."""
    pairs = [(0, k) for k in range(1, leaves + 1)]
    pairs += [(k, k + 1) for k in range(1, leaves, 2)]
    if repeat:
        pairs.append((0, 1))
    return L.from_undirected_pairs(leaves + 1, pairs)


def test_repeat_free_hub_rows(lpa):
    """Hub rows of 5,001 to 40,001 entries in repeat-free graphs: the first
    sweep picks each row's first heaviest entry without a table, and the
    later sweeps see few distinct labels; labels, sweep counts and changed
    counts stay exact, and the asynchronous runs meet the acceptance rule."""
    for leaves in (5000, 9000, 40000):
        assert_sync_parity(lpa, hub_graph(leaves))
    check_async(lpa, hub_graph(40000))


def test_hub_rows_through_the_sliced_overflow_path(lpa):
    """A hub whose row lists a leaf twice makes the graph not repeat-free, so
    the first sweep takes the general path: the hub's row then holds `leaves`
    distinct labels, more than the 8192 slots of the last bin's table, and
    goes through the sliced overflow path (slices grouped by label partition,
    then one block per partition).  Synchronous labels, sweep counts and
    changed counts equal the oracle's; asynchronous labels stay inside the
    component."""
    for leaves in (9000, 40000):
        g = hub_graph(leaves, repeat=True)
        assert _props_rows_distinct(lpa, g) == 0
        assert_sync_parity(lpa, g)
        got, info, h = run_gpu(lpa, g, "async")
        lpa.lpa_graph_destroy(h)
        assert np.all((got >= 0) & (got < g.n))
        assert O.count_labels_outside_component(g.off, g.idx, got) == 0


def test_nonstrict_sync_matches_oracle(lpa):
    """The non-strict tie-break (LPA_NONSTRICT, Section 4.1.5) is deterministic,
    so the synchronous runs must match the oracle's non-strict runs exactly,
    through every degree bin, batched graphs included."""
    import torch
    graphs = [L.planted_partition(n=3000, blocks=6, seed=8), L.road_grid(80, 61, seed=3),
              L.rmat(14, 16, seed=4), hub_graph(9000)]
    for g in graphs:
        ref, it, ch = O.lpa_sync(g.off, g.idx, g.w, nonstrict=True)
        for mode in ("sync+nonstrict", "sync_full+nonstrict"):
            got, info, h = run_gpu(lpa, g, mode, 0.05, 20, None)
            lpa.lpa_graph_destroy(h)
            assert info["iterations"] == it and info["changed"] == ch.tolist()[:64], mode
            assert np.array_equal(got, ref), (mode, int((got != ref).sum()))
    batch = [L.batched_sbm_graph(gi, n_max=4000) for gi in range(8)]
    vo, eo, off, idx, w = _batch_inputs(batch)
    b = lpa.lpa_batch_create(len(batch), vo, eo, off, idx, w)
    out = torch.empty(int(vo[-1]), dtype=torch.int32, device="cuda")
    try:
        infos = lpa.lpa_batch_run(b, len(batch), "sync+nonstrict", 0.05, 20, out)
        got = out.cpu().numpy()
        for k, gr in enumerate(batch):
            ref, it, ch = O.lpa_sync(gr.off, gr.idx, gr.w, nonstrict=True)
            assert np.array_equal(got[vo[k]:vo[k + 1]], ref), k
            assert infos[k].iterations == it, k
    finally:
        lpa.lpa_batch_destroy(b)


def test_nonstrict_async_invariants(lpa):
    for g in (L.planted_partition(n=3000, blocks=6, seed=9), L.road_grid(120, 90, seed=5)):
        got, info, h = run_gpu(lpa, g, "async+nonstrict", 0.05, 20, None)
        lpa.lpa_graph_destroy(h)
        assert O.count_labels_outside_component(g.off, g.idx, got) == 0
        assert 1 <= info["iterations"] <= 20


def test_prune_other_needs_async(lpa):
    """LPA_PRUNE_OTHER (FLPA's pruning rule, Section 2) changes the algorithm,
    so the synchronous modes refuse it."""
    g = L.planted_partition(n=500, blocks=5, seed=3)
    h = lpa.lpa_graph_create(g.n, g.nnz, g.off, g.idx, g.w)
    try:
        for mode in ("sync+prune_other", "sync_full+prune_other", "sync+nonstrict+prune_other"):
            with pytest.raises(lpa.LpaError) as e:
                lpa.lpa_run(h, mode, 0.05, 20, None)
            assert e.value.status == lpa.LPA_ERR_INVALID_ARG
    finally:
        lpa.lpa_graph_destroy(h)


def test_prune_other_async_invariants(lpa):
    """Asynchronous runs under FLPA's pruning rule (a vertex whose label
    changes to c marks only the neighbours not already in c): the invariants
    and the modularity bound of check_async against serial runs under the same
    rule; batched graphs too, over five batch runs (fifteen when a graph's
    serial runs are not concentrated)."""
    import torch
    graphs = [L.planted_partition(n=3000, blocks=6, seed=31), L.road_grid(120, 90, seed=6),
              L.rmat(14, 16, seed=7), hub_graph(40000)]
    for g in graphs:
        check_async(lpa, g, mode="async+prune_other")
    batch = [L.batched_sbm_graph(gi, n_max=4000) for gi in range(8)]
    vo, eo, off, idx, w = _batch_inputs(batch)
    b = lpa.lpa_batch_create(len(batch), vo, eo, off, idx, w)
    out = torch.empty(int(vo[-1]), dtype=torch.int32, device="cuda")
    try:
        serial = [serial_qs(gr, prune_other=True) for gr in batch]
        qs = [[] for _ in batch]
        for r in range(max(gpu_runs(sq) for sq in serial)):
            infos = lpa.lpa_batch_run(b, len(batch), "async+prune_other", 0.05, 20, out)
            got = out.cpu().numpy()
            for k, gr in enumerate(batch):
                lab = got[vo[k]:vo[k + 1]]
                assert O.count_labels_outside_component(gr.off, gr.idx, lab) == 0, k
                assert_local_max_bound(gr, lab, infos[k], 0.05, f"batch graph {k}")
                qs[k].append(O.modularity(gr.off, gr.idx, gr.w, lab))
        for k, gr in enumerate(batch):
            assert_async_quality(qs[k][:gpu_runs(serial[k])], serial[k], f"prune_other batch graph {k}")
    finally:
        lpa.lpa_batch_destroy(b)


def test_pool_reuse_and_release(lpa):
    """Graph memory comes from the library's pool: graphs created after others
    were destroyed (reusing their pages), and after the cache was released,
    still give the oracle's labels."""
    graphs = [L.planted_partition(n=3000, blocks=6, seed=21), L.road_grid(70, 50, seed=2),
              L.planted_partition(n=3000, blocks=6, seed=21)]
    for k, g in enumerate(graphs):
        assert_sync_parity(lpa, g)
        if k == 1:
            lpa.lpa_release_cached_memory()
    lpa.lpa_release_cached_memory()


def check_async(lpa, g, tau=0.05, iters=20, cfg=None, runs=5, mode="async"):
    """Asynchronous runs held to: labels in range and inside the vertex's
    component; GPU modularity equal to the fp64 oracle's on the same labels
    (1e-6 rel); each sweep scans a vertex at most once and the first sweep
    every vertex with an entry; at an exit by tolerance the vertices off
    their local argmax within the neighbourhood bound of async_bounds (at
    most the sum of the largest degrees, as many as the last sweep changed);
    and over `runs` runs (15 where the
    serial runs are not concentrated) the modularity bound of async_bounds
    against the oracle's serial runs in seeded random
    vertex orders (median within 0.02 of their median, or of their lower
    quartile where they are not concentrated; every run within 0.02 of their
    lowest)."""
    import torch
    with_entries = int(np.count_nonzero(np.diff(g.off)))
    serial = serial_qs(g, tau, iters, prune_other="prune_other" in mode)
    qs, infos = [], []
    for r in range(gpu_runs(serial, runs)):
        got, info, h = run_gpu(lpa, g, mode, tau, iters, cfg)
        try:
            assert np.all((got >= 0) & (got < g.n))
            assert O.count_labels_outside_component(g.off, g.idx, got) == 0
            q_gpu = lpa.lpa_modularity(h, torch.from_numpy(got).cuda())
        finally:
            lpa.lpa_graph_destroy(h)
        q_ref_gpu_labels = O.modularity(g.off, g.idx, g.w, got)
        assert abs(q_gpu - q_ref_gpu_labels) <= 1e-6 * max(1.0, abs(q_ref_gpu_labels))
        # a sweep scans each vertex at most once (Algorithm 1 marks a vertex
        # processed when it scans it), and the first sweep scans every vertex
        # that has an entry
        assert info["active"][0] == with_entries, (info["active"][0], with_entries)
        assert all(a <= with_entries for a in info["active"]), info["active"]
        off_max = assert_local_max_bound(g, got, info, tau, f"n={g.n} run {r}")
        print(f"async n={g.n} run {r}: Q={q_gpu:.4f} sweeps={info['iterations']} exit={info['exit_reason']} "
              f"off_local_max={off_max} ({off_max / max(g.n, 1):.4f} of N)")
        qs.append(q_gpu)
        infos.append(info)
    assert_async_quality(qs, serial, f"{mode} n={g.n}")
    return infos, qs, serial


def test_async_invariants_small(lpa):
    rng = np.random.default_rng(5)
    for t in range(60):
        n = int(rng.integers(2, 80))
        g = L.random_small(n, float(rng.uniform(0.05, 0.5)), seed=80000 + t, wmax=int(rng.integers(0, 4)))
        got, info, h = run_gpu(lpa, g, "async")
        lpa.lpa_graph_destroy(h)
        assert O.count_labels_outside_component(g.off, g.idx, got) == 0
        assert 1 <= info["iterations"] <= 20


def test_async_planted_partition(lpa):
    check_async(lpa, L.planted_partition())


def test_async_rmat_and_grid_medium(lpa):
    check_async(lpa, L.rmat(16, 16, seed=1))
    check_async(lpa, L.road_grid(512, 512, seed=1))


def test_modularity_parity(lpa):
    import torch
    rng = np.random.default_rng(9)
    for g in (L.planted_partition(), L.road_grid(100, 77, seed=3), L.rmat(13, 16, seed=2),
              L.from_undirected_pairs(3, [(0, 0), (0, 1), (1, 2)], [2.0, 1.0, 3.0])):
        h = lpa.lpa_graph_create(g.n, g.nnz, g.off, g.idx, g.w)
        for lab in (np.arange(g.n), np.zeros(g.n), rng.integers(0, max(1, g.n // 7), g.n)):
            lab = lab.astype(np.int32)
            q = lpa.lpa_modularity(h, torch.from_numpy(lab).cuda())
            q_ref = O.modularity(g.off, g.idx, g.w, lab)
            assert abs(q - q_ref) <= 1e-6 * max(1.0, abs(q_ref)), (q, q_ref)
        with pytest.raises(lpa.LpaError):
            lpa.lpa_modularity(h, torch.full((g.n,), g.n, dtype=torch.int32, device="cuda"))
        lpa.lpa_graph_destroy(h)


def _batch_inputs(graphs):
    vo, eo, off, idx_global, w = L.pack(graphs)
    idx_local = np.concatenate([gr.idx for gr in graphs]) if graphs else np.zeros(0, np.int32)
    return vo, eo, off, idx_local.astype(np.int32), w


def test_batch_matches_solo_sync(lpa):
    import torch
    graphs = [L.batched_sbm_graph(g, n_max=6000) for g in range(24)]
    graphs.insert(5, L.from_undirected_pairs(1, []))                 # single isolated vertex
    graphs.insert(9, L.from_undirected_pairs(2, [(0, 1)]))           # oscillates to the cap
    vo, eo, off, idx, w = _batch_inputs(graphs)
    b = lpa.lpa_batch_create(len(graphs), vo, eo, off, idx, w)
    out = torch.empty(int(vo[-1]), dtype=torch.int32, device="cuda")
    try:
        for mode in ("sync", "sync_full"):
            infos = lpa.lpa_batch_run(b, len(graphs), mode, 0.05, 20, out)
            got = out.cpu().numpy()
            for k, gr in enumerate(graphs):
                ref, it, ch = O.lpa_sync(gr.off, gr.idx, gr.w)
                assert np.array_equal(got[vo[k]:vo[k + 1]], ref), (mode, k)
                assert infos[k].iterations == it and list(infos[k].changed[:it]) == ch.tolist(), (mode, k)
        infos = lpa.lpa_batch_run(b, len(graphs), "async", 0.05, 20, out)
        got = out.cpu().numpy()
        for k, gr in enumerate(graphs):
            lab = got[vo[k]:vo[k + 1]]
            assert O.count_labels_outside_component(gr.off, gr.idx, lab) == 0
            q = lpa.lpa_batch_modularity(b, k, out[vo[k]:vo[k + 1]])
            assert abs(q - O.modularity(gr.off, gr.idx, gr.w, lab)) <= 1e-6
    finally:
        lpa.lpa_batch_destroy(b)


# ---------------------------------------------------------------- full size --
@pytest.fixture(scope="module")
def rmat22():
    return L.rmat(22, 16, seed=1)


@pytest.fixture(scope="module")
def grid4096():
    return L.road_grid(4096, 4096, seed=1)


def test_full_size_rmat22_sync(lpa, rmat22):
    assert_sync_parity(lpa, rmat22, modes=("sync",))


def test_full_size_grid_sync(lpa, grid4096):
    assert_sync_parity(lpa, grid4096, modes=("sync",))


def test_full_size_async(lpa, rmat22, grid4096):
    for g in (rmat22, grid4096):
        check_async(lpa, g)
