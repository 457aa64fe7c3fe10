"""Serving loop (lpa_serve_*): requests admitted while others run share one
device arena; in the synchronous mode each result must equal the oracle's
(hence a run on its own) label for label, with the same sweep count and
per-sweep changed counts; admission refuses what does not fit and accepts it
once space is released; large requests take the solo lane."""
import time

import numpy as np
import pytest

import lpa_inputs as L
import oracle as O
from async_bounds import assert_async_quality, assert_local_max_bound, gpu_runs, serial_qs


def test_serve_config_is_validated_before_any_device_call():
    import paper_2312_08140_gb300 as lpa
    from paper_2312_08140_gb300 import _build
    lpa.load(_build.build())
    for bad in (dict(arena_vertices=0, arena_entries=10), dict(arena_vertices=10, arena_entries=10, max_slots=1),
                dict(arena_vertices=10, arena_entries=10, tolerance=2.0),
                dict(arena_vertices=10, arena_entries=10, mode=9)):
        args = dict(hbm_budget_bytes=1 << 30, max_slots=4)
        args.update(bad)
        with pytest.raises(lpa.LpaError) as e:
            lpa.lpa_serve_create(**args)
        assert e.value.status == lpa.LPA_ERR_INVALID_ARG


def _drain(lpa, srv, tickets, timeout=120.0):
    done = set()
    t0 = time.time()
    while len(done) < len(tickets):
        done.update(lpa.lpa_serve_poll(srv))
        assert time.time() - t0 < timeout, "serving did not finish"
        time.sleep(0.001)
    return done


@pytest.mark.gpu
def test_serve_mix_equals_alone_sync():
    import paper_2312_08140_gb300 as lpa
    lpa.load()
    graphs = [L.batched_sbm_graph(g, n_max=8000) for g in range(40)]
    hub = 20000                 # a row wider than the shared table: the arena's overflow (rescan) path
    graphs += [L.from_undirected_pairs(hub + 1, [(0, k) for k in range(1, hub + 1)] +
                                       [(k, k + 1) for k in range(1, hub, 2)])]
    graphs += [L.road_grid(60, 41, seed=7), L.rmat(12, 16, seed=9), L.from_undirected_pairs(5, []),
               L.from_undirected_pairs(2, [(0, 1)]), L.Graph(np.zeros(1, np.int64), np.zeros(0, np.int32), None)]
    srv = lpa.lpa_serve_create(hbm_budget_bytes=4 << 30, arena_vertices=400_000, arena_entries=20_000_000,
                               max_slots=48, mode="sync")
    try:
        tickets = {}
        for k, g in enumerate(graphs):            # staggered: later requests join running cycles
            tickets[lpa.lpa_serve_submit(srv, g.n, g.nnz, g.off, g.idx, g.w)] = k
            if k % 7 == 3:
                time.sleep(0.002)
        _drain(lpa, srv, tickets)
        assert lpa.lpa_serve_stats(srv)["cycles"] > 0
        for t, k in tickets.items():
            g = graphs[k]
            lab, info = lpa.lpa_serve_fetch(srv, t, g.n)
            ref, it, ch = O.lpa_sync(g.off, g.idx, g.w)
            assert np.array_equal(lab, ref), k
            if g.n:
                assert info.iterations == it and list(info.changed[:it]) == ch.tolist(), k
            lpa.lpa_serve_release(srv, t)
    finally:
        lpa.lpa_serve_destroy(srv)


@pytest.mark.gpu
def test_serve_busy_then_admitted_and_solo_lane():
    import paper_2312_08140_gb300 as lpa
    lpa.load()
    g = L.planted_partition(n=3000, blocks=6, seed=3)
    big = L.rmat(14, 16, seed=2)
    srv = lpa.lpa_serve_create(hbm_budget_bytes=2 << 30, arena_vertices=4000, arena_entries=g.nnz + 100,
                               max_slots=4, mode="sync", solo_min_entries=200_000)
    try:
        t1 = lpa.lpa_serve_submit(srv, g.n, g.nnz, g.off, g.idx, g.w)
        with pytest.raises(lpa.LpaError) as e:      # arena full until t1 leaves
            lpa.lpa_serve_submit(srv, g.n, g.nnz, g.off, g.idx, g.w)
        assert e.value.status == lpa.LPA_ERR_BUSY
        tb = lpa.lpa_serve_submit(srv, big.n, big.nnz, big.off, big.idx, big.w)   # solo lane
        _drain(lpa, srv, [t1, tb])
        t2 = lpa.lpa_serve_submit(srv, g.n, g.nnz, g.off, g.idx, g.w)
        _drain(lpa, srv, [t2])
        ref, _, _ = O.lpa_sync(g.off, g.idx, g.w)
        for t in (t1, t2):
            lab, _ = lpa.lpa_serve_fetch(srv, t, g.n)
            assert np.array_equal(lab, ref)
        lab, info = lpa.lpa_serve_fetch(srv, tb, big.n)
        refb, itb, _ = O.lpa_sync(big.off, big.idx, big.w)
        assert np.array_equal(lab, refb) and info.iterations == itb
        with pytest.raises(lpa.LpaError) as e:
            lpa.lpa_serve_fetch(srv, 987654, 1)
        assert e.value.status == lpa.LPA_ERR_NOT_FOUND
        # a malformed solo-lane request is validated on the device and fails at fetch
        bad_idx = big.idx.copy()
        bad_idx[big.nnz // 3] = big.n
        tbad = lpa.lpa_serve_submit(srv, big.n, big.nnz, big.off, bad_idx, big.w)
        _drain(lpa, srv, [tbad])
        with pytest.raises(lpa.LpaError) as e:
            lpa.lpa_serve_fetch(srv, tbad, big.n)
        assert e.value.status == lpa.LPA_ERR_INVALID_GRAPH
    finally:
        lpa.lpa_serve_destroy(srv)


@pytest.mark.gpu
def test_serve_async_invariants():
    """Asynchronous requests served in the mix, each graph five times (fifteen
    if a graph's serial runs are not concentrated): labels inside components,
    the off-local-argmax bound at a tolerance exit, and the modularity bound
    of async_bounds per graph over its results."""
    import paper_2312_08140_gb300 as lpa
    lpa.load()
    graphs = [L.batched_sbm_graph(g, n_max=5000) for g in range(50, 70)]
    srv = lpa.lpa_serve_create(hbm_budget_bytes=4 << 30, arena_vertices=200_000, arena_entries=10_000_000,
                               max_slots=32, mode="async")
    try:
        serial = [serial_qs(g) for g in graphs]
        qs = [[] for _ in graphs]
        for r in range(max(gpu_runs(sq) for sq in serial)):
            tickets = {lpa.lpa_serve_submit(srv, g.n, g.nnz, g.off, g.idx, g.w): k for k, g in enumerate(graphs)}
            _drain(lpa, srv, tickets)
            for t, k in tickets.items():
                g = graphs[k]
                lab, info = lpa.lpa_serve_fetch(srv, t, g.n)
                lpa.lpa_serve_release(srv, t)
                assert O.count_labels_outside_component(g.off, g.idx, lab) == 0
                assert 1 <= info.iterations <= 20
                assert_local_max_bound(g, lab, info, 0.05, f"served graph {k}")
                qs[k].append(O.modularity(g.off, g.idx, g.w, lab))
        for k, g in enumerate(graphs):
            assert_async_quality(qs[k][:gpu_runs(serial[k])], serial[k], f"served graph {k}")
    finally:
        lpa.lpa_serve_destroy(srv)


@pytest.mark.gpu
def test_serve_rejects_malformed_requests_on_device_and_runs_the_rest():
    """Arena requests are checked while they are admitted (row order and range,
    index range, finite non-negative weights); a malformed one is reported as
    LPA_ERR_INVALID_GRAPH at fetch and never disturbs the requests around it.
    Page-locked inputs take the direct-copy path and must give the same labels."""
    import torch
    import paper_2312_08140_gb300 as lpa
    lpa.load()
    good = [L.batched_sbm_graph(g, n_max=4000) for g in range(80, 92)]
    base = L.planted_partition(n=600, blocks=3, seed=11)
    w = np.ones(base.nnz, np.float32)
    bad = []
    idx = base.idx.copy(); idx[base.nnz // 2] = base.n                     # index == n
    bad.append((base.off, idx, None))
    idx = base.idx.copy(); idx[7] = -3                                     # negative index
    bad.append((base.off, idx, None))
    off = base.off.copy(); off[5] = off[6] + 1                             # rows out of order
    bad.append((off, base.idx, None))
    wn = w.copy(); wn[3] = -1.0                                            # negative weight
    bad.append((base.off, base.idx, wn))
    wn = w.copy(); wn[base.nnz - 1] = np.nan                               # weight not finite
    bad.append((base.off, base.idx, wn))
    srv = lpa.lpa_serve_create(hbm_budget_bytes=4 << 30, arena_vertices=200_000, arena_entries=10_000_000,
                               max_slots=32, mode="sync")
    try:
        kinds = {}
        for k in range(max(len(good), len(bad))):
            if k < len(good):
                g = good[k]
                if k % 2:                                                  # page-locked copies of the inputs
                    off_p = torch.from_numpy(g.off).pin_memory().numpy()
                    idx_p = torch.from_numpy(g.idx).pin_memory().numpy()
                    w_p = None if g.w is None else torch.from_numpy(g.w).pin_memory().numpy()
                    t = lpa.lpa_serve_submit(srv, g.n, g.nnz, off_p, idx_p, w_p)
                else:
                    t = lpa.lpa_serve_submit(srv, g.n, g.nnz, g.off, g.idx, g.w)
                kinds[t] = ("good", k)
            if k < len(bad):
                o, i, ww = bad[k]
                kinds[lpa.lpa_serve_submit(srv, base.n, base.nnz, o, i, ww)] = ("bad", k)
        _drain(lpa, srv, kinds)
        for t, (kind, k) in kinds.items():
            if kind == "bad":
                with pytest.raises(lpa.LpaError) as e:
                    lpa.lpa_serve_fetch(srv, t, base.n)
                assert e.value.status == lpa.LPA_ERR_INVALID_GRAPH, k
            else:
                g = good[k]
                lab, info = lpa.lpa_serve_fetch(srv, t, g.n)
                ref, it, ch = O.lpa_sync(g.off, g.idx, g.w)
                assert np.array_equal(lab, ref), k
                assert info.iterations == it and list(info.changed[:it]) == ch.tolist(), k
            lpa.lpa_serve_release(srv, t)
        # a slot and range freed by a rejected request are reusable
        t = lpa.lpa_serve_submit(srv, base.n, base.nnz, base.off, base.idx, None)
        _drain(lpa, srv, [t])
        lab, _ = lpa.lpa_serve_fetch(srv, t, base.n)
        assert np.array_equal(lab, O.lpa_sync(base.off, base.idx, None)[0])
        # the O(1) host checks still refuse at submit
        off = base.off.copy(); off[-1] += 1
        with pytest.raises(lpa.LpaError) as e:
            lpa.lpa_serve_submit(srv, base.n, base.nnz, off, base.idx, None)
        assert e.value.status == lpa.LPA_ERR_INVALID_GRAPH
    finally:
        lpa.lpa_serve_destroy(srv)
