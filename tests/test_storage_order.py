"""Storage orders (LPA_REORDER_DEGREE, LPA_REORDER_SHUFFLE, the batch default):
the library stores the vertices in an order of its own, but labels stay the
caller's ids (Algorithm 1 starts from C_i = i and ties go to the smallest id),
so the synchronous modes must give exactly the oracle's labels, sweep counts
and per-sweep changes on the caller's graph, under either tie-break, and the
modularity (Eq. 1) of the caller's labelling is the oracle's."""
import numpy as np
import pytest

import lpa_inputs as L
import oracle as O

pytestmark = pytest.mark.gpu

TAU, ITERS = 0.05, 20


@pytest.fixture(scope="module")
def lpa():
    import paper_2312_08140_gb300 as m
    m.load()
    return m


def _graphs():
    rng = np.random.default_rng(23)
    gs = [L.rmat(15, 16, seed=8), L.planted_partition(n=3000, blocks=6, seed=5), L.road_grid(90, 70, seed=4),
          L.rmat(12, 16, seed=9, dedup=False, drop_self=False), L.batched_sbm_graph(7, n_max=20_000)]
    gs += [L.random_small(int(rng.integers(1, 60)), float(rng.uniform(0.05, 0.5)), seed=700 + s,
                          wmax=int(rng.integers(0, 5)), self_loops=0.2, multi=bool(s % 2)) for s in range(30)]
    return gs


def _run(lpa, g, flags, mode):
    import torch
    h = lpa.lpa_graph_create(g.n, g.nnz, g.off, g.idx, g.w, lpa.LPA_HOST_PTRS | flags)
    out = torch.full((max(g.n, 1),), -7, dtype=torch.int32, device="cuda")
    try:
        info = lpa.lpa_run(h, mode, TAU, ITERS, out)
        props = lpa.lpa_graph_props_get(h)
        q = lpa.lpa_modularity(h, out[:g.n]) if g.n else 0.0
        return out[:g.n].cpu().numpy(), info, props, q
    finally:
        lpa.lpa_graph_destroy(h)


@pytest.mark.parametrize("order", ["degree", "shuffle"])
def test_sync_labels_are_the_callers_in_every_order(lpa, order):
    flags = {"degree": lpa.LPA_REORDER_DEGREE, "shuffle": lpa.LPA_REORDER_SHUFFLE}[order]
    for g in _graphs():
        for mode, ns in (("sync", False), ("sync_full", False), ("sync+nonstrict", True)):
            ref, it, ch = O.lpa_sync(g.off, g.idx, g.w, TAU, ITERS, nonstrict=ns)
            got, info, props, q = _run(lpa, g, flags, mode)
            assert props["storage_order"] == (1 if order == "degree" else 2) or g.n == 0
            assert np.array_equal(got, ref), (order, mode, g.n)
            assert info.iterations == it and list(info.changed[:it]) == ch.tolist(), (order, mode, g.n)
            if g.n:
                q_ref = O.modularity(g.off, g.idx, g.w, ref)
                assert abs(q - q_ref) <= 1e-6 * max(1.0, abs(q_ref)), (order, g.n)


@pytest.mark.parametrize("order", ["degree", "shuffle"])
def test_async_invariants_in_every_order(lpa, order):
    flags = {"degree": lpa.LPA_REORDER_DEGREE, "shuffle": lpa.LPA_REORDER_SHUFFLE}[order]
    for g in _graphs()[:5]:
        got, info, _, q = _run(lpa, g, flags, "async")
        assert np.all((got >= 0) & (got < g.n))
        assert O.count_labels_outside_component(g.off, g.idx, got) == 0
        q_ref = O.modularity(g.off, g.idx, g.w, got)
        assert abs(q - q_ref) <= 1e-6 * max(1.0, abs(q_ref))


def test_borrowed_arrays_are_left_as_given(lpa):
    import torch
    g = L.rmat(13, 16, seed=4)
    off, idx = torch.from_numpy(g.off).cuda(), torch.from_numpy(g.idx).cuda()
    off0, idx0 = off.clone(), idx.clone()
    h = lpa.lpa_graph_create(g.n, g.nnz, off, idx, None,
                             lpa.LPA_DEVICE_PTRS | lpa.LPA_BORROW | lpa.LPA_REORDER_DEGREE)
    out = torch.empty(g.n, dtype=torch.int32, device="cuda")
    try:
        lpa.lpa_run(h, "sync", TAU, ITERS, out)
        assert torch.equal(off, off0) and torch.equal(idx, idx0)
        assert np.array_equal(out.cpu().numpy(), O.lpa_sync(g.off, g.idx, None, TAU, ITERS)[0])
    finally:
        lpa.lpa_graph_destroy(h)


def test_order_flags_are_checked(lpa):
    g = L.rmat(8, 8, seed=1)
    with pytest.raises(lpa.LpaError) as e:
        lpa.lpa_graph_create(g.n, g.nnz, g.off, g.idx, None, lpa.LPA_REORDER_DEGREE | lpa.LPA_REORDER_SHUFFLE)
    assert e.value.status == lpa.LPA_ERR_INVALID_ARG
    graphs = [L.rmat(7, 8, seed=s) for s in range(3)]
    vo, eo, off, _, w = L.pack(graphs)
    idx = np.concatenate([gr.idx for gr in graphs]).astype(np.int32)
    with pytest.raises(lpa.LpaError) as e:
        lpa.lpa_batch_create(3, vo, eo, off, idx, w, lpa.LPA_HOST_PTRS | lpa.LPA_REORDER_DEGREE)
    assert e.value.status == lpa.LPA_ERR_INVALID_ARG
    for flags, order in ((lpa.LPA_HOST_PTRS, 2), (lpa.LPA_KEEP_ORDER, 0)):
        b = lpa.lpa_batch_create(3, vo, eo, off, idx, w, flags)
        assert lpa.lpa_batch_props_get(b)["storage_order"] == order
        lpa.lpa_batch_destroy(b)


def test_batches_in_both_orders_match_the_oracle(lpa):
    """The batch default (each graph shuffled) and LPA_KEEP_ORDER: every
    graph's synchronous labels, sweeps and changes equal its own oracle run,
    in local ids, and lpa_batch_modularity equals the oracle's Q."""
    import torch
    graphs = [L.batched_sbm_graph(gi, n_max=30_000) for gi in range(40, 52)] + [L.rmat(10, 8, seed=3)]
    vo, eo, off, _, w = L.pack(graphs)
    idx = np.concatenate([gr.idx for gr in graphs]).astype(np.int32)
    G = len(graphs)
    for flags in (lpa.LPA_HOST_PTRS, lpa.LPA_KEEP_ORDER):
        b = lpa.lpa_batch_create(G, vo, eo, off, idx, w, flags)
        out = torch.empty(int(vo[-1]), dtype=torch.int32, device="cuda")
        try:
            infos = lpa.lpa_batch_run(b, G, "sync", TAU, ITERS, out)
            got = out.cpu().numpy()
            for k, gr in enumerate(graphs):
                ref, it, ch = O.lpa_sync(gr.off, gr.idx, gr.w, TAU, ITERS)
                assert np.array_equal(got[vo[k]:vo[k + 1]], ref), (flags, k)
                assert infos[k].iterations == it and list(infos[k].changed[:it]) == ch.tolist(), (flags, k)
                q = lpa.lpa_batch_modularity(b, k, out[vo[k]:vo[k + 1]])
                q_ref = O.modularity(gr.off, gr.idx, gr.w, ref)
                assert abs(q - q_ref) <= 1e-6 * max(1.0, abs(q_ref)), (flags, k)
        finally:
            lpa.lpa_batch_destroy(b)
