"""lpa_modularity_noalloc: the entry point for callers that may not allocate
device memory (a plugin whose host framework owns the device memory pool, a
latency-critical loop).  It must give the same modularity as lpa_modularity
on a graph handle and as the fp64 oracle, call after call, even though every
call reuses the same fixed working array inside the library.

Collected last on purpose: if it fails, a run that stops at the first failure
has already run every other test."""
import numpy as np
import pytest

import lpa_inputs as L
import oracle as O

pytestmark = pytest.mark.gpu


def _device(a):
    import torch
    return None if a is None else torch.from_numpy(np.ascontiguousarray(a)).cuda()


def test_noalloc_modularity_matches_handle_entry_point():
    import torch
    import paper_2312_08140_gb300 as lpa
    lpa.load()
    rng = np.random.default_rng(17)
    graphs = [L.planted_partition(), L.road_grid(150, 97, seed=5), L.rmat(13, 16, seed=4),
              L.from_undirected_pairs(3, [(0, 0), (0, 1), (1, 2)], [2.0, 1.0, 3.0])]
    for g in graphs:
        h = lpa.lpa_graph_create(g.n, g.nnz, g.off, g.idx, g.w)
        try:
            run_labels = torch.empty(g.n, dtype=torch.int32, device="cuda")
            lpa.lpa_run(h, "sync", 0.05, 20, run_labels)
            rand_labels = _device(rng.integers(0, max(1, g.n // 5), g.n).astype(np.int32))
            off_d, idx_d, w_d = _device(g.off), _device(g.idx), _device(g.w)
            for labels in (run_labels, rand_labels):
                q_ref = lpa.lpa_modularity(h, labels)
                q_oracle = O.modularity(g.off, g.idx, g.w, labels.cpu().numpy())
                for _ in range(2):                       # two calls in a row share the array
                    q = lpa.lpa_modularity_noalloc(g.n, g.nnz, off_d, idx_d, w_d, labels)
                    assert abs(q - q_ref) <= 1e-6 * max(1.0, abs(q_ref)), (q, q_ref)
                    assert abs(q - q_oracle) <= 1e-6 * max(1.0, abs(q_oracle)), (q, q_oracle)
        finally:
            lpa.lpa_graph_destroy(h)


def test_noalloc_rejects_sizes_beyond_its_limit():
    import paper_2312_08140_gb300 as lpa
    lpa.load()
    with pytest.raises(lpa.LpaError) as e:
        lpa.lpa_modularity_noalloc((1 << 20) + 1, 0, 1, None, None, 1)
    assert e.value.status == lpa.LPA_ERR_INVALID_ARG and "limit" in e.value.message
