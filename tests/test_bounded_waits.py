"""The row kernels' bounded waits, made to run out without a GPU fault.

Every wait of the row kernels on a bulk copy is bounded (2 s of GPU time);
one that gives up sets error code 5, the block's warps leave together once
the copies still in flight have landed, and the run reports LPA_ERR_TIMEOUT.
The test hook lpa_graph_debug_stall makes the first block of one row kernel to
produce a tile leave that tile's index copy unissued, so the waits on it run
out; the next run must start clean and still match the oracle label for
label."""
import time

import numpy as np
import pytest

import lpa_inputs as L
import oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lpa():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    import paper_2312_08140_gb300 as m
    m.load()
    return m


@pytest.mark.parametrize("block_threads", [512, 256, 128])
def test_a_stalled_copy_reports_timeout_and_leaves_the_context_usable(lpa, block_threads):
    import torch
    # raw R-MAT rows repeat neighbours, so no first-sweep shortcut: every row
    # kernel streams its rows through the copied index tiles from sweep 1
    g = L.rmat(15, 16, seed=3, dedup=False)
    deg = np.diff(g.off)
    assert deg.max() > 2048 and ((deg > 128) & (deg <= 512)).any() and ((deg > 512) & (deg <= 2048)).any()
    h = lpa.lpa_graph_create(g.n, g.nnz, g.off, g.idx, g.w)
    try:
        assert lpa.lpa_graph_props_get(h)["rows_distinct"] == 0
        out = torch.empty(g.n, dtype=torch.int32, device="cuda")
        lpa.lpa_graph_debug_stall(h, block_threads)
        t0 = time.time()
        with pytest.raises(lpa.LpaError) as e:
            lpa.lpa_run(h, "async", 0.05, 20, out)
        assert e.value.status == lpa.LPA_ERR_TIMEOUT, e.value
        assert time.time() - t0 < 60
        # the next run starts clean and is exact
        ref, it, changed = O.lpa_sync(g.off, g.idx, g.w, 0.05, 20)
        info = lpa.lpa_run(h, "sync", 0.05, 20, out)
        assert info.iterations == it
        assert np.array_equal(out.cpu().numpy(), ref)
    finally:
        lpa.lpa_graph_destroy(h)


def test_the_hook_rejects_other_sizes(lpa):
    g = L.rmat(8, 8, seed=1)
    h = lpa.lpa_graph_create(g.n, g.nnz, g.off, g.idx, g.w)
    try:
        with pytest.raises(lpa.LpaError) as e:
            lpa.lpa_graph_debug_stall(h, 64)
        assert e.value.status == lpa.LPA_ERR_INVALID_ARG
        lpa.lpa_graph_debug_stall(h, 0)
    finally:
        lpa.lpa_graph_destroy(h)
