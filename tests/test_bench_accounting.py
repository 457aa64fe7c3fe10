"""Host logic of bench.py's roofline accounting (kernel_bytes): the
algorithmic bytes per launch of each degree-bin kernel from the per-sweep
counts of a profiled run, worked by hand on a two-sweep profile."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _profile():
    # sweep 0: bins 0, 1 and 4 have vertices (2, 3 are statically empty)
    return {"iterations": 2,
            "sweep_ms": [[1.0, 2.0, 0.002, 0.002, 4.0], [0.5, 1.0, 0.002, 0.002, 2.0]],
            "bin_vertices": [[10, 5, 0, 0, 1], [4, 5, 0, 0, 1]],
            "bin_entries": [[30, 100, 0, 0, 5000], [12, 100, 0, 0, 5000]],
            "bin_changed": [[10, 5, 0, 0, 1], [2, 0, 0, 0, 0]],
            "bin_changed_entries": [[30, 100, 0, 0, 5000], [6, 0, 0, 0, 0]]}


def test_sync_bytes_by_hand():
    # per vertex 24 B, per entry 4 + weight bytes + 4 (label), per changed
    # vertex 8 B in sync mode, plus 1 B per entry of a changed row
    out = bench.kernel_bytes(_profile(), wbytes=1, sync=True, passes=1)
    small = (10 * 24 + 30 * 9 + 10 * 8 + 30) + (4 * 24 + 12 * 9 + 2 * 8 + 6)
    assert out["k_sweep_small"]["bytes"] == small
    assert out["k_sweep_small"]["launches"] == 2 and out["k_sweep_small"]["ms"] == 1.5
    # statically empty bins are never launched: no bytes, time or launches
    for b in ("k_sweep_block128", "k_sweep_block256"):
        assert out[b] == {"bytes": 0.0, "ms": 0.0, "launches": 0}


def test_first_sync_sweep_of_repeat_free_graph_reads_no_labels():
    plain = bench.kernel_bytes(_profile(), wbytes=0, sync=True, passes=1)
    rf = bench.kernel_bytes(_profile(), wbytes=0, sync=True, passes=1, rows_distinct=True)
    # only sweep 0 drops the 4 B label gather per entry
    for b, e0 in (("k_sweep_small", 30), ("k_sweep_warp", 100), ("k_sweep_block512", 5000)):
        assert plain[b]["bytes"] - rf[b]["bytes"] == 4 * e0


def test_async_counts_two_passes_and_4_byte_changes():
    out = bench.kernel_bytes(_profile(), wbytes=0, sync=False, passes=2, rows_distinct=True)
    # async: labels are always gathered, a change writes 4 B
    warp = (5 * 24 + 100 * 8 + 5 * 4 + 100) + (5 * 24 + 100 * 8)
    assert out["k_sweep_warp"]["bytes"] == warp and out["k_sweep_warp"]["launches"] == 4
