"""Host logic of bench.py: the roofline accounting (kernel_bytes: the
algorithmic bytes per launch of each degree-bin kernel from the per-sweep
counts of a profiled run, worked by hand on a two-sweep profile), the
validity of the recorded ncu traffic, the clock summary, and the modes and
config the two arms share."""
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
    for b in ("k_sweep_rows<128>", "k_sweep_rows<256>"):
        assert out[b] == {"bytes": 0.0, "ms": 0.0, "launches": 0}


def test_first_sync_sweep_of_repeat_free_graph_reads_no_labels():
    plain = bench.kernel_bytes(_profile(), wbytes=0, sync=True, passes=1)
    rf = bench.kernel_bytes(_profile(), wbytes=0, sync=True, passes=1, rows_distinct=True)
    # only sweep 0 drops the 4 B label gather per entry
    for b, e0 in (("k_sweep_small", 30), ("k_sweep_warp", 100), ("k_sweep_rows<512>", 5000)):
        assert plain[b]["bytes"] - rf[b]["bytes"] == 4 * e0


def test_async_counts_two_passes_and_4_byte_changes():
    out = bench.kernel_bytes(_profile(), wbytes=0, sync=False, passes=2, rows_distinct=True)
    # async: labels are always gathered, a change writes 4 B
    warp = (5 * 24 + 100 * 8 + 5 * 4 + 100) + (5 * 24 + 100 * 8)
    assert out["k_sweep_warp"]["bytes"] == warp and out["k_sweep_warp"]["launches"] == 4


def test_traffic_is_reported_only_for_the_captured_sources(monkeypatch):
    """The ncu DRAM bytes stand for the kernel sources, workload and storage
    order they were captured from: another sha1 (any edit to those files),
    workload or order turns them into null."""
    import argparse
    args = argparse.Namespace(workload="rmat27", order="caller")
    assert bench.measured_traffic("k_no_such_kernel", args) is None
    k = "k_sweep_rows<512>"
    rec = dict(bench.TRAFFIC[k])
    got = bench.measured_traffic(k, args)
    assert got is None or got == rec["bytes_per_launch"]
    assert bench.measured_traffic(k, argparse.Namespace(workload="rmat27", order="degree")) is None
    assert bench.measured_traffic(k, argparse.Namespace(workload="rmat25", order="caller")) is None
    monkeypatch.setitem(bench.TRAFFIC, k, dict(rec, sha1="0" * 40))
    assert bench.measured_traffic(k, args) is None


def test_clock_summary_takes_the_median_and_every_active_reason():
    """nvidia-smi CSV rows (index, sm, max sm, power, active mask, then four
    reasons) become the median SM clock and the set of reasons seen Active;
    malformed rows are skipped."""
    class _Done:
        def terminate(self):
            pass

        def wait(self, timeout=None):
            return 0

        def join(self, timeout=None):
            pass

    cs = bench.ClockSampler(0)
    cs.proc, cs.thread = _Done(), _Done()
    cs.lines = ["0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
                "0, 1980, 2070, 1390.5, 0x4, Not Active, Not Active, Not Active, Active",
                "0, 2040, 2070, 1200.0, 0x0, Not Active, Not Active, Not Active, Not Active",
                "garbled",
                "0, [N/A], 2070, 0, 0x0, Not Active, Not Active, Not Active, Not Active"]
    got = cs.stop()
    assert got == {"sm_mhz": 2040.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    assert bench.ClockSampler(0).stop() is None


def test_both_arms_share_modes_and_config():
    """The oracle arm runs the same mode strings as the GPU arm, each through
    the matching oracle function, and prints the same config object."""
    import argparse

    import lpa_inputs as L
    import oracle as O
    args = argparse.Namespace(workload="rmat22+grid4096", tie="strict", prune="paper", order="caller")
    assert bench.workload_modes(args) == ("sync", "async")
    assert bench.run_config(args, 1)["tie_break"] == "strict"
    args = argparse.Namespace(workload="rmat22+grid4096", tie="nonstrict", prune="other", order="caller")
    assert bench.workload_modes(args) == ("sync+nonstrict", "async+nonstrict+prune_other")
    cfg = bench.run_config(args, 2)
    assert cfg["async_pruning"] == "FLPA rule" and cfg["parallelism"] == "replicas x2"
    g = L.planted_partition(n=600, blocks=6, intra=10.0, inter=1.0, seed=2)
    want = {"sync": O.lpa_sync(g.off, g.idx, g.w, bench.TAU, 20),
            "sync+nonstrict": O.lpa_sync(g.off, g.idx, g.w, bench.TAU, 20, nonstrict=True),
            "async": O.lpa_async(g.off, g.idx, g.w, bench.TAU, 20),
            "async+nonstrict": O.lpa_async(g.off, g.idx, g.w, bench.TAU, 20, nonstrict=True),
            "async+prune_other": O.lpa_async_ex(g.off, g.idx, g.w, bench.TAU, 20, prune_other=True)[:3]}
    for mode, (C, it, ch) in want.items():
        C2, it2, ch2 = bench.oracle_run(g, mode, 20)
        assert C2.tolist() == C.tolist() and it2 == it and ch2.tolist() == ch.tolist(), mode


def test_oracle_row_sample_times_the_sampled_rows():
    """The CPU baseline of a graph too large for a whole oracle sweep times
    the oracle's first sweep over a contiguous range of rows: the entries it
    reports are exactly those rows' entries, and the range starts where asked."""
    import lpa_inputs as L
    g = L.rmat(13, 16, seed=2)
    for mode in ("async", "sync"):
        e, t, (v0, v1) = bench.oracle_rows_sample(g, mode, 1000, 20_000)
        assert v0 == 1000 and e == int(g.off[v1] - g.off[v0]) >= 20_000 and t > 0
    e, t, (v0, v1) = bench.oracle_rows_baseline(g, "async", target_s=0.05)
    assert e == int(g.off[v1] - g.off[v0]) and v0 == g.n // 3
    info = bench.host_cpu()
    assert info["nproc"] >= 1
