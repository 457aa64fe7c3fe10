"""The acceptance rule of the asynchronous mode (async_bounds) on made-up
modularity samples: which serial statistic the GPU median is held to, and
that the rule rejects what it should."""
import pytest

from async_bounds import MULTIMODAL_RUNS, SLACK, assert_async_quality, gpu_runs, quality_reference


def test_concentrated_serial_runs_use_the_median():
    qs = [0.750, 0.752, 0.753, 0.753, 0.754, 0.755, 0.756, 0.741]
    ref, kind = quality_reference(qs)
    assert kind == "median" and ref == pytest.approx(0.753)


def test_wide_serial_runs_keep_only_the_range_rule():
    # serial runs from 0 to 0.61: a block floods or not by the order alone
    qs = [0.0, 0.0, 0.25, 0.26, 0.26, 0.36, 0.37, 0.47, 0.47, 0.51, 0.54, 0.58, 0.58, 0.61, 0.26, 0.26]
    ref, kind = quality_reference(qs)
    assert ref is None and kind == "range"
    assert_async_quality([0.14, 0.14, 0.0, 0.14, 0.0], qs)
    with pytest.raises(AssertionError):
        assert_async_quality([0.14, 0.14, -0.03, 0.14, 0.0], qs)


def test_bimodal_serial_runs_use_the_lower_quartile():
    # seven runs flood a block, nine recover it (a range of 0.23)
    qs = [0.34, 0.25, 0.44, 0.29, 0.42, 0.31, 0.22, 0.44, 0.45, 0.44, 0.33, 0.44, 0.43, 0.42, 0.34, 0.45]
    ref, kind = quality_reference(qs)
    assert kind == "lower quartile"
    # sorted runs 0.22, 0.25, 0.29, 0.31, 0.33, ...: position 15 / 4 = 3.75 -> 0.31 + 0.75 * 0.02
    assert ref == pytest.approx(0.325)


def test_rule_accepts_and_rejects():
    qs = [0.750, 0.752, 0.753, 0.753, 0.754, 0.755, 0.756, 0.741]
    assert_async_quality([0.74, 0.74, 0.735, 0.75, 0.745], qs)        # median 0.74 >= 0.753 - 0.02
    with pytest.raises(AssertionError):
        assert_async_quality([0.73, 0.73, 0.73, 0.75, 0.75], qs)       # median 0.73 < 0.733
    with pytest.raises(AssertionError):
        assert_async_quality([0.75, 0.75, 0.75, 0.75, 0.72 - SLACK], qs)   # one run below min - 0.02


def test_spread_serial_runs_take_more_gpu_runs():
    concentrated = [0.750, 0.752, 0.753, 0.753, 0.754, 0.755, 0.756, 0.741]
    spread = [0.0, 0.24, 0.24, 0.37, 0.52, 0.57, 0.62, 0.71]
    assert gpu_runs(concentrated) == 5
    assert gpu_runs(spread) == MULTIMODAL_RUNS and gpu_runs(spread, 20) == 20


def test_neighbourhood_bound_of_the_local_argmax_check():
    import numpy as np
    import lpa_inputs as L
    from async_bounds import assert_local_max_bound, neighbourhood_bound
    # a star with centre 0 and 5 leaves, plus an edge 6-7: degrees 5, 1 x 5, 1, 1
    g = L.from_undirected_pairs(8, [(0, k) for k in range(1, 6)] + [(6, 7)])
    assert neighbourhood_bound(g, 0) == 0
    assert neighbourhood_bound(g, 1) == 5
    assert neighbourhood_bound(g, 2) == 6
    assert neighbourhood_bound(g, 100) == 8
    # the centre and its five leaves off their argmax (each leaf carries its
    # own id, the centre a label none of its neighbours has): six vertices,
    # allowed when the last sweep changed two vertices (bound 5 + 1), not one
    lab = np.array([7, 1, 2, 3, 4, 5, 6, 6], dtype=np.int32)
    assert assert_local_max_bound(g, lab, {"iterations": 2, "exit_reason": 0, "changed": [8, 2]}) == 6
    for last in (1, 0):
        with pytest.raises(AssertionError):
            assert_local_max_bound(g, lab, {"iterations": 2, "exit_reason": 0, "changed": [8, last]})
    # an exit by the cap is not bounded
    assert assert_local_max_bound(g, lab, {"iterations": 2, "exit_reason": 1, "changed": [8, 0]}) == 6


def test_tolerance_fraction_of_the_local_argmax_check():
    import numpy as np
    import lpa_inputs as L
    from async_bounds import LOCAL_MAX_MIN_N, assert_local_max_bound
    # a path of 2000 vertices in pairs (0-1, 2-3, ...) joined in a chain; the
    # pair partner labels make every vertex its pair's label -> at argmax
    n = 2000
    assert n >= LOCAL_MAX_MIN_N
    pairs = [(2 * i, 2 * i + 1) for i in range(n // 2)]
    g = L.from_undirected_pairs(n, pairs)
    lab = np.repeat(np.arange(0, n, 2), 2).astype(np.int32)
    info = {"iterations": 1, "exit_reason": 0, "changed": [200]}
    assert assert_local_max_bound(g, lab, info) == 0
    # 101 pairs split: 202 vertices off, above floor(0.05 * 2000) = 100
    bad = lab.copy()
    bad[1:404:4] = np.arange(1, 404, 4)[: bad[1:404:4].size]
    assert O_count(g, bad) > 100
    # within the neighbourhood bound (every vertex changed last), above tau N
    with pytest.raises(AssertionError, match="off|202"):
        assert_local_max_bound(g, bad, {"iterations": 1, "exit_reason": 0, "changed": [n]})


def O_count(g, lab):
    import oracle as O
    return O.count_not_local_max(g.off, g.idx, g.w, lab)
