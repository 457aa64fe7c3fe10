"""The acceptance rule of the asynchronous mode (async_bounds) on made-up
modularity samples: which serial statistic the GPU median is held to, and
that the rule rejects what it should."""
import pytest

from async_bounds import SLACK, assert_async_quality, quality_reference


def test_concentrated_serial_runs_use_the_median():
    qs = [0.750, 0.752, 0.753, 0.753, 0.754, 0.755, 0.756, 0.741]
    ref, kind = quality_reference(qs)
    assert kind == "median" and ref == pytest.approx(0.753)


def test_bimodal_serial_runs_use_the_lower_quartile():
    # seven runs flood a block, nine recover it
    qs = [0.14, 0.05, 0.44, 0.09, 0.32, 0.11, 0.02, 0.44, 0.45, 0.44, 0.13, 0.44, 0.43, 0.42, 0.14, 0.45]
    ref, kind = quality_reference(qs)
    assert kind == "lower quartile"
    # sorted runs 0.02, 0.05, 0.09, 0.11, 0.13, ...: position 15 / 4 = 3.75 -> 0.11 + 0.75 * 0.02
    assert ref == pytest.approx(0.125)


def test_rule_accepts_and_rejects():
    qs = [0.750, 0.752, 0.753, 0.753, 0.754, 0.755, 0.756, 0.741]
    assert_async_quality([0.74, 0.74, 0.735, 0.75, 0.745], qs)        # median 0.74 >= 0.753 - 0.02
    with pytest.raises(AssertionError):
        assert_async_quality([0.73, 0.73, 0.73, 0.75, 0.75], qs)       # median 0.73 < 0.733
    with pytest.raises(AssertionError):
        assert_async_quality([0.75, 0.75, 0.75, 0.75, 0.72 - SLACK], qs)   # one run below min - 0.02
