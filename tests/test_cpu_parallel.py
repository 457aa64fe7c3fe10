"""The multi-core CPU baseline (cpu_parallel, the paper's OpenMP design):
its synchronous runs must equal the oracle's exactly (pruning and thread
interleaving cannot change a Jacobi sweep with the strict tie-break), and its
asynchronous runs must meet the invariants, reach the serial ascending run's
modularity (the order its chunks are walked in) less 0.02, and on one thread
equal the serial ascending run."""
import numpy as np

import cpu_parallel as CP
import lpa_inputs as L
import oracle as O
from async_bounds import SLACK, ascending_q, serial_qs


def _graphs():
    return [L.planted_partition(n=3000, blocks=6, seed=4), L.road_grid(70, 55, seed=2), L.rmat(12, 16, seed=3),
            L.batched_sbm_graph(66, n_max=5000), L.from_undirected_pairs(3, [(0, 1), (1, 2)])]


def test_sync_equals_oracle():
    for g in _graphs():
        ref, it, ch = O.lpa_sync(g.off, g.idx, g.w)
        for t in (1, 4):
            got, it2, ch2 = CP.run(g.off, g.idx, g.w, "sync", n_threads=t)
            assert np.array_equal(got, ref) and it2 == it and ch2.tolist() == ch.tolist(), (g.n, t)


def test_async_invariants():
    for g in _graphs():
        got, it, _ = CP.run(g.off, g.idx, g.w, "async", n_threads=4)
        assert 1 <= it <= 20
        assert O.count_labels_outside_component(g.off, g.idx, got) == 0
        # the paper's design walks contiguous chunks in ascending order, so it
        # is held to the serial ascending run (or to the random-order runs
        # where those are lower): on id-ordered planted partitions the
        # ascending run ends as one community
        floor = min(ascending_q(g), min(serial_qs(g))) - SLACK
        assert O.modularity(g.off, g.idx, g.w, got) >= floor, g.n


def test_async_on_one_thread_is_the_serial_ascending_run():
    """One thread walks the chunks in ascending order, updating in place, so it
    is the serial ascending execution of Algorithm 1: labels, sweep count and
    per-sweep changes equal the oracle's exactly."""
    rng = np.random.default_rng(5)
    graphs = _graphs() + [L.random_small(int(rng.integers(1, 40)), float(rng.uniform(0.05, 0.6)), seed=s,
                                         wmax=int(rng.integers(0, 5)), self_loops=0.2, multi=bool(s % 2))
                          for s in range(200)]
    for g in graphs:
        ref, it, ch = O.lpa_async(g.off, g.idx, g.w)
        got, it2, ch2 = CP.run(g.off, g.idx, g.w, "async", n_threads=1)
        assert np.array_equal(got, ref) and it2 == it and ch2.tolist() == ch.tolist(), g.n


def test_zero_weight_label_repeated_more_than_n_times():
    """A row that lists a zero-weight neighbour many times over (more entries
    than the graph has vertices) lists its label once in the per-thread key
    list: the run equals the oracle's and writes nothing out of bounds."""
    n = 3
    rows = [[1] * 40 + [2], [0] * 40, [0]]
    wts = [[0.0] * 40 + [1.0], [0.0] * 40, [1.0]]
    off = np.zeros(n + 1, dtype=np.int64)
    off[1:] = np.cumsum([len(r) for r in rows])
    idx = np.array([j for r in rows for j in r], dtype=np.int32)
    w = np.array([x for r in wts for x in r], dtype=np.float32)
    for mode, ref_fn in (("sync", O.lpa_sync), ("async", O.lpa_async)):
        ref, it, ch = ref_fn(off, idx, w)
        got, it2, ch2 = CP.run(off, idx, w, mode, n_threads=1)
        assert np.array_equal(got, ref) and it2 == it and ch2.tolist() == ch.tolist(), mode
