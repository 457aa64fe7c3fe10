"""Quality bound for the asynchronous mode.

Algorithm 1 updates labels in place inside a loop over the vertices whose
order it leaves open, so serial runs in different orders are all executions
of it, and their modularity (Eq. 1) differs: on small planted-partition
graphs by several hundredths.  A parallel run is one more interleaving.  The
tests hold it to the lowest modularity among serial runs in seeded random
vertex orders, less a slack (a parallel pass updates many vertices at once
and lands 0.01-0.03 below the serial runs on planted partitions); above max_n
vertices, where several serial runs take minutes, to the ascending run less
the same slack (the 4096x4096 grid's async runs that stop after 3 sweeps
reach 0.633 against the ascending run's 0.648).

Serial runs in monotone id order (ascending or descending) are left out of
the floor when random orders are available: with the smallest-id tie-break a
monotone visit order lets the smallest ids sweep through the graph, and on
planted partitions such runs end with one community (Q = 0) where random
orders reach 0.3-0.8 -- a floor at 0 would test nothing.  The paper's own
CPU design walks contiguous chunks in ascending order and can end the same
way (cpu_parallel: Q = 0 with 1 or 16 threads on a 3000-vertex planted
partition), so its test keeps the monotone orders (include_monotone), and so
do the tests of batched and served runs: inside a batch, a graph's
asynchronous runs spread much more widely than alone (graph 0 of a batch of
eight 140K-vertex planted partitions: Q 0.45-0.76 across runs, 0.73-0.76
alone).
"""
import numpy as np

import oracle as O

SLACK_ORDERS = 0.03
SLACK_ASCENDING = 0.03


def async_floor(g, tau=0.05, iters=20, random_orders=6, seed=0, max_n=300_000, prune_other=False,
                include_monotone=False):
    """Modularity the asynchronous GPU run must reach on graph g (with
    prune_other: runs under FLPA's pruning rule, against serial runs under the
    same rule)."""
    orders = [None]
    if g.n <= max_n:
        rng = np.random.default_rng(seed)
        orders = [rng.permutation(g.n) for _ in range(random_orders)]
        if include_monotone:
            orders += [None, np.arange(g.n)[::-1]]
    qs = [O.modularity(g.off, g.idx, g.w,
                       O.lpa_async_ex(g.off, g.idx, g.w, tau, iters, order=o, prune_other=prune_other)[0])
          for o in orders]
    return min(qs) - (SLACK_ORDERS if len(orders) > 1 else SLACK_ASCENDING)
