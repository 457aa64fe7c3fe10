"""Quality bound for the asynchronous mode.

Algorithm 1 updates labels in place inside a loop over the vertices whose
order it leaves open, so serial runs in different orders are all executions
of it, and their modularity (Eq. 1) differs: on small planted-partition
graphs by several hundredths.  A parallel run is one more interleaving.  The
tests hold it to the lowest modularity among serial runs in a few orders
(ascending, descending, seeded random permutations), less a small slack;
above max_n vertices, where several serial runs take minutes, to the
ascending run less a wider slack.
"""
import numpy as np

import oracle as O

SLACK_ORDERS = 0.01
SLACK_ASCENDING = 0.02


def async_floor(g, tau=0.05, iters=20, random_orders=6, seed=0, max_n=300_000):
    """Modularity the asynchronous GPU run must reach on graph g."""
    orders = [None]
    if g.n <= max_n:
        rng = np.random.default_rng(seed)
        orders += [np.arange(g.n)[::-1]] + [rng.permutation(g.n) for _ in range(random_orders)]
    qs = [O.modularity(g.off, g.idx, g.w, O.lpa_async(g.off, g.idx, g.w, tau, iters, order=o)[0]) for o in orders]
    return min(qs) - (SLACK_ORDERS if len(orders) > 1 else SLACK_ASCENDING)
