"""A lockstep model of the asynchronous warp schedule (test infrastructure).

In an asynchronous pass the GPU hands each warp a batch of B consecutive
frontier vertices, and the warps run side by side.  The model advances every
batch by one vertex per round.  Each round reads the labels as they stood
before it and applies its changes at its end, with Algorithm 1's pick (Eq. 2,
the smallest label among the most weighted) and re-marking (Section 4.1.4).

* B = 1 puts the whole frontier in one round: a Jacobi sweep, which is the
  synchronous mode (tests/test_async_model.py checks that the model then
  gives the synchronous oracle's labels and counts exactly).
* Larger B lets the later vertices of a batch see the changes of the earlier
  ones, as the serial loop of Algorithm 1 does; with one batch holding the
  whole frontier, a sweep walks the frontier in order like the serial loop
  (vertices re-marked during the sweep wait for the next one here).

The model has no catch-up pass and ignores timing, so it predicts the
quality of a schedule, not its labels.  Plain Python loops: small graphs only.
"""
import numpy as np

import oracle as O


def lockstep_run(g, B, tau=0.05, max_iters=20):
    """Runs the model with batches of B frontier vertices; returns
    (labels int32[n], sweeps, per-sweep changed counts)."""
    n, off, idx = g.n, g.off, g.idx
    w = g.w if g.w is not None else np.ones(g.nnz)
    C = np.arange(n, dtype=np.int64)
    unprocessed = np.ones(n, dtype=bool)
    thr = int(np.floor(tau * n))
    changed = []
    for _ in range(max_iters):
        front = np.flatnonzero(unprocessed)
        nb = (len(front) + B - 1) // B
        dn = 0
        for r in range(B):
            before = C.copy()
            updates = []
            for b in range(nb):
                k = b * B + r
                if k >= len(front):
                    continue
                v = int(front[k])
                unprocessed[v] = False
                sums = {}
                for e in range(off[v], off[v + 1]):
                    j = int(idx[e])
                    if j != v:
                        c = int(before[j])
                        sums[c] = sums.get(c, 0.0) + float(w[e])
                if not sums:
                    continue
                best = max(sums.values())
                pick = min(c for c, s in sums.items() if s == best)
                if pick != before[v]:
                    updates.append((v, pick))
            for v, pick in updates:
                C[v] = pick
                dn += 1
                for e in range(off[v], off[v + 1]):
                    if int(idx[e]) != v:
                        unprocessed[idx[e]] = True
        changed.append(dn)
        if dn <= thr:
            break
    return C.astype(np.int32), len(changed), changed


def lockstep_q(g, B, tau=0.05, max_iters=20):
    labels, _, _ = lockstep_run(g, B, tau, max_iters)
    return O.modularity(g.off, g.idx, g.w, labels)
