"""Pins for the CPU oracle: each check ties it to something other than itself.

- hand-worked runs derived on paper from Algorithm 1 and Eq. 2 (tests/golden),
- brute-force enumeration of the label space for the update rule (Eq. 2),
- invariants any label propagation run has (labels travel along edges only;
  a synchronous fixed point is stable),
- modularity (Eq. 1) closed forms and the networkx library routine,
- connected components from scipy for the component checker, and enumerated
  Eq. 2 sums for the local-maximum checker,
- planted mistakes: broken copies of the oracle source must fail these pins.
"""
import json
import os
import subprocess

from fractions import Fraction

import numpy as np
import pytest

import lpa_inputs as L
import oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _golden_cases():
    with open(os.path.join(ROOT, "tests", "golden", "hand_worked.json")) as f:
        return json.load(f)["cases"]


def _case_graph(case):
    if "clique" in case:
        k = case["clique"]
        pairs = [(u, v) for u in range(k) for v in range(u + 1, k)]
        return L.from_undirected_pairs(case["n"], pairs)
    return L.from_undirected_pairs(case["n"], [tuple(p) for p in case["pairs"]], case.get("weights"))


def _run_case(case, mod=O):
    g = _case_graph(case)
    kw = dict(tau=case.get("tau", 0.05), max_iters=case.get("max_iters", 20))
    if "order" in case:
        kw["order"] = case["order"]
    fn = mod.lpa_sync if case["mode"] == "sync" else mod.lpa_async
    return fn(g.off, g.idx, g.w, **kw)


@pytest.mark.parametrize("case", _golden_cases(), ids=lambda c: c["name"])
def test_hand_worked(case):
    C, it, changed = _run_case(case)
    assert C.tolist() == case["labels"]
    assert it == case["iterations"]
    assert changed.tolist() == case["changed"]


# ---------------------------------------------------------------- Eq. 2 --
def _label_sums(g, C, i):
    """{c: K_{i->c}} over i's entries other than self-loops (Eq. 2's sums)."""
    sums = {}
    for e in range(int(g.off[i]), int(g.off[i + 1])):
        j = int(g.idx[e])
        if j == i:
            continue
        c = int(C[j])
        sums[c] = sums.get(c, 0.0) + (1.0 if g.w is None else float(g.w[e]))
    return sums


def _enumerated_pick(g, C, i):
    """Eq. 2 by enumerating every candidate label c = 0..n-1 in increasing order:
    K_{i->c} is summed over the row directly; the first c reaching the maximum
    wins.  A vertex with no neighbour besides itself keeps C[i]."""
    n = g.n
    row = range(int(g.off[i]), int(g.off[i + 1]))
    others = [e for e in row if int(g.idx[e]) != i]
    if not others:
        return int(C[i])
    present = {int(C[int(g.idx[e])]) for e in others}
    best, best_w = None, None
    for c in range(n):
        if c not in present:
            continue
        K_ic = sum((1.0 if g.w is None else float(g.w[e])) for e in others if int(C[int(g.idx[e])]) == c)
        if best_w is None or K_ic > best_w:
            best, best_w = c, K_ic
    return best


def _random_cases(count, seed0=0):
    rng = np.random.default_rng(12345)
    for t in range(count):
        n = int(rng.integers(1, 13))
        g = L.random_small(n, float(rng.uniform(0.1, 0.8)), seed=seed0 + t,
                           wmax=int(rng.integers(0, 5)), self_loops=0.2, multi=bool(t % 2))
        C = rng.integers(0, n, size=n).astype(np.int32) if n else np.zeros(0, np.int32)
        yield g, C


def test_pick_matches_enumeration():
    checked = 0
    for g, C in _random_cases(1500):
        Cn, dN = O.sync_sweep(g.off, g.idx, g.w, C)
        for i in range(g.n):
            assert Cn[i] == _enumerated_pick(g, C, i)
            checked += 1
        assert dN == int(np.sum(Cn != C))
    assert checked > 5000


def test_sync_run_is_iterated_sweeps():
    """lpa_sync equals sweeps applied from C = [0..n) until dN/N <= tau or the cap."""
    for g, _ in _random_cases(300, seed0=5000):
        if g.n == 0:
            continue
        for tau, cap in ((0.05, 20), (0.3, 7), (0.0, 3)):
            C = np.arange(g.n, dtype=np.int32)
            hist = []
            for _ in range(cap):
                Cn = np.array([_enumerated_pick(g, C, i) for i in range(g.n)], dtype=np.int32)
                hist.append(int(np.sum(Cn != C)))
                C = Cn
                if Fraction(hist[-1]) <= Fraction(str(tau)) * g.n:
                    break
            Co, it, ho = O.lpa_sync(g.off, g.idx, g.w, tau=tau, max_iters=cap)
            assert Co.tolist() == C.tolist() and it == len(hist) and ho.tolist() == hist


def _serial_async_restated(g, tau, cap, order=None, prune_other=False):
    """Algorithm 1 with one thread, written as a worklist of pending vertices
    scanned in increasing id order (or in `order`); each pick is the
    enumerated Eq. 2.  prune_other: a changed vertex adds only neighbours not
    already carrying its new label (the FLPA rule, Section 2)."""
    n = g.n
    C = np.arange(n, dtype=np.int32)
    pending = set(range(n))
    hist = []
    seq = list(range(n)) if order is None else [int(x) for x in order]
    for _ in range(cap):
        dN = 0
        for i in seq:
            if i in pending:
                pending.discard(i)
                c = _enumerated_pick(g, C, i)
                if c != C[i]:
                    C[i] = c
                    dN += 1
                    for e in range(int(g.off[i]), int(g.off[i + 1])):
                        j = int(g.idx[e])
                        if j != i and not (prune_other and C[j] == c):
                            pending.add(j)
        hist.append(dN)
        if Fraction(dN) <= Fraction(str(tau)) * n:
            break
    return C, len(hist), hist


def test_async_matches_restatement():
    for g, _ in _random_cases(400, seed0=9000):
        if g.n == 0:
            continue
        C, it, h = _serial_async_restated(g, 0.05, 20)
        Co, ito, ho = O.lpa_async(g.off, g.idx, g.w)
        assert Co.tolist() == C.tolist() and ito == it and ho.tolist() == h


# ----------------------------------------------------------- invariants --
def _component_ids(g):
    import scipy.sparse as sp
    from scipy.sparse.csgraph import connected_components
    A = sp.csr_matrix((np.ones(g.nnz), g.idx, g.off), shape=(g.n, g.n))
    return connected_components(A, directed=False)[1]


@pytest.mark.parametrize("mode", ["sync", "async"])
def test_labels_stay_in_component(mode):
    fn = O.lpa_sync if mode == "sync" else O.lpa_async
    for g, _ in _random_cases(300, seed0=20000):
        if g.n == 0:
            continue
        C, _, _ = fn(g.off, g.idx, g.w)
        comp = _component_ids(g)
        assert np.all(comp[C] == comp[np.arange(g.n)])
        assert O.count_labels_outside_component(g.off, g.idx, C) == 0


def test_sync_fixed_point_is_stable():
    g = L.planted_partition()
    C, it, h = O.lpa_sync(g.off, g.idx, g.w, tau=0.0, max_iters=100)
    assert h[-1] == 0
    C2, dN = O.sync_sweep(g.off, g.idx, g.w, C)
    assert dN == 0 and np.array_equal(C, C2)
    assert O.count_not_local_max(g.off, g.idx, g.w, C) == 0


def test_bridged_cliques_split_in_sync_mode():
    for k in range(3, 9):
        pairs = [(u, v) for u in range(k) for v in range(u + 1, k)]
        pairs += [(u + k, v + k) for u, v in pairs] + [(k - 1, k)]
        g = L.from_undirected_pairs(2 * k, pairs)
        C, it, _ = O.lpa_sync(g.off, g.idx, None)
        assert len(set(C[:k].tolist())) == 1 and len(set(C[k:].tolist())) == 1 and C[0] != C[k]
        assert it == (4 if k == 3 else 3)


def test_component_checker_matches_scipy():
    rng = np.random.default_rng(7)
    for g, _ in _random_cases(200, seed0=30000):
        if g.n == 0:
            continue
        comp = _component_ids(g)
        C = rng.integers(0, g.n, size=g.n).astype(np.int32)
        assert O.count_labels_outside_component(g.off, g.idx, C) == int(np.sum(comp[C] != comp))


def test_local_max_checker_closed_cases():
    n = 6
    g = L.from_undirected_pairs(n, [(u, v) for u in range(n) for v in range(u + 1, n)])
    # distinct labels in K_n: each vertex's own label is absent among its neighbours
    assert O.count_not_local_max(g.off, g.idx, None, np.arange(n, dtype=np.int32)) == n
    assert O.count_not_local_max(g.off, g.idx, None, np.zeros(n, dtype=np.int32)) == 0


def _enumerated_not_local_max(g, C):
    """Vertices whose own label's weight K_{i->C_i} is below the best label's
    (Eq. 2's sums, enumerated); a label outside [0, n) counts, a vertex with no
    neighbour but itself does not."""
    bad = 0
    for i in range(g.n):
        if not 0 <= int(C[i]) < g.n:
            bad += 1
            continue
        sums = _label_sums(g, C, i)
        if sums and sums.get(int(C[i]), 0.0) < max(sums.values()):
            bad += 1
    return bad


def test_local_max_checker_matches_enumeration():
    rng = np.random.default_rng(11)
    checked = 0
    for g, C in _random_cases(600, seed0=70000):
        if g.n == 0:
            continue
        # few distinct labels make ties common, which a tie-sensitive checker would miscount
        for lab in (C, rng.integers(0, min(g.n, 3), size=g.n).astype(np.int32),
                    O.lpa_sync(g.off, g.idx, g.w, tau=0.0, max_iters=2)[0]):
            assert O.count_not_local_max(g.off, g.idx, g.w, lab) == _enumerated_not_local_max(g, lab)
            checked += 1
    assert checked > 1500


def _checker_pins_pass(mod):
    rng = np.random.default_rng(13)
    for g, C in _random_cases(150, seed0=80000):
        if g.n == 0:
            continue
        if mod.count_labels_outside_component(g.off, g.idx, C) != int(np.sum(_component_ids(g)[C] != _component_ids(g))):
            return False
        few = rng.integers(0, min(g.n, 3), size=g.n).astype(np.int32)
        for lab in (C, few):
            if mod.count_not_local_max(g.off, g.idx, g.w, lab) != _enumerated_not_local_max(g, lab):
                return False
    return True


# ----------------------------------------------------------- modularity --
def test_modularity_closed_forms():
    # K_n, all singletons: sigma = 0, Sigma_c = n-1 each: Q = -n (n-1)^2 / (n(n-1))^2 = -1/n
    for n in (2, 3, 5, 9):
        g = L.from_undirected_pairs(n, [(u, v) for u in range(n) for v in range(u + 1, n)])
        assert O.modularity(g.off, g.idx, None, np.arange(n, dtype=np.int32)) == pytest.approx(-1.0 / n, abs=1e-14)
        # all in one community: sigma = 2m, Sigma = 2m: Q = 0
        assert O.modularity(g.off, g.idx, None, np.zeros(n, dtype=np.int32)) == pytest.approx(0.0, abs=1e-14)
    # c disjoint equal cliques, each its own community: Q = 1 - 1/c
    for c, k in ((2, 4), (3, 5), (5, 3)):
        pairs = [(u + b * k, v + b * k) for b in range(c) for u in range(k) for v in range(u + 1, k)]
        g = L.from_undirected_pairs(c * k, pairs)
        lab = np.repeat(np.arange(c) * k, k).astype(np.int32)
        assert O.modularity(g.off, g.idx, None, lab) == pytest.approx(1.0 - 1.0 / c, abs=1e-14)
    # two K5 joined by one edge, split at the bridge: m = 21, sigma_c = 20, Sigma_c = 21 -> 19/42
    pairs = [(u, v) for u in range(5) for v in range(u + 1, 5)]
    pairs += [(u + 5, v + 5) for u, v in pairs] + [(4, 5)]
    g = L.from_undirected_pairs(10, pairs)
    lab = np.array([0] * 5 + [5] * 5, dtype=np.int32)
    assert O.modularity(g.off, g.idx, None, lab) == pytest.approx(19.0 / 42.0, abs=1e-14)
    # weighted: a single weighted edge, both ends together -> 0; apart -> -1/2
    g = L.from_undirected_pairs(2, [(0, 1)], [3.0])
    assert O.modularity(g.off, g.idx, g.w, np.array([0, 0], np.int32)) == pytest.approx(0.0, abs=1e-15)
    assert O.modularity(g.off, g.idx, g.w, np.array([0, 1], np.int32)) == pytest.approx(-0.5, abs=1e-15)


def test_modularity_matches_networkx():
    nx = pytest.importorskip("networkx")
    rng = np.random.default_rng(3)
    for t in range(40):
        n = int(rng.integers(2, 60))
        g = L.random_small(n, float(rng.uniform(0.05, 0.5)), seed=40000 + t, wmax=int(rng.integers(0, 4)))
        if g.nnz == 0:
            continue
        C = rng.integers(0, max(1, n // 3), size=n).astype(np.int32)
        G = nx.Graph()
        G.add_nodes_from(range(n))
        for i in range(n):
            for e in range(int(g.off[i]), int(g.off[i + 1])):
                j = int(g.idx[e])
                if i < j:
                    G.add_edge(i, j, weight=1.0 if g.w is None else float(g.w[e]))
        comms = [set(np.flatnonzero(C == c).tolist()) for c in np.unique(C)]
        ref = nx.community.modularity(G, comms, weight="weight")
        assert O.modularity(g.off, g.idx, g.w, C) == pytest.approx(ref, abs=1e-12)


def test_planted_partition_true_blocks_modularity():
    """Expected value for 10 blocks with 14 intra / 2 inter mean degree: 14/16 - 1/10 = 0.775."""
    nx = pytest.importorskip("networkx")
    g = L.planted_partition()
    blocks = (np.arange(g.n) // 1000 * 1000).astype(np.int32)
    q = O.modularity(g.off, g.idx, g.w, blocks)
    assert abs(q - 0.775) < 0.01
    G = nx.Graph()
    G.add_nodes_from(range(g.n))
    src = np.repeat(np.arange(g.n), np.diff(g.off))
    G.add_edges_from(zip(src.tolist(), g.idx.tolist()))
    ref = nx.community.modularity(G, [set(range(b, b + 1000)) for b in range(0, g.n, 1000)])
    assert q == pytest.approx(ref, abs=1e-12)


# ------------------------------------------------------- planted mistakes --
# Each entry breaks one step of lpa_oracle.c in a plausible way; the pins
# above must catch every one of them.
MUTANTS = {
    "self_loops_counted": ("if ((int64_t)j == i) continue;            /* self-loops are skipped */", ""),
    "tie_to_largest": ("(v == best_w && c < best)", "(v == best_w && c > best)"),
    "strict_tolerance": ("return (double)dN <= thr;", "return (double)dN < thr;"),
    "tolerance_in_fp32": ("floor(tau * (double)n)", "floor((double)(float)tau * (double)n)"),
    "tolerance_rounded_up": ("floor(tau * (double)n)", "ceil(tau * (double)n)"),
    "unit_weights_ignored": ("return w ? (double)w[e] : 1.0;", "return 1.0;"),
    "sync_reads_in_place": ("C_out[i] = pick_t(&H, n, off, idx, w, prev, i, nonstrict ? it + 1 : 0);",
                            "C_out[i] = pick_t(&H, n, off, idx, w, C_out, i, nonstrict ? it + 1 : 0);"),
    "nonstrict_is_strict": ("c = most_weighted_label_rotated(H, n, r);", "c = most_weighted_label(H);"),
    "nonstrict_rotation_reversed": ("int64_t key = ((int64_t)c - (int64_t)r) % n;", "int64_t key = ((int64_t)r - (int64_t)c) % n;"),
    "async_no_remark": ("                unprocessed[j] = 1;\n", "                (void)j;\n"),
    "flpa_rule_ignored": ("if (prune_other && C_out[j] == c) continue;", ""),
    "flpa_rule_inverted": ("if (prune_other && C_out[j] == c) continue;", "if (prune_other && C_out[j] != c) continue;"),
    "async_counts_visits": ("if (c == C_out[i]) continue;", "if (c == C_out[i]) { ++dN; continue; }"),
    "async_order_ignored": ("const int64_t i = order ? order[k] : k;", "const int64_t i = k;"),
    "isolated_takes_zero": ("int32_t c = C[i];\n    if (used) {", "int32_t c = 0;\n    if (used) {"),
    "modularity_null_term_dropped": ("q = sigma / two_m - null_term;", "q = sigma / two_m;"),
    "modularity_sigma_by_other_end": ("Sigma[C[i]] += K_i;", "Sigma[C[idx[off[i]]]] += K_i;"),
    "local_max_tie_sensitive": ("if (own < H.val[best]) ++bad;", "if (own <= H.val[best] && C[i] != best) ++bad;"),
    "component_union_dropped": ("if (a != b) parent[a < b ? b : a] = (a < b ? a : b);", "(void)a; (void)b;"),
    "cap_off_by_one": ("while (it < max_iters) {\n        memcpy", "while (it <= max_iters) {\n        memcpy"),
}


def _tied_star(n=1000, labels=(5, 300, 301)):
    """Vertex 0 of an n-vertex graph joined to len(labels) vertices carrying
    the given distinct labels (unit weights): every label of vertex 0's row
    is tied at weight 1."""
    g = L.from_undirected_pairs(n, [(0, k + 1) for k in range(len(labels))])
    C = np.arange(n, dtype=np.int32)
    for k, lab in enumerate(labels):
        C[k + 1] = lab
    return g, C


def _nonstrict_frequencies(mod, sweeps=4000):
    g, C = _tied_star()
    picks = [mod.pick(g.off, g.idx, None, C, 0, sweep=t) for t in range(1, sweeps + 1)]
    return {lab: picks.count(lab) / sweeps for lab in (5, 300, 301)}, set(picks)


def _nonstrict_pins_pass(mod):
    """Non-strict tie-break (Section 4.1.5, read as a rotation of the label
    space by a per-(vertex, sweep) draw): the pick is always a most weighted
    label, equals the strict pick when the maximum is unique, and over many
    sweeps each tied label wins in proportion to the gap before it in cyclic
    label order (label 5 of {5, 300, 301} out of 1000: 704/1000; 300:
    295/1000; 301: 1/1000)."""
    freq, seen = _nonstrict_frequencies(mod)
    if not seen <= {5, 300, 301}:
        return False
    for lab, p in ((5, 0.704), (300, 0.295)):
        sd = (p * (1 - p) / 4000) ** 0.5
        if abs(freq[lab] - p) > 4 * sd:
            return False
    rng = np.random.default_rng(91)
    for g, C in _random_cases(60, seed0=90000):
        for i in range(g.n):
            sums = _label_sums(g, C, i)
            if not sums:
                continue
            m = max(sums.values())
            tied = [c for c, v in sums.items() if v == m]
            t = int(rng.integers(1, 30))
            c = mod.pick(g.off, g.idx, g.w, C, i, sweep=t)
            if c not in tied or (len(tied) == 1 and c != tied[0]):
                return False
    return True


def _flpa_pins_pass(mod):
    """FLPA pruning rule (Section 2).  Star K_{1,7}, ascending order, worked by
    hand: the centre takes label 1 (all of its labels tie at weight 1), leaf
    1 keeps 1, leaves 2..7 take 1: 7 changes, then none.  Every leaf change
    re-marks the centre under the plain rule (8 then 1 vertices scanned); under
    FLPA the centre already carries label 1 and is not re-marked (8 then 0).
    And on random graphs the rule equals the worklist restatement."""
    g = L.from_undirected_pairs(8, [(0, k) for k in range(1, 8)])
    for po, act in ((False, [8, 1]), (True, [8, 0])):
        C, it, ch, a = mod.lpa_async_ex(g.off, g.idx, None, 0.05, 20, prune_other=po)
        if C.tolist() != [1] * 8 or it != 2 or ch.tolist() != [7, 0] or a.tolist() != act:
            return False
    for g, _ in _random_cases(60, seed0=61000):
        if g.n == 0:
            continue
        C, it, h = _serial_async_restated(g, 0.05, 20, prune_other=True)
        Co, ito, ho, _ = mod.lpa_async_ex(g.off, g.idx, g.w, 0.05, 20, prune_other=True)
        if Co.tolist() != C.tolist() or ito != it or ho.tolist() != h:
            return False
    return True


def _tolerance_pins_pass(mod):
    """The tolerance test of Algorithm 1 (Section 4.1.3), dN / N <= tau,
    against exact rational arithmetic on the decimal tolerance as written
    (Fraction("0.05") is exactly 1/20): random N below 2^31 and dN on both
    sides of the threshold for the paper's 0.05 and the sweep's 0.1, 0.01,
    1e-5; the paper's 0.05 at N = 100,000,019 (0.05 N = 5,000,000.95: dN =
    5,000,000 stops, 5,000,001 does not -- the fp32 value of 0.05 would stop
    there); and the ends tau = 0 and tau = 1 (inclusive)."""
    from fractions import Fraction
    n = 100_000_019
    if not mod.converged(5_000_000, n, 0.05) or mod.converged(5_000_001, n, 0.05):
        return False
    if not mod.converged(0, 7, 0.0) or mod.converged(1, 7, 0.0) or not mod.converged(7, 7, 1.0):
        return False
    rng = np.random.default_rng(4)
    for text in ("0.05", "0.1", "0.01", "0.00001", "0.25", "0.3"):
        tau_q, tau = Fraction(text), float(text)
        for _ in range(500):
            N = int(rng.integers(1, 2**31 - 1))
            base = int(tau_q * N)                     # floor(tau N), exact
            for dN in (base - 1, base, base + 1):
                if 0 <= dN <= N and mod.converged(dN, N, tau) != (dN <= tau_q * N):
                    return False
    return True


def _pins_pass(mod):
    try:
        for case in _golden_cases():
            C, it, ch = _run_case(case, mod)
            if C.tolist() != case["labels"] or it != case["iterations"] or ch.tolist() != case["changed"]:
                return False
        for g, C in _random_cases(120, seed0=50000):
            Cn, _ = mod.sync_sweep(g.off, g.idx, g.w, C)
            if any(Cn[i] != _enumerated_pick(g, C, i) for i in range(g.n)):
                return False
        for g, _ in _random_cases(60, seed0=60000):
            if g.n == 0:
                continue
            C, it, h = _serial_async_restated(g, 0.05, 20)
            Co, ito, ho = mod.lpa_async(g.off, g.idx, g.w)
            if Co.tolist() != C.tolist() or ito != it:
                return False
        if not _nonstrict_pins_pass(mod):
            return False
        if not _flpa_pins_pass(mod):
            return False
        if not _checker_pins_pass(mod):
            return False
        if not _tolerance_pins_pass(mod):
            return False
        pairs = [(u, v) for u in range(5) for v in range(u + 1, 5)]
        pairs += [(u + 5, v + 5) for u, v in pairs] + [(4, 5)]
        g = L.from_undirected_pairs(10, pairs)
        if abs(mod.modularity(g.off, g.idx, None, np.array([0] * 5 + [5] * 5, np.int32)) - 19 / 42) > 1e-12:
            return False
        g = L.from_undirected_pairs(4, [(u, v) for u in range(4) for v in range(u + 1, 4)])
        if abs(mod.modularity(g.off, g.idx, None, np.arange(4, dtype=np.int32)) + 0.25) > 1e-12:
            return False
        return True
    except Exception:
        return False


def test_unmodified_oracle_passes_pin_battery():
    assert _pins_pass(O)


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_is_caught(name, tmp_path):
    src = open(os.path.join(ROOT, "oracle", "lpa_oracle.c")).read()
    old, new = MUTANTS[name]
    assert src.count(old) == 1, f"mutation anchor for {name} not found once"
    path = tmp_path / "mutant.c"
    path.write_text(src.replace(old, new))
    so = tmp_path / f"lib_{name}.so"
    subprocess.check_call(["gcc", "-O1", "-std=c11", "-fPIC", "-shared", "-o", str(so), str(path), "-lm"])
    assert not _pins_pass(O.load_variant(str(so)))


def test_async_order_ascending_equals_default_and_rejects_non_permutations():
    """The ordered serial run with the identity order is the ascending run;
    an order that is not a permutation of 0..n-1 is refused."""
    for g, _ in _random_cases(40, seed0=70000):
        if g.n == 0:
            continue
        a = O.lpa_async(g.off, g.idx, g.w)
        b = O.lpa_async(g.off, g.idx, g.w, order=np.arange(g.n))
        assert a[0].tolist() == b[0].tolist() and a[1] == b[1] and a[2].tolist() == b[2].tolist()
    g = L.from_undirected_pairs(3, [(0, 1), (1, 2)])
    for bad in ([0, 0, 1], [0, 1, 3], [2, 1, -1]):
        with pytest.raises(Exception):
            O.lpa_async(g.off, g.idx, None, order=bad)


def test_async_order_matches_restatement_in_that_order():
    """A second restatement of Algorithm 1 in Python, visiting a random order,
    agrees with the ordered oracle on random small graphs."""
    rng = np.random.default_rng(5)
    for g, _ in _random_cases(40, seed0=80000):
        if g.n == 0:
            continue
        order = rng.permutation(g.n)
        C, it, hist = _serial_async_restated(g, 0.05, 20, order=order)
        Co, ito, ho = O.lpa_async(g.off, g.idx, g.w, order=order)
        assert Co.tolist() == C.tolist() and ito == it and ho.tolist() == hist


def test_nonstrict_tie_break_pins():
    assert _nonstrict_pins_pass(O)
    freq, _ = _nonstrict_frequencies(O)
    print("non-strict tie frequencies", freq)
