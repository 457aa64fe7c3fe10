/*
 * lpa_oracle.c -- plain, slow, single-threaded CPU oracle for GVE-LPA
 * (Sahu, "GVE-LPA: Fast Label Propagation Algorithm (LPA) for Community
 * Detection in Shared Memory Setting", arXiv 2312.08140).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this file.  The product path
 * (the CUDA library) never calls it and shares no code with it.
 *
 * What it computes, in the paper's order and notation:
 *   - oracle_pick:       the label update rule (Eq. 2, Section 3.3): the
 *                        label c maximising K_{i->c}, the summed weight of
 *                        i's neighbours j != i with C_j = c, as the
 *                        scanCommunities step of Algorithm 1 accumulates it
 *                        (self-loops skipped).  Ties go to the smallest label
 *                        id (strict LPA, Section 4.1.5 and Section 2).
 *                        A vertex with no neighbour other than itself keeps
 *                        its label.  Sums are taken in fp64 in CSR order.
 *   - oracle_lpa_sync:   a synchronous (Jacobi) reading of Algorithm 1: every
 *                        vertex of sweep t reads the labels of sweep t-1; no
 *                        pruning.  Stops after the sweep whose changed count
 *                        satisfies dN/N <= tau, or after max_iters sweeps
 *                        (Section 4.1.2, 4.1.3).
 *   - oracle_lpa_async:  Algorithm 1 run by one thread in ascending vertex
 *                        order (oracle_lpa_async_order: in a given order of
 *                        the vertex loop): labels updated in place, a vertex is marked
 *                        processed when visited and, when its label changes,
 *                        all of its neighbours other than itself are marked
 *                        unprocessed (vertex pruning, Section 4.1.4).
 *   - oracle_lpa_async_ex: the same with options: the non-strict tie-break;
 *                        the pruning rule of FLPA (Section 2), under which a
 *                        vertex whose label changes to c marks unprocessed
 *                        only the neighbours whose label is not c; and the
 *                        number of vertices scanned in each sweep.
 *   - *_nonstrict:       the same with the non-strict tie-break (Section
 *                        4.1.5: a pseudo-random choice among the tied
 *                        labels through a modulo of the label id), read as: in
 *                        sweep t, vertex i draws r = SplitMix64((t << 32) | i)
 *                        mod n and takes the most weighted label c minimising
 *                        (c - r) mod n.
 *   - oracle_modularity: Eq. 1 (Section 3.2) in its community form, all sums
 *                        in fp64.
 *   - checkers used by the tests on any output (labels inside the vertex's
 *     connected component; count of vertices not at a local maximum).
 *
 * The per-vertex accumulator is the paper's collision-free table
 * (Section 4.1.6): a list of touched keys plus a value array of size |V|
 * indexed by label, reset through the key list after each vertex.
 *
 * Every function returns a negative value on invalid input and never aborts.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_BAD_ARG (-1)
#define ORACLE_NO_MEM  (-2)

/* Collision-free accumulator of Section 4.1.6: keys[] lists the labels seen
 * for the current vertex, val[] (size n) holds their summed weights and
 * seen[] (size n) marks whether a label is already in keys[]. */
typedef struct {
    int64_t  n;
    int32_t *keys;
    int64_t  nkeys;
    double  *val;
    uint8_t *seen;
} kv_table;

static int kv_init(kv_table *t, int64_t n) {
    t->n = n;
    t->nkeys = 0;
    t->keys = (int32_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
    t->val = (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
    t->seen = (uint8_t *)calloc((size_t)(n > 0 ? n : 1), 1);
    if (!t->keys || !t->val || !t->seen) {
        free(t->keys); free(t->val); free(t->seen);
        return ORACLE_NO_MEM;
    }
    return 0;
}

static void kv_free(kv_table *t) {
    free(t->keys); free(t->val); free(t->seen);
}

static void kv_add(kv_table *t, int32_t key, double w) {
    if (!t->seen[key]) {
        t->seen[key] = 1;
        t->keys[t->nkeys++] = key;
    }
    t->val[key] += w;
}

static void kv_clear(kv_table *t) {
    for (int64_t k = 0; k < t->nkeys; ++k) {
        t->val[t->keys[k]] = 0.0;
        t->seen[t->keys[k]] = 0;
    }
    t->nkeys = 0;
}

static double edge_weight(const float *w, int64_t e) {
    return w ? (double)w[e] : 1.0;
}

/* scanCommunities of Algorithm 1: for every CSR entry (j, w) of row i with
 * j != i, H[C[j]] += w.  Returns the number of entries accumulated. */
static int64_t scan_communities(kv_table *H, const int64_t *off, const int32_t *idx,
                                const float *w, const int32_t *C, int64_t i) {
    int64_t used = 0;
    for (int64_t e = off[i]; e < off[i + 1]; ++e) {
        int32_t j = idx[e];
        if ((int64_t)j == i) continue;            /* self-loops are skipped */
        kv_add(H, C[j], edge_weight(w, e));
        ++used;
    }
    return used;
}

/* The most weighted label in H (Eq. 2); ties go to the smallest label id. */
static int32_t most_weighted_label(const kv_table *H) {
    int32_t best = -1;
    double best_w = 0.0;
    for (int64_t k = 0; k < H->nkeys; ++k) {
        int32_t c = H->keys[k];
        double v = H->val[c];
        if (best < 0 || v > best_w || (v == best_w && c < best)) {
            best = c;
            best_w = v;
        }
    }
    return best;
}

/* SplitMix64 (Steele, Lea & Flood, OOPSLA 2014; the generator's output
 * function applied to state x): the counter-based draw of the non-strict
 * tie-break. */
static uint64_t splitmix64(uint64_t x) {
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* Non-strict LPA (Section 4.1.5) picks one of the most weighted labels at
 * random with a modulo on the label id.  Read here as: for vertex i in sweep t
 * (1-based), draw r = SplitMix64((t << 32) | i) mod n and take, among the
 * most weighted labels, the first one at or after r in cyclic label order,
 * i.e. the one minimising (c - r) mod n. */
static int32_t most_weighted_label_rotated(const kv_table *H, int64_t n, uint64_t r) {
    int32_t best = -1;
    double best_w = 0.0;
    int64_t best_key = 0;
    for (int64_t k = 0; k < H->nkeys; ++k) {
        int32_t c = H->keys[k];
        double v = H->val[c];
        int64_t key = ((int64_t)c - (int64_t)r) % n;
        if (key < 0) key += n;
        if (best < 0 || v > best_w || (v == best_w && key < best_key)) {
            best = c;
            best_w = v;
            best_key = key;
        }
    }
    return best;
}

/* Pick for vertex i; sweep t >= 1 selects the non-strict tie-break, t == 0
 * the strict one. */
static int32_t pick_t(kv_table *H, int64_t n, const int64_t *off, const int32_t *idx, const float *w,
                      const int32_t *C, int64_t i, int64_t t) {
    int64_t used = scan_communities(H, off, idx, w, C, i);
    int32_t c = C[i];
    if (used) {
        if (t > 0) {
            const uint64_t r = splitmix64(((uint64_t)t << 32) | (uint64_t)i) % (uint64_t)n;
            c = most_weighted_label_rotated(H, n, r);
        } else {
            c = most_weighted_label(H);
        }
    }
    kv_clear(H);
    return c;
}

static int32_t pick(kv_table *H, const int64_t *off, const int32_t *idx, const float *w,
                    const int32_t *C, int64_t i) {
    return pick_t(H, 0, off, idx, w, C, i, 0);
}

static int check_csr(int64_t n, const int64_t *off, const int32_t *idx) {
    if (n < 0 || !off) return ORACLE_BAD_ARG;
    if (off[0] != 0) return ORACLE_BAD_ARG;
    for (int64_t i = 0; i < n; ++i)
        if (off[i + 1] < off[i]) return ORACLE_BAD_ARG;
    if (off[n] > 0 && !idx) return ORACLE_BAD_ARG;
    for (int64_t e = 0; e < off[n]; ++e)
        if (idx[e] < 0 || (int64_t)idx[e] >= n) return ORACLE_BAD_ARG;
    return 0;
}

/* Convergence test of Algorithm 1: dN / N <= tau, read as the integer test
 * dN <= floor(tau * N) with the product tau * N rounded once to fp64.  For
 * the tolerances one writes as decimals (0.05, 0.1, 1e-5 ...) and N < 2^31
 * this threshold is floor of the exact decimal tau times N: the fp64 error
 * of tau * N (a few 1e-9 at most) never crosses an integer that the exact
 * product does not reach.  A threshold is one integer per graph, so every
 * implementation that forms it the same way stops after the same sweep. */
static int converged(int64_t dN, int64_t n, double tau) {
    const double thr = floor(tau * (double)n);
    return (double)dN <= thr;
}

/* The tolerance test above as an entry point (1: dN / N <= tau). */
int64_t oracle_converged(int64_t dN, int64_t n, double tau) {
    if (dN < 0 || n < 0 || !(tau >= 0.0)) return ORACLE_BAD_ARG;
    return converged(dN, n, tau);
}

/* One label for vertex i given labels C (Eq. 2 with the strict tie-break). */
int32_t oracle_pick(int64_t n, const int64_t *off, const int32_t *idx, const float *w,
                    const int32_t *C, int64_t i) {
    if (check_csr(n, off, idx) || i < 0 || i >= n || !C) return ORACLE_BAD_ARG;
    kv_table H;
    if (kv_init(&H, n)) return ORACLE_NO_MEM;
    int32_t c = pick(&H, off, idx, w, C, i);
    kv_free(&H);
    return c;
}

/* One synchronous sweep: C_out[i] = pick(i, C_in) for every i.  Returns dN,
 * the number of vertices whose label changed. */
int64_t oracle_sync_sweep(int64_t n, const int64_t *off, const int32_t *idx, const float *w,
                          const int32_t *C_in, int32_t *C_out) {
    if (check_csr(n, off, idx) || !C_in || !C_out) return ORACLE_BAD_ARG;
    kv_table H;
    if (kv_init(&H, n)) return ORACLE_NO_MEM;
    int64_t dN = 0;
    for (int64_t i = 0; i < n; ++i) {
        C_out[i] = pick(&H, off, idx, w, C_in, i);
        dN += (C_out[i] != C_in[i]);
    }
    kv_free(&H);
    return dN;
}

/* Synchronous LPA.  C_out: int32[n]; changed_hist (nullable): int64[max_iters]
 * receives dN of each sweep.  Returns the number of sweeps performed. */
static int64_t lpa_sync_impl(int64_t n, const int64_t *off, const int32_t *idx, const float *w,
                             double tau, int64_t max_iters, int nonstrict, int32_t *C_out,
                             int64_t *changed_hist) {
    if (check_csr(n, off, idx) || !C_out || max_iters < 0 || !(tau >= 0.0)) return ORACLE_BAD_ARG;
    for (int64_t i = 0; i < n; ++i) C_out[i] = (int32_t)i;          /* C <- [0 .. |V|) */
    if (n == 0) return 0;
    int32_t *prev = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    if (!prev) return ORACLE_NO_MEM;
    kv_table H;
    if (kv_init(&H, n)) { free(prev); return ORACLE_NO_MEM; }
    int64_t it = 0;
    while (it < max_iters) {
        memcpy(prev, C_out, (size_t)n * sizeof(int32_t));
        int64_t dN = 0;
        for (int64_t i = 0; i < n; ++i) {
            C_out[i] = pick_t(&H, n, off, idx, w, prev, i, nonstrict ? it + 1 : 0);
            dN += (C_out[i] != prev[i]);
        }
        if (changed_hist) changed_hist[it] = dN;
        ++it;
        if (converged(dN, n, tau)) break;
    }
    kv_free(&H);
    free(prev);
    return it;
}

/* Synchronous LPA, strict tie-break. */
int64_t oracle_lpa_sync(int64_t n, const int64_t *off, const int32_t *idx, const float *w,
                        double tau, int64_t max_iters, int32_t *C_out, int64_t *changed_hist) {
    return lpa_sync_impl(n, off, idx, w, tau, max_iters, 0, C_out, changed_hist);
}

/* Synchronous LPA with the non-strict tie-break (sweeps t = 1, 2, ...). */
int64_t oracle_lpa_sync_nonstrict(int64_t n, const int64_t *off, const int32_t *idx, const float *w,
                                  double tau, int64_t max_iters, int32_t *C_out, int64_t *changed_hist) {
    return lpa_sync_impl(n, off, idx, w, tau, max_iters, 1, C_out, changed_hist);
}

/* Algorithm 1 (lpa / lpaMove / scanCommunities) run by a single thread that
 * visits the vertices in the order given by `order` (a permutation of
 * 0..n-1; NULL: ascending) in every sweep.  Algorithm 1 leaves the order of
 * its vertex loop open; any order is one of its executions.  nonstrict: the
 * non-strict tie-break of sweep it + 1.  Returns the number of sweeps. */
static int64_t lpa_async_impl(int64_t n, const int64_t *off, const int32_t *idx, const float *w,
                              double tau, int64_t max_iters, const int64_t *order, int nonstrict,
                              int prune_other, int32_t *C_out, int64_t *changed_hist, int64_t *active_hist) {
    if (check_csr(n, off, idx) || !C_out || max_iters < 0 || !(tau >= 0.0)) return ORACLE_BAD_ARG;
    if (order) {                                                     /* must be a permutation */
        uint8_t *hit = (uint8_t *)calloc((size_t)(n > 0 ? n : 1), 1);
        if (!hit) return ORACLE_NO_MEM;
        for (int64_t k = 0; k < n; ++k) {
            if (order[k] < 0 || order[k] >= n || hit[order[k]]) { free(hit); return ORACLE_BAD_ARG; }
            hit[order[k]] = 1;
        }
        free(hit);
    }
    for (int64_t i = 0; i < n; ++i) C_out[i] = (int32_t)i;          /* C <- [0 .. |V|) */
    if (n == 0) return 0;
    uint8_t *unprocessed = (uint8_t *)malloc((size_t)n);
    if (!unprocessed) return ORACLE_NO_MEM;
    memset(unprocessed, 1, (size_t)n);                               /* all unprocessed */
    kv_table H;
    if (kv_init(&H, n)) { free(unprocessed); return ORACLE_NO_MEM; }
    int64_t it = 0;
    while (it < max_iters) {
        int64_t dN = 0, active = 0;                                  /* lpaMove */
        for (int64_t k = 0; k < n; ++k) {
            const int64_t i = order ? order[k] : k;
            if (!unprocessed[i]) continue;
            unprocessed[i] = 0;                                      /* prune */
            ++active;
            int32_t c = pick_t(&H, n, off, idx, w, C_out, i, nonstrict ? it + 1 : 0);
            if (c == C_out[i]) continue;
            C_out[i] = c;
            ++dN;
            for (int64_t e = off[i]; e < off[i + 1]; ++e) {          /* re-mark neighbours */
                const int32_t j = idx[e];
                if ((int64_t)j == i) continue;
                if (prune_other && C_out[j] == c) continue;          /* FLPA: already in c */
                unprocessed[j] = 1;
            }
        }
        if (changed_hist) changed_hist[it] = dN;
        if (active_hist) active_hist[it] = active;
        ++it;
        if (converged(dN, n, tau)) break;
    }
    kv_free(&H);
    free(unprocessed);
    return it;
}

/* Eq. 2 for vertex i with the non-strict tie-break of sweep t (t >= 1). */
int32_t oracle_pick_nonstrict(int64_t n, const int64_t *off, const int32_t *idx, const float *w,
                              const int32_t *C, int64_t i, int64_t t) {
    if (check_csr(n, off, idx) || i < 0 || i >= n || !C || t < 1) return ORACLE_BAD_ARG;
    kv_table H;
    if (kv_init(&H, n)) return ORACLE_NO_MEM;
    int32_t c = pick_t(&H, n, off, idx, w, C, i, t);
    kv_free(&H);
    return c;
}

/* Algorithm 1 by one thread in the given vertex order, strict tie-break. */
int64_t oracle_lpa_async_order(int64_t n, const int64_t *off, const int32_t *idx, const float *w,
                               double tau, int64_t max_iters, const int64_t *order, int32_t *C_out,
                               int64_t *changed_hist) {
    return lpa_async_impl(n, off, idx, w, tau, max_iters, order, 0, 0, C_out, changed_hist, NULL);
}

/* Algorithm 1 by one thread in the given vertex order (NULL: ascending) with
 * the non-strict tie-break. */
int64_t oracle_lpa_async_nonstrict(int64_t n, const int64_t *off, const int32_t *idx, const float *w,
                                   double tau, int64_t max_iters, const int64_t *order, int32_t *C_out,
                                   int64_t *changed_hist) {
    return lpa_async_impl(n, off, idx, w, tau, max_iters, order, 1, 0, C_out, changed_hist, NULL);
}

/* Algorithm 1 by one thread in the given vertex order (NULL: ascending),
 * with the non-strict tie-break if `nonstrict`, the FLPA pruning rule if
 * `prune_other`, and the vertices scanned per sweep in active_hist (NULL:
 * not recorded). */
int64_t oracle_lpa_async_ex(int64_t n, const int64_t *off, const int32_t *idx, const float *w, double tau,
                            int64_t max_iters, const int64_t *order, int nonstrict, int prune_other,
                            int32_t *C_out, int64_t *changed_hist, int64_t *active_hist) {
    return lpa_async_impl(n, off, idx, w, tau, max_iters, order, nonstrict, prune_other, C_out, changed_hist,
                          active_hist);
}

/* Algorithm 1 by one thread in ascending vertex order. */
int64_t oracle_lpa_async(int64_t n, const int64_t *off, const int32_t *idx, const float *w,
                         double tau, int64_t max_iters, int32_t *C_out, int64_t *changed_hist) {
    return oracle_lpa_async_order(n, off, idx, w, tau, max_iters, NULL, C_out, changed_hist);
}

/* Modularity, Eq. 1 in community form: Q = sum_c [sigma_c/2m - (Sigma_c/2m)^2]
 * with 2m = sum of all stored entries' weights, sigma_c = weight of entries
 * (i,j) with C_i = C_j = c and Sigma_c = sum of K_i over i in c.
 * Returns 0 when the graph has no weight (2m == 0).  *q_out receives Q. */
int oracle_modularity(int64_t n, const int64_t *off, const int32_t *idx, const float *w,
                      const int32_t *C, double *q_out) {
    if (check_csr(n, off, idx) || !C || !q_out) return ORACLE_BAD_ARG;
    for (int64_t i = 0; i < n; ++i)
        if (C[i] < 0 || (int64_t)C[i] >= n) return ORACLE_BAD_ARG;
    double two_m = 0.0, sigma = 0.0;
    double *Sigma = (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
    if (!Sigma) return ORACLE_NO_MEM;
    for (int64_t i = 0; i < n; ++i) {
        double K_i = 0.0;
        for (int64_t e = off[i]; e < off[i + 1]; ++e) {
            double wij = edge_weight(w, e);
            K_i += wij;
            if (C[idx[e]] == C[i]) sigma += wij;
        }
        two_m += K_i;
        Sigma[C[i]] += K_i;
    }
    double q = 0.0;
    if (two_m > 0.0) {
        double null_term = 0.0;
        for (int64_t c = 0; c < n; ++c) null_term += (Sigma[c] / two_m) * (Sigma[c] / two_m);
        q = sigma / two_m - null_term;
    }
    free(Sigma);
    *q_out = q;
    return 0;
}

/* ---- checkers (properties any correct output has) ---------------------- */

static int64_t uf_find(int64_t *parent, int64_t x) {
    while (parent[x] != x) {
        parent[x] = parent[parent[x]];
        x = parent[x];
    }
    return x;
}

/* Number of vertices i whose label C[i] is not a vertex of i's connected
 * component (labels only travel along edges, so a correct run returns 0).
 * Also fails labels outside [0, n). */
int64_t oracle_count_labels_outside_component(int64_t n, const int64_t *off, const int32_t *idx,
                                              const int32_t *C) {
    if (check_csr(n, off, idx) || !C) return ORACLE_BAD_ARG;
    int64_t *parent = (int64_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
    if (!parent) return ORACLE_NO_MEM;
    for (int64_t i = 0; i < n; ++i) parent[i] = i;
    for (int64_t i = 0; i < n; ++i)
        for (int64_t e = off[i]; e < off[i + 1]; ++e) {
            int64_t a = uf_find(parent, i), b = uf_find(parent, idx[e]);
            if (a != b) parent[a < b ? b : a] = (a < b ? a : b);
        }
    int64_t bad = 0;
    for (int64_t i = 0; i < n; ++i) {
        if (C[i] < 0 || (int64_t)C[i] >= n) { ++bad; continue; }
        if (uf_find(parent, i) != uf_find(parent, C[i])) ++bad;
    }
    free(parent);
    return bad;
}

/* Number of vertices not at a local maximum: K_{i->C_i} < max_c K_{i->c}
 * (tie-insensitive).  Vertices with no neighbour other than themselves count
 * as at a maximum. */
int64_t oracle_count_not_local_max(int64_t n, const int64_t *off, const int32_t *idx,
                                   const float *w, const int32_t *C) {
    if (check_csr(n, off, idx) || !C) return ORACLE_BAD_ARG;
    kv_table H;
    if (kv_init(&H, n)) return ORACLE_NO_MEM;
    int64_t bad = 0;
    for (int64_t i = 0; i < n; ++i) {
        if (C[i] < 0 || (int64_t)C[i] >= n) { ++bad; continue; }
        int64_t used = scan_communities(&H, off, idx, w, C, i);
        if (used) {
            int32_t best = most_weighted_label(&H);
            double own = H.seen[C[i]] ? H.val[C[i]] : 0.0;
            if (own < H.val[best]) ++bad;
        }
        kv_clear(&H);
    }
    kv_free(&H);
    return bad;
}
