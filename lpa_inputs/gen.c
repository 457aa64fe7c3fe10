/*
 * gen.c -- seeded synthetic graph generators shared by the tests, the
 * benchmark and the oracle runs.  Nothing here computes any part of label
 * propagation: it only draws edges and lays them out as symmetric CSR.
 *
 * Randomness is counter-based so that every output is independent of the
 * thread count: each draw is mix64 applied to (seed, stream, counter), where
 * mix64 is the SplitMix64 output function (Steele, Lea & Flood, "Fast
 * splittable pseudorandom number generators", OOPSLA 2014).
 *
 * Generators:
 *   gen_rmat_edges     R-MAT (Chakrabarti, Zhan & Faloutsos, SDM 2004),
 *                      no noise, no vertex permutation.
 *   gen_sbm_count/fill planted partition (stochastic block model) over
 *                      contiguous blocks, pairs u < v drawn with geometric
 *                      skipping (Batagelj & Brandes, Phys. Rev. E 71, 2005).
 *   gen_grid_count/fill 2-D 4-neighbour lattice with a kept fraction of its
 *                      edges plus random long-range shortcuts.
 *   csr_*              edge list -> symmetric CSR with rows sorted ascending,
 *                      optional de-duplication and self-loop removal, and
 *                      symmetric integer weights hashed from the vertex pair.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

static inline uint64_t mix64(uint64_t z) {
    z += 0x9e3779b97f4a7c15ULL;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

static inline uint64_t draw(uint64_t seed, uint64_t stream, uint64_t ctr) {
    return mix64(mix64(seed ^ mix64(stream)) + ctr * 0xd1342543de82ef95ULL);
}

/* uniform double in (0, 1] from the top 53 bits */
static inline double unit_open0(uint64_t r) {
    return ((double)(r >> 11) + 1.0) * (1.0 / 9007199254740992.0);
}

static inline uint64_t prob_threshold(double p) {
    if (p <= 0.0) return 0;
    if (p >= 1.0) return UINT64_MAX;
    return (uint64_t)(p * 18446744073709551616.0);
}

/* ---------------------------------------------------------------- R-MAT */
void gen_rmat_edges(int32_t scale, int64_t m, double a, double b, double c, uint64_t seed,
                    int32_t *src, int32_t *dst) {
    const uint64_t ta = prob_threshold(a), tab = prob_threshold(a + b),
                   tabc = prob_threshold(a + b + c);
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < m; ++e) {
        uint32_t u = 0, v = 0;
        for (int32_t l = 0; l < scale; ++l) {
            uint64_t r = draw(seed, 1, (uint64_t)e * 64u + (uint64_t)l);
            uint32_t bu, bv;
            if (r < ta) { bu = 0; bv = 0; }
            else if (r < tab) { bu = 0; bv = 1; }
            else if (r < tabc) { bu = 1; bv = 0; }
            else { bu = 1; bv = 1; }
            u = (u << 1) | bu;
            v = (v << 1) | bv;
        }
        src[e] = (int32_t)u;
        dst[e] = (int32_t)v;
    }
}

/* ------------------------------------------------------------------ SBM */
/* Vertex u draws its partners v > u.  Blocks are the contiguous ranges
 * [bstart[k], bstart[k+1]); a pair in one block is present with probability
 * p_in, a pair across blocks with p_out.  emit == NULL counts only. */
static int64_t sbm_row(int64_t u, int32_t nb, const int64_t *bstart, double p_in, double p_out,
                       uint64_t seed, int32_t *emit_dst) {
    int32_t bu = 0;
    while (bstart[bu + 1] <= u) ++bu;
    int64_t cnt = 0;
    uint64_t ctr = 0;
    for (int32_t k = bu; k < nb; ++k) {
        double p = (k == bu) ? p_in : p_out;
        int64_t lo = bstart[k], hi = bstart[k + 1];
        if (lo < u + 1) lo = u + 1;
        if (lo >= hi || p <= 0.0) continue;
        if (p >= 1.0) {
            for (int64_t v = lo; v < hi; ++v) {
                if (emit_dst) emit_dst[cnt] = (int32_t)v;
                ++cnt;
            }
            continue;
        }
        double lq = log1p(-p);
        int64_t v = lo - 1;
        for (;;) {
            double skip = floor(log(unit_open0(draw(seed, (uint64_t)u + 7, ctr++))) / lq);
            if (skip >= (double)(hi - v)) break;
            v += 1 + (int64_t)skip;
            if (v >= hi) break;
            if (emit_dst) emit_dst[cnt] = (int32_t)v;
            ++cnt;
        }
    }
    return cnt;
}

/* rowcnt[u] receives the number of partners v > u of vertex u. */
void gen_sbm_count(int64_t n, int32_t nb, const int64_t *bstart, double p_in, double p_out,
                   uint64_t seed, int64_t *rowcnt) {
#pragma omp parallel for schedule(dynamic, 1024)
    for (int64_t u = 0; u < n; ++u) rowcnt[u] = sbm_row(u, nb, bstart, p_in, p_out, seed, NULL);
}

/* rowstart: exclusive prefix of rowcnt; fills (src, dst) pairs u < v. */
void gen_sbm_fill(int64_t n, int32_t nb, const int64_t *bstart, double p_in, double p_out,
                  uint64_t seed, const int64_t *rowstart, int32_t *src, int32_t *dst) {
#pragma omp parallel for schedule(dynamic, 1024)
    for (int64_t u = 0; u < n; ++u) {
        int64_t s = rowstart[u];
        int64_t c = sbm_row(u, nb, bstart, p_in, p_out, seed, dst + s);
        for (int64_t k = 0; k < c; ++k) src[s + k] = (int32_t)u;
    }
}

/* ----------------------------------------------------------------- grid */
/* Lattice edge id e < rows*(cols-1) is horizontal (r, c)-(r, c+1) with
 * r = e / (cols-1); the rest are vertical (r, c)-(r+1, c). */
static inline void grid_edge(int64_t e, int64_t rows, int64_t cols, int64_t *u, int64_t *v) {
    int64_t nh = rows * (cols - 1);
    if (e < nh) {
        int64_t r = e / (cols - 1), c = e % (cols - 1);
        *u = r * cols + c;
        *v = *u + 1;
    } else {
        int64_t f = e - nh;
        int64_t r = f / cols, c = f % cols;
        *u = r * cols + c;
        *v = *u + cols;
    }
}

static inline int grid_keep(uint64_t seed, int64_t e, uint64_t keep_thr) {
    return draw(seed, 3, (uint64_t)e) < keep_thr;
}

int64_t gen_grid_count(int64_t rows, int64_t cols, double keep_p, uint64_t seed) {
    int64_t ne = rows * (cols - 1) + (rows - 1) * cols, kept = 0;
    uint64_t thr = prob_threshold(keep_p);
#pragma omp parallel for reduction(+ : kept) schedule(static)
    for (int64_t e = 0; e < ne; ++e) kept += grid_keep(seed, e, thr);
    return kept;
}

/* Writes the kept lattice edges followed by n_short shortcuts (u != v). */
void gen_grid_fill(int64_t rows, int64_t cols, double keep_p, uint64_t seed, int64_t n_short,
                   int32_t *src, int32_t *dst) {
    int64_t ne = rows * (cols - 1) + (rows - 1) * cols;
    uint64_t thr = prob_threshold(keep_p);
    int64_t out = 0;
    for (int64_t e = 0; e < ne; ++e) {       /* sequential: preserves edge order */
        if (!grid_keep(seed, e, thr)) continue;
        int64_t u, v;
        grid_edge(e, rows, cols, &u, &v);
        src[out] = (int32_t)u;
        dst[out] = (int32_t)v;
        ++out;
    }
    int64_t n = rows * cols;
    for (int64_t k = 0; k < n_short; ++k) {
        uint64_t r1 = draw(seed, 4, (uint64_t)k), r2 = draw(seed, 5, (uint64_t)k);
        int64_t u = (int64_t)(r1 % (uint64_t)n);
        int64_t v = (u + 1 + (int64_t)(r2 % (uint64_t)(n - 1))) % n;
        src[out + k] = (int32_t)u;
        dst[out + k] = (int32_t)v;
    }
}

/* ------------------------------------------------------------------ CSR */
/* deg[i] (zeroed by the caller, int64[n]) += entries row i receives. */
void csr_degrees(int64_t n, int64_t m, const int32_t *src, const int32_t *dst, int32_t symmetrise,
                 int32_t drop_self, int64_t *deg) {
    (void)n;
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < m; ++e) {
        int32_t u = src[e], v = dst[e];
        if (drop_self && u == v) continue;
        __atomic_fetch_add(&deg[u], 1, __ATOMIC_RELAXED);
        if (symmetrise) __atomic_fetch_add(&deg[v], 1, __ATOMIC_RELAXED);
    }
}

static int cmp_i32(const void *a, const void *b) {
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

/* Scatters the edges into idx using off (exclusive prefix of csr_degrees,
 * int64[n+1]) and sorts every row ascending.  cursor: scratch int64[n]. */
void csr_fill_sorted(int64_t n, int64_t m, const int32_t *src, const int32_t *dst, int32_t symmetrise,
                     int32_t drop_self, const int64_t *off, int64_t *cursor, int32_t *idx) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) cursor[i] = off[i];
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < m; ++e) {
        int32_t u = src[e], v = dst[e];
        if (drop_self && u == v) continue;
        idx[__atomic_fetch_add(&cursor[u], 1, __ATOMIC_RELAXED)] = v;
        if (symmetrise) idx[__atomic_fetch_add(&cursor[v], 1, __ATOMIC_RELAXED)] = u;
    }
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t i = 0; i < n; ++i)
        if (off[i + 1] - off[i] > 1) qsort(idx + off[i], (size_t)(off[i + 1] - off[i]), sizeof(int32_t), cmp_i32);
}

/* Removes repeated neighbours from each sorted row, in place.  off is
 * rewritten; returns the new entry count. */
int64_t csr_dedup(int64_t n, int64_t *off, int32_t *idx, int64_t *uniq) {
#pragma omp parallel for schedule(dynamic, 1024)
    for (int64_t i = 0; i < n; ++i) {
        int64_t c = 0;
        for (int64_t e = off[i]; e < off[i + 1]; ++e)
            if (e == off[i] || idx[e] != idx[e - 1]) ++c;
        uniq[i] = c;
    }
    int64_t out = 0;
    for (int64_t i = 0; i < n; ++i) {        /* sequential left shift: rows never overlap badly */
        int64_t s = off[i], t = off[i + 1];
        off[i] = out;
        for (int64_t e = s; e < t; ++e)
            if (e == s || idx[e] != idx[e - 1]) idx[out++] = idx[e];
    }
    off[n] = out;
    return out;
}

/* w[e] = 1 + h(min(i,j), max(i,j)) mod wmax: integer, symmetric in (i, j). */
void csr_pair_weights(int64_t n, const int64_t *off, const int32_t *idx, int32_t wmax, uint64_t seed,
                      float *w) {
#pragma omp parallel for schedule(dynamic, 1024)
    for (int64_t i = 0; i < n; ++i)
        for (int64_t e = off[i]; e < off[i + 1]; ++e) {
            uint64_t a = (uint64_t)(i < idx[e] ? i : idx[e]), b = (uint64_t)(i < idx[e] ? idx[e] : i);
            w[e] = (float)(1 + (int32_t)(draw(seed, 6, (a << 32) | b) % (uint64_t)wmax));
        }
}
