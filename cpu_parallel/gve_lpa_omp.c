/*
 * gve_lpa_omp.c -- multi-core CPU label propagation in the paper's own design
 * (Section 4.1), run on the host cores as a comparison point for the GPU
 * library.  Not test infrastructure and not used by the GPU path.
 *
 * Design choices taken from the paper:
 *   - threads take chunks of 2048 consecutive vertices from an OpenMP dynamic
 *     schedule (Section 4.1.1);
 *   - each thread owns a collision-free table: a list of the labels seen for
 *     the current vertex plus a |V|-sized array of their summed weights,
 *     allocated separately per thread (Section 4.1.6);
 *   - 8-bit flags mark unprocessed vertices; a vertex is marked processed
 *     when visited and, when its label changes, its neighbours other than
 *     itself are marked unprocessed (vertex pruning, Section 4.1.4);
 *   - the changed count of a sweep is a reduction, and a run stops when
 *     dN/N <= tau or after max_iters sweeps (Sections 4.1.2, 4.1.3);
 *   - strict tie-break: the smallest label among the most weighted (Section
 *     4.1.5 with the reading of Section 2).
 * Asynchronous mode updates labels in place while other threads read them
 * (Algorithm 1); the synchronous mode reads the previous sweep's labels and
 * writes a second buffer (a Jacobi reading; with the strict tie-break pruning
 * does not change its result).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <omp.h>

#define CHUNK 2048

typedef struct {
    int32_t *keys;
    double *val;
    uint8_t *seen;      /* label already listed in keys (a zero weight leaves val at 0) */
    int64_t nkeys;
} table_t;

static int32_t pick(table_t *T, const int64_t *off, const int32_t *idx, const float *w, const int32_t *C,
                    int64_t i) {
    T->nkeys = 0;
    for (int64_t e = off[i]; e < off[i + 1]; ++e) {
        const int32_t j = idx[e];
        if ((int64_t)j == i) continue;
        const int32_t c = C[j];
        if (!T->seen[c]) {
            T->seen[c] = 1;
            T->keys[T->nkeys++] = c;
        }
        T->val[c] += w ? (double)w[e] : 1.0;
    }
    if (T->nkeys == 0) return C[i];
    int32_t best = -1;
    double best_w = 0.0;
    for (int64_t k = 0; k < T->nkeys; ++k) {
        const int32_t c = T->keys[k];
        const double v = T->val[c];
        if (best < 0 || v > best_w || (v == best_w && c < best)) {
            best = c;
            best_w = v;
        }
        T->val[c] = 0.0;
        T->seen[c] = 0;
    }
    return best;
}

/* mode 0: synchronous, 1: asynchronous.  Returns the number of sweeps, or a
 * negative value on allocation failure.  threads <= 0: the OpenMP default. */
int64_t cpu_lpa_run(int64_t n, const int64_t *off, const int32_t *idx, const float *w, int mode, double tau,
                    int64_t max_iters, int threads, int32_t *C, int64_t *changed_hist) {
    if (threads > 0) omp_set_num_threads(threads);
    const int nt = omp_get_max_threads();
    uint8_t *flag = (uint8_t *)malloc((size_t)(n > 0 ? n : 1));
    /* synchronous mode: marks of sweep t go to a second array read in t+1, and
     * labels to a second buffer */
    uint8_t *flag_next = mode == 0 ? (uint8_t *)calloc((size_t)(n > 0 ? n : 1), 1) : NULL;
    int32_t *Cn = mode == 0 ? (int32_t *)malloc((size_t)(n > 0 ? n : 1) * 4) : NULL;
    table_t *T = (table_t *)calloc((size_t)nt, sizeof(table_t));
    if (!flag || (mode == 0 && (!Cn || !flag_next)) || !T) {
        free(flag); free(flag_next); free(Cn); free(T);
        return -1;
    }
    int fail = 0;
#pragma omp parallel num_threads(nt)
    {
        const int t = omp_get_thread_num();
        T[t].keys = (int32_t *)malloc((size_t)(n > 0 ? n : 1) * 4);
        T[t].val = (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
        T[t].seen = (uint8_t *)calloc((size_t)(n > 0 ? n : 1), 1);
        if (!T[t].keys || !T[t].val || !T[t].seen) {
#pragma omp atomic write
            fail = 1;
        }
#pragma omp for schedule(static)
        for (int64_t i = 0; i < n; ++i) {
            C[i] = (int32_t)i;
            flag[i] = 1;
            if (Cn) Cn[i] = (int32_t)i;
        }
    }
    int64_t it = 0;
    if (!fail && n > 0) {
        while (it < max_iters) {
            int64_t dN = 0;
#pragma omp parallel num_threads(nt) reduction(+ : dN)
            {
                table_t *Tt = &T[omp_get_thread_num()];
#pragma omp for schedule(dynamic, CHUNK)
                for (int64_t i = 0; i < n; ++i) {
                    if (!flag[i]) continue;
                    flag[i] = 0;
                    if (mode == 1) {
                        const int32_t c = pick(Tt, off, idx, w, C, i);
                        if (c == C[i]) continue;
                        C[i] = c;
                    } else {
                        const int32_t c = pick(Tt, off, idx, w, C, i);
                        Cn[i] = c;
                        if (c == C[i]) continue;
                    }
                    ++dN;
                    uint8_t *mark = mode == 0 ? flag_next : flag;
                    for (int64_t e = off[i]; e < off[i + 1]; ++e)
                        if ((int64_t)idx[e] != i) mark[idx[e]] = 1;
                }
            }
            if (mode == 0) {
                /* unscanned vertices kept their label, which Cn still holds */
#pragma omp parallel for num_threads(nt) schedule(static)
                for (int64_t i = 0; i < n; ++i) C[i] = Cn[i];
                uint8_t *tmp = flag;                  /* every flag of `flag` was cleared */
                flag = flag_next;
                flag_next = tmp;
            }
            if (changed_hist) changed_hist[it] = dN;
            ++it;
            if ((double)dN <= floor(tau * (double)n)) break;    /* dN <= floor(tau N), product in fp64 */
        }
    }
    for (int t = 0; t < nt; ++t) {
        free(T[t].keys);
        free(T[t].val);
        free(T[t].seen);
    }
    free(T);
    free(flag);
    free(flag_next);
    free(Cn);
    return fail ? -1 : it;
}

int cpu_lpa_threads(void) { return omp_get_max_threads(); }
