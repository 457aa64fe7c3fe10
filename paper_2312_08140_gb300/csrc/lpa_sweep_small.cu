// lpa_sweep_small.cu -- sweep for low-degree vertices (degree <= small_max <= 8):
// one thread per frontier vertex.  The thread loads its row's neighbour ids,
// weights and neighbour labels into registers and evaluates the update rule
// (Eq. 2, Section 3.3) by comparing every pair of entries: the sum for the
// label of entry q is the total weight of entries carrying the same label.
// Self-loops are skipped (scanCommunities, Algorithm 1); ties go to the
// smallest label id (Section 4.1.5).  When the label changes the thread marks
// all other neighbours unprocessed (vertex pruning, Section 4.1.4).
//
// Asynchronous mode: each thread takes a run of kAsyncRun consecutive
// frontier entries and processes them one after another, so a vertex reads the
// labels its predecessors in the run have just written -- the GPU counterpart
// of the paper's threads walking contiguous chunks of vertices (Section 4.1,
// 4.1.1).  One vertex per thread would make every thread of a sweep read the
// labels left by the previous sweep, which turns the sweep into a Jacobi
// update that oscillates on bipartite structure such as lattices.
//
// Memory per vertex: two offsets, d indices, d weights, d label gathers, one
// own-label load; on change one label write and d flag bytes.
#include "lpa_device.cuh"

namespace lpa {

constexpr int kSmallThreads = 256;
constexpr int kAsyncRun = 32;

template <bool ASYNC, int WK, bool BATCH, int MAXD>
__global__ void __launch_bounds__(kSmallThreads) k_sweep_small(DevState s, int flag_neighbours) {
    using T = typename Acc<WK>::T;
    const BinView bv = bin_view(s, 0);
    const Labels L = labels_of(s);
    const bool marks = marks_on(s, flag_neighbours);
    const unsigned cnt = bv.cnt;
    const unsigned stride = gridDim.x * blockDim.x;
    constexpr int RUN = ASYNC ? kAsyncRun : 1;
    const unsigned nruns = (cnt + RUN - 1) / RUN;
    unsigned long long my_changed = 0, my_changed_entries = 0;
    for (unsigned rbase = blockIdx.x * blockDim.x; rbase < nruns; rbase += stride)
    for (int step = 0; step < RUN; ++step) {
        const unsigned run = rbase + threadIdx.x;
        const unsigned k = run * RUN + step;
        const bool slot = run < nruns && k < cnt;
        bool act = slot;
        const int32_t v = slot ? bv.list[k] : 0;
        if constexpr (BATCH) {
            if (act && s.done[s.gid[v]]) act = false;
        }
        int64_t st = 0;
        int d = 0;
        int32_t own = 0;
        if (slot) own = ASYNC ? __ldcg(L.C + v) : L.C[v];
        if (act) {
            st = s.off[v];
            d = (int)(s.off[v + 1] - st);
        }
        int32_t nb[MAXD];
        int32_t lab[MAXD];
        T wt[MAXD];
#pragma unroll
        for (int q = 0; q < MAXD; ++q) {
            bool ok = q < d;
            const int32_t j = ok ? load_index(s.idx, st + q) : v;
            nb[q] = j;
            ok = ok && (j != v);
            lab[q] = ok ? load_label<ASYNC>(L.C, j) : kEmptyKey;
            wt[q] = ok ? load_weight<WK>(s.w, st + q) : (T)0;
        }
        bool any = false;
        T best_w = 0;
        int32_t best = 0x7fffffff;
#pragma unroll
        for (int q = 0; q < MAXD; ++q) {
            T sum = 0;
#pragma unroll
            for (int r = 0; r < MAXD; ++r) sum += (lab[r] == lab[q]) ? wt[r] : (T)0;
            const bool better = lab[q] != kEmptyKey &&
                                (!any || sum > best_w || (sum == best_w && lab[q] < best));
            if (better) {
                any = true;
                best_w = sum;
                best = lab[q];
            }
        }
        const bool changed = act && any && best != own;
        if (slot) record_label<ASYNC>(L, bv.chg + k, v, own, best, changed);
        if (changed) {
            if (marks) {
#pragma unroll
                for (int q = 0; q < MAXD; ++q)
                    if (q < d && nb[q] != v) s.flags[nb[q]] = 1;
            }
            ++my_changed;
            my_changed_entries += (unsigned)d;
        }
        count_graph_changes<BATCH>(s, changed, v);
    }
    flush_bin_counts(s, 0, my_changed, my_changed_entries);
}

cudaError_t launch_sweep_small(const DevState& s, int mode, cudaStream_t st, int sms) {
    const bool async = mode == MODE_ASYNC;
    const int flag = mode != MODE_SYNC_FULL;
    const bool batch = s.G > 1;
    const bool four = s.small_max <= 4;
    dim3 grid(sms * 8), block(kSmallThreads);
#define LPA_SMALL(A, W, B)                                                          \
    do {                                                                            \
        if (four) k_sweep_small<A, W, B, 4><<<grid, block, 0, st>>>(s, flag);       \
        else k_sweep_small<A, W, B, 8><<<grid, block, 0, st>>>(s, flag);            \
    } while (0)
#define LPA_SMALL_W(A, B)                                      \
    switch (s.weight_kind) {                                   \
        case W_UNIT: LPA_SMALL(A, W_UNIT, B); break;           \
        case W_U32: LPA_SMALL(A, W_U32, B); break;             \
        default: LPA_SMALL(A, W_F32, B); break;                \
    }
    if (async) {
        if (batch) { LPA_SMALL_W(true, true) } else { LPA_SMALL_W(true, false) }
    } else {
        if (batch) { LPA_SMALL_W(false, true) } else { LPA_SMALL_W(false, false) }
    }
#undef LPA_SMALL_W
#undef LPA_SMALL
    return cudaGetLastError();
}

}  // namespace lpa
