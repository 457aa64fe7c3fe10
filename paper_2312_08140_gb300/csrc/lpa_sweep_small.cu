// lpa_sweep_small.cu -- sweep for low-degree vertices (degree <= small_max <= 8):
// one thread per frontier vertex.  The thread loads its row's neighbour ids,
// weights and neighbour labels into registers and evaluates the update rule
// (Eq. 2, Section 3.3) by comparing every pair of entries: the sum for the
// label of entry q is the total weight of entries carrying the same label.
// Self-loops are skipped (scanCommunities, Algorithm 1); ties go to the
// smallest label id (Section 4.1.5).  When the label changes the thread marks
// all other neighbours unprocessed (vertex pruning, Section 4.1.4).  One
// resident wave of threads walks the frontier, each thread as a three-stage
// software pipeline (offsets and own label -> row -> neighbour labels) over
// its slots, so the loads of three consecutive slots overlap.
//
// Asynchronous mode (k_sweep_small_async): each thread takes a run of kRun
// consecutive frontier entries and processes them one after another, so a
// vertex reads the labels its predecessors in the run have just written --
// the GPU counterpart of the paper's threads walking contiguous chunks of
// vertices (Sections 4.1, 4.1.1).  One vertex per thread would make every
// thread of a sweep read the labels left by the previous sweep, which turns
// the sweep into a Jacobi update that oscillates on bipartite structure such
// as lattices.  Walking runs straight from global memory scatters each warp's
// loads over 32 rows and re-reads the CSR from DRAM many times over, so the
// block first stages a tile of kRun x 256 rows (frontier id, row length,
// indices, weights) into shared memory with loads in which the lanes of a
// warp read consecutive rows, then each thread walks its run out of shared
// memory (run stride kRun + 1 words: conflict-free banks).  Neighbour labels
// are still read from global memory at processing time, so updates made
// during the sweep are seen.
//
// Memory per vertex: two offsets, d indices, d weights, d label gathers, one
// own-label load; on change one label write and d flag bytes.
#include "lpa_device.cuh"

namespace lpa {

constexpr int kSmallThreads = 256;
constexpr int kRun = 8;                               // async run length
constexpr int kTile = kRun * kSmallThreads;           // frontier entries staged per block step
constexpr int kStride = kRun + 1;                     // shared-memory words per run

// Eq. 2 over the at most MAXD entries of one row held in registers: the sum
// of each entry's label (empty entries hold kEmptyKey and weight 0), then the
// largest sum, then the smallest tie key among the entries that hold it.
// Integer sums are exact in any order, so each pair of entries is compared
// once and adds both ways; fp32 sums keep ascending entry order.  Returns the
// winning label, or -1 when the row has no candidate.
template <int WK, int MAXD>
__device__ __forceinline__ int32_t small_argmax(const int32_t (&lab)[MAXD], const typename Acc<WK>::T (&wt)[MAXD],
                                                const TieRule& tr) {
    using T = typename Acc<WK>::T;
    uint32_t sk[MAXD];
    if constexpr (WK == W_F32) {
#pragma unroll
        for (int q = 0; q < MAXD; ++q) {
            T sum = 0;
#pragma unroll
            for (int r = 0; r < MAXD; ++r) sum += (lab[r] == lab[q]) ? wt[r] : (T)0;
            sk[q] = lab[q] != kEmptyKey ? sum_key(sum) : 0u;
        }
    } else {
        T sum[MAXD];
#pragma unroll
        for (int q = 0; q < MAXD; ++q) sum[q] = wt[q];
#pragma unroll
        for (int q = 0; q < MAXD; ++q) {
#pragma unroll
            for (int r = q + 1; r < MAXD; ++r) {
                if (lab[q] == lab[r]) {
                    sum[q] += wt[r];
                    sum[r] += wt[q];
                }
            }
        }
#pragma unroll
        for (int q = 0; q < MAXD; ++q) sk[q] = lab[q] != kEmptyKey ? sum_key(sum[q]) : 0u;
    }
    uint32_t m = 0;
#pragma unroll
    for (int q = 0; q < MAXD; ++q) m = sk[q] > m ? sk[q] : m;
    uint32_t best_k = 0xffffffffu;
#pragma unroll
    for (int q = 0; q < MAXD; ++q) {
        const uint32_t kq = tr.key(lab[q]);
        if (sk[q] == m && kq < best_k) best_k = kq;
    }
    return m != 0u ? tr.label(best_k) : -1;
}

template <bool NS, int WK, bool BATCH, int MAXD>
__global__ void __launch_bounds__(kSmallThreads) k_sweep_small(DevState s, int flag_neighbours) {
    using T = typename Acc<WK>::T;
    const BinView bv = bin_view(s, 0);
    const Labels L = labels_of(s);
    const bool marks = marks_on(s, flag_neighbours);
    const uint32_t sweep = NS ? (uint32_t)s.ctrl->iter + 1u : 0u;   // non-strict tie-break (Section 4.1.5)
    // A dense pass over a bin holding most vertices walks the vertex ids
    // themselves (coalesced offsets, one dependent load less than the list)
    // and keeps those of this bin.
    const bool iota = L.dense && s.small_iota;
    const bool ident = identity_sweep<false, BATCH>(s);
    const unsigned cnt = iota ? (unsigned)s.N : bv.cnt;
    const unsigned stride = gridDim.x * blockDim.x;
    const int small_max = s.small_max;

    // Each thread walks the frontier slots k, k + stride, ... as a software
    // pipeline: while slot k is evaluated (its neighbour labels in flight),
    // the row of the next slot and the offsets and own label of the one after
    // are loaded too, so a step waits for about one load latency instead of
    // the whole chain frontier id -> offsets -> row -> labels.
    struct Head {
        int64_t st, en;
        int32_t v, own, g;
    };
    struct Row {
        int32_t v, own, g, done;
        int d;
        bool slot;
        int32_t nb[MAXD];
        T wt[MAXD];
    };
    auto vertex_of = [&](unsigned k) -> int32_t { return k < cnt ? (iota ? (int32_t)k : bv.list[k]) : -1; };
    auto head_of = [&](int32_t v) -> Head {
        Head h{0, 0, v, 0, 0};
        if (v >= 0) {
            h.st = s.off[v];
            h.en = s.off_end[v];
            h.own = L.C[v];
            if constexpr (BATCH) h.g = s.gid[v];
        }
        return h;
    };
    auto row_of = [&](const Head& h) -> Row {
        Row r;
        r.v = h.v;
        r.own = h.own;
        r.g = h.g;
        const int64_t dd = h.en - h.st;
        r.slot = h.v >= 0 && (!iota || (dd >= 1 && dd <= small_max));
        r.d = r.slot ? (int)dd : 0;
#pragma unroll
        for (int q = 0; q < MAXD; ++q) {
            r.nb[q] = q < r.d ? load_index(s.idx, h.st + q) : h.v;
            r.wt[q] = q < r.d ? load_weight<WK>(s.w, h.st + q) : (T)0;
        }
        r.done = 0;
        if constexpr (BATCH) r.done = r.slot ? s.done[r.g] : 0;
        return r;
    };

    const unsigned k0 = blockIdx.x * blockDim.x + threadIdx.x;
    Row cur = row_of(head_of(vertex_of(k0)));
    Head nxt = head_of(vertex_of(k0 + stride));
    int32_t vn = vertex_of(k0 + 2 * stride);
    unsigned long long my_changed = 0, my_changed_entries = 0;
    for (unsigned rbase = blockIdx.x * blockDim.x; rbase < cnt; rbase += stride) {
        const unsigned k = rbase + threadIdx.x;
        const int32_t v = cur.v;
        const bool act = cur.slot && !(BATCH && cur.done);
        int32_t lab[MAXD];
        T wt[MAXD];
#pragma unroll
        for (int q = 0; q < MAXD; ++q) {
            const bool ok = act && q < cur.d && cur.nb[q] != v;
            lab[q] = ok ? (ident ? initial_label(s, cur.nb[q]) : load_label<false>(L.C, cur.nb[q])) : kEmptyKey;
            wt[q] = ok ? cur.wt[q] : (T)0;
        }
        // the next stages, issued before this slot's labels are consumed
        const Row r_next = row_of(nxt);
        const Head h_next = head_of(vn);
        const int32_t v_next = vertex_of(k + 3 * stride);

        const TieRule tr = tie_rule(s, NS && act, sweep, v);
        const int32_t best = small_argmax<WK, MAXD>(lab, wt, tr);
        const bool changed = act && best >= 0 && best != cur.own;
        if (cur.slot) record_label<false>(L, bv.chg + k, v, cur.own, best, changed);
        if (changed) {
            if (marks) {
#pragma unroll
                for (int q = 0; q < MAXD; ++q)
                    if (q < cur.d && cur.nb[q] != v) s.flags[cur.nb[q]] = 1;
            }
            ++my_changed;
            my_changed_entries += (unsigned)cur.d;
        }
        count_graph_changes<BATCH>(s, changed, v);
        cur = r_next;
        nxt = h_next;
        vn = v_next;
    }
    flush_bin_counts(s, 0, my_changed, my_changed_entries);
}

// Staged asynchronous variant (see the file comment).
template <int WK, int MAXD>
__host__ __device__ constexpr size_t async_smem_bytes() {
    return (size_t)kSmallThreads * kStride * (4 + 4 + 4 * MAXD + (WK == W_UNIT ? 0 : 4 * MAXD) + 1);
}

template <int WK, bool BATCH, int MAXD, bool NS>
__global__ void __launch_bounds__(kSmallThreads) k_sweep_small_async(DevState s, int flag_neighbours) {
    using T = typename Acc<WK>::T;
    constexpr int SL = kSmallThreads * kStride;              // slots per array
    extern __shared__ __align__(16) unsigned char smem_raw[];
    int32_t* sv = reinterpret_cast<int32_t*>(smem_raw);       // vertex, -1 = inactive slot
    int32_t* sown = sv + SL;                                   // its label before the sweep
    int32_t* sidx = sown + SL;                                 // [MAXD][SL] row indices
    T* sw = reinterpret_cast<T*>(sidx + MAXD * SL);            // [MAXD][SL] weights (not for unit weights)
    uint8_t* sd = reinterpret_cast<uint8_t*>(sidx + MAXD * SL + (WK == W_UNIT ? 0 : MAXD * SL));
    const BinView bv = bin_view(s, 0);
    const Labels L = labels_of(s);
    const bool marks = marks_on(s, flag_neighbours);
    const uint32_t sweep = NS ? (uint32_t)s.ctrl->iter + 1u : 0u;   // non-strict tie-break (Section 4.1.5)
    const bool po = s.ctrl->prune_other != 0;                        // FLPA's pruning rule
    const unsigned cnt = bv.cnt;
    unsigned long long my_changed = 0, my_changed_entries = 0;
    for (unsigned tile = blockIdx.x * (unsigned)kTile; tile < cnt; tile += gridDim.x * (unsigned)kTile) {
        // stage: entry i of the tile goes to run i / kRun, position i % kRun
#pragma unroll 1
        for (int r = 0; r < kRun; ++r) {
            const unsigned i = (unsigned)r * kSmallThreads + threadIdx.x;
            const unsigned pos = (i / kRun) * kStride + (i % kRun);
            const unsigned k = tile + i;
            int32_t v = -1;
            int d = 0;
            int64_t st = 0;
            if (k < cnt) {
                v = bv.list[k];
                bool act = true;
                if constexpr (BATCH) act = !s.done[s.gid[v]];
                if (act) {
                    st = s.off[v];
                    d = (int)(s.off_end[v] - st);
                } else {
                    v = -1;
                }
            }
            sv[pos] = v;
            sd[pos] = (uint8_t)d;
            sown[pos] = v >= 0 ? __ldcg(L.C + v) : 0;
#pragma unroll
            for (int q = 0; q < MAXD; ++q) {
                const bool ok = q < d;
                sidx[q * SL + pos] = ok ? load_index(s.idx, st + q) : -1;
                if constexpr (WK != W_UNIT) sw[q * SL + pos] = ok ? load_weight<WK>(s.w, st + q) : (T)0;
            }
        }
        __syncthreads();
        // walk this thread's run in order
        for (int step = 0; step < kRun; ++step) {
            const unsigned pos = threadIdx.x * kStride + step;
            const int32_t v = sv[pos];
            bool changed = false;
            if (v >= 0) {
                const int d = sd[pos];
                int32_t lab[MAXD];
                T wt[MAXD];
#pragma unroll
                for (int q = 0; q < MAXD; ++q) {
                    const int32_t j = sidx[q * SL + pos];
                    const bool ok = q < d && j != v;
                    lab[q] = ok ? load_label<true>(L.C, j) : kEmptyKey;
                    if constexpr (WK == W_UNIT) wt[q] = ok ? (T)1 : (T)0;
                    else wt[q] = ok ? sw[q * SL + pos] : (T)0;
                }
                const TieRule tr = tie_rule(s, NS, sweep, v);
                const int32_t best = small_argmax<WK, MAXD>(lab, wt, tr);
                const int32_t own = sown[pos];
                changed = best >= 0 && best != own;
                if (changed) {
                    L.C[v] = best;
                    if (marks) {
#pragma unroll
                        for (int q = 0; q < MAXD; ++q) {
                            const int32_t j = sidx[q * SL + pos];
                            // FLPA's rule: a neighbour already carrying `best` stays unmarked
                            if (q < d && j != v && !(po && lab[q] == best)) s.flags[j] = 1;
                        }
                    }
                    ++my_changed;
                    my_changed_entries += (unsigned)d;
                }
            }
            count_graph_changes<BATCH>(s, changed, v);
        }
        __syncthreads();    // the tile is consumed before the next one is staged
    }
    flush_bin_counts(s, 0, my_changed, my_changed_entries);
}

template <int WK, bool BATCH, int MAXD, bool NS>
static cudaError_t launch_small_async_t(const DevState& s, int flag, int sms, cudaStream_t st) {
    const size_t smem = async_smem_bytes<WK, MAXD>();
    auto kern = k_sweep_small_async<WK, BATCH, MAXD, NS>;
    cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    int per_sm = 0;
    err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kSmallThreads, smem);
    if (err != cudaSuccess) return err;
    kern<<<sms * (per_sm > 0 ? per_sm : 1), kSmallThreads, smem, st>>>(s, flag);
    return cudaGetLastError();
}

// One resident wave: each thread runs its pipeline over many slots.
template <bool NS, int WK, bool BATCH, int MAXD>
static cudaError_t launch_small_sync_t(const DevState& s, int flag, int sms, cudaStream_t st) {
    auto kern = k_sweep_small<NS, WK, BATCH, MAXD>;
    int per_sm = 0;
    cudaError_t err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kSmallThreads, 0);
    if (err != cudaSuccess) return err;
    kern<<<sms * (per_sm > 0 ? per_sm : 1), kSmallThreads, 0, st>>>(s, flag);
    return cudaGetLastError();
}

template <int WK, bool BATCH, bool NS>
static cudaError_t launch_small_t(const DevState& s, bool async, int flag, int sms, cudaStream_t st) {
    const bool four = s.small_max <= 4;
    if (async) {
        return four ? launch_small_async_t<WK, BATCH, 4, NS>(s, flag, sms, st)
                    : launch_small_async_t<WK, BATCH, 8, NS>(s, flag, sms, st);
    }
    return four ? launch_small_sync_t<NS, WK, BATCH, 4>(s, flag, sms, st)
                : launch_small_sync_t<NS, WK, BATCH, 8>(s, flag, sms, st);
}

template <int WK, bool NS>
static cudaError_t launch_small_w(const DevState& s, bool async, int flag, int sms, cudaStream_t st) {
    return s.G > 1 ? launch_small_t<WK, true, NS>(s, async, flag, sms, st)
                   : launch_small_t<WK, false, NS>(s, async, flag, sms, st);
}

template <bool NS>
static cudaError_t launch_small_ns(const DevState& s, bool async, int flag, int sms, cudaStream_t st) {
    switch (s.weight_kind) {
        case W_UNIT: return launch_small_w<W_UNIT, NS>(s, async, flag, sms, st);
        case W_U32: return launch_small_w<W_U32, NS>(s, async, flag, sms, st);
        case W_U8: return launch_small_w<W_U8, NS>(s, async, flag, sms, st);
        default: return launch_small_w<W_F32, NS>(s, async, flag, sms, st);
    }
}

cudaError_t launch_sweep_small(const DevState& s, int mode, cudaStream_t st, int sms) {
    const bool ns = (mode & kModeNonstrict) != 0;
    mode &= ~kModeNonstrict;
    const bool async = mode == MODE_ASYNC;
    const int flag = mode != MODE_SYNC_FULL;
    return ns ? launch_small_ns<true>(s, async, flag, sms, st) : launch_small_ns<false>(s, async, flag, sms, st);
}

}  // namespace lpa
