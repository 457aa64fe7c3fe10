// lpa_sweep_block.cu -- sweep for vertices with degree above warp_max: one
// thread block per frontier vertex, the block size growing with the degree
// bin (128 threads up to mid_max, 256 up to large_max, 512 above) so that the
// shared table (2^ceil(log2(2d)) slots) per warp stays about constant and the
// SM keeps enough warps in flight.
//
// Warps read the row in 32-entry chunks and group equal labels with
// __match_any_sync as in the warp kernel; group leaders add their sums into a
// shared-memory open-addressing table.  In the last bin, when the row could
// hold more distinct labels than half the shared table (2d > slots), inserts
// probe at most kSharedProbes slots and then go to a spill table in global
// memory private to this block (2^ceil(log2(2d)) slots, so it never fills).  Each label lives in exactly one of the two tables, so scanning both
// yields every K_{i->c} (Eq. 3).  The block then reduces (sum, smallest label)
// to the winner (Section 4.1.5), clears what it used, and on change marks the
// neighbours unprocessed (Section 4.1.4).
#include "lpa_device.cuh"

namespace lpa {

constexpr int kSharedProbes = 16;

template <bool ASYNC, int WK, bool BATCH>
__global__ void k_sweep_block(DevState s, int bin, int flag_neighbours) {
    using T = typename Acc<WK>::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int S = s.block_slots[bin - 2];
    int32_t* keys = reinterpret_cast<int32_t*>(smem_raw);
    T* vals = reinterpret_cast<T*>(keys + S);
    __shared__ uint32_t red_key[32];
    __shared__ int32_t red_lab[32];
    __shared__ int spilled;
    __shared__ int32_t winner;

    const unsigned lane = lane_id();
    const int wib = threadIdx.x >> 5;
    const int nw = blockDim.x >> 5;
    for (int q = threadIdx.x; q < S; q += blockDim.x) {
        keys[q] = kEmptyKey;
        vals[q] = (T)0;
    }
    if (threadIdx.x == 0) spilled = 0;
    const bool last_bin = bin == kBins - 1;
    int32_t* gkeys = (last_bin && s.spill_keys) ? s.spill_keys + (size_t)blockIdx.x * s.spill_slots : nullptr;
    T* gvals = gkeys ? static_cast<T*>(s.spill_vals) + (size_t)blockIdx.x * s.spill_slots : nullptr;
    __syncthreads();

    const BinView bv = bin_view(s, bin);
    const Labels L = labels_of(s);
    const unsigned cnt = bv.cnt;
    unsigned long long my_changed = 0, my_changed_entries = 0;
    for (unsigned k = blockIdx.x; k < cnt; k += gridDim.x) {
        const int32_t v = bv.list[k];
        const int32_t own = ASYNC ? __ldcg(L.C + v) : L.C[v];
        if constexpr (BATCH) {
            if (s.done[s.gid[v]]) {             // block-uniform
                if (threadIdx.x == 0) record_label<ASYNC>(L, bv.chg + k, v, own, own, false);
                continue;
            }
        }
        const int64_t st = s.off[v];
        const int64_t en = s.off[v + 1];
        const int64_t d = en - st;
        const int log_full = ceil_log2((unsigned)(2 * d));
        const bool fits = (1ll << log_full) <= S;
        const int log_s = fits ? log_full : ceil_log2((unsigned)S);
        // the spill table needs 2^log_full slots; the host sizes it for the max degree
        const bool may_spill = !fits && gkeys != nullptr && (1ll << log_full) <= s.spill_slots;
        for (int64_t e0 = st + (int64_t)wib * 32; e0 < en; e0 += (int64_t)nw * 32) {
            const int64_t e = e0 + lane;
            const bool in = e < en;
            const int32_t j = in ? load_index(s.idx, e) : v;
            const bool ok = in && j != v;
            const int32_t lab = ok ? load_label<ASYNC>(L.C, j) : kEmptyKey;
            T w = ok ? load_weight<WK>(s.w, e) : (T)0;
            bool lead = ok;
            if constexpr (WK != W_F32) {
                const unsigned peers = __match_any_sync(kFull, lab);
                if constexpr (WK == W_UNIT) {
                    w = (T)__popc(peers);
                } else {
                    w = __reduce_add_sync(peers, w);
                }
                lead = ok && lane == (unsigned)(__ffs(peers) - 1);
            }
            if (lead) {
                if (fits) {
                    if (!table_add<T>(keys, vals, log_s, lab, w)) atomicExch(&s.ctrl->error, 3);
                } else if (!table_add_bounded<T>(keys, vals, log_s, lab, w, kSharedProbes)) {
                    if (may_spill) {
                        if (!table_add<T>(gkeys, gvals, log_full, lab, w)) atomicExch(&s.ctrl->error, 3);
                        spilled = 1;
                    } else {
                        atomicExch(&s.ctrl->error, 1);   // host sized the spill table too small
                    }
                }
            }
        }
        __syncthreads();
        bool any = false;
        T best_w = 0;
        int32_t best = 0x7fffffff;
        const int slots_s = 1 << log_s;
        for (int q = threadIdx.x; q < slots_s; q += blockDim.x) {
            const int32_t kq = keys[q];
            if (kq != kEmptyKey) {
                const T vq = vals[q];
                if (!any || vq > best_w || (vq == best_w && kq < best)) {
                    any = true;
                    best_w = vq;
                    best = kq;
                }
                keys[q] = kEmptyKey;
                vals[q] = (T)0;
            }
        }
        if (spilled) {
            const int64_t slots_g = 1ll << log_full;
            for (int64_t q = threadIdx.x; q < slots_g; q += blockDim.x) {
                const int32_t kq = gkeys[q];
                if (kq != kEmptyKey) {
                    const T vq = gvals[q];
                    if (!any || vq > best_w || (vq == best_w && kq < best)) {
                        any = true;
                        best_w = vq;
                        best = kq;
                    }
                    gkeys[q] = kEmptyKey;
                    gvals[q] = (T)0;
                }
            }
        }
        // block argmax: per warp, then warp 0 over the warp winners
        uint32_t key = any ? sum_key(best_w) : 0u;
        uint32_t m = __reduce_max_sync(kFull, key);
        uint32_t c = __reduce_min_sync(kFull, (m != 0 && key == m) ? (uint32_t)best : 0xffffffffu);
        if (lane == 0) {
            red_key[wib] = m;
            red_lab[wib] = (int32_t)c;
        }
        __syncthreads();
        if (wib == 0) {
            uint32_t kk = (int)lane < nw ? red_key[lane] : 0u;
            int32_t ll = (int)lane < nw ? red_lab[lane] : 0;
            int32_t wlab = warp_argmax(kk, ll);
            if (lane == 0) {
                winner = wlab;
                spilled = 0;
            }
        }
        __syncthreads();
        const int32_t best_lab = winner;
        const bool changed = best_lab >= 0 && best_lab != own;   // block-uniform
        if (threadIdx.x == 0) record_label<ASYNC>(L, bv.chg + k, v, own, best_lab, changed);
        if (changed) {
            if (threadIdx.x == 0) {
                ++my_changed;
                my_changed_entries += (unsigned long long)d;
            }
            if (flag_neighbours) {
                for (int64_t e = st + threadIdx.x; e < en; e += blockDim.x) {
                    const int32_t j = s.idx[e];
                    if (j != v) s.flags[j] = 1;
                }
            }
        }
        if constexpr (BATCH) {
            if (threadIdx.x == 0 && changed) atomicAdd(&s.dN[s.gid[v]], 1ull);
        }
        __syncthreads();    // tables clear and `winner` consumed before the next vertex
    }
    flush_bin_counts(s, bin, my_changed, my_changed_entries);
}

int block_grid_for(const DevState& s, int bin, int sms) {
    const int threads = kBlockThreads[bin - 2];
    const size_t smem = (size_t)s.block_slots[bin - 2] * 8 + 512;
    int by_smem = (int)((220 * 1024) / smem);
    int by_threads = 2048 / threads;
    int per_sm = by_smem < by_threads ? by_smem : by_threads;
    if (per_sm < 1) per_sm = 1;
    return sms * per_sm;
}

template <bool ASYNC, int WK, bool BATCH>
static cudaError_t launch_block_t(const DevState& s, int bin, int flag, int blocks, cudaStream_t st) {
    const size_t smem = (size_t)s.block_slots[bin - 2] * 8;
    auto kern = k_sweep_block<ASYNC, WK, BATCH>;
    cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    kern<<<blocks, kBlockThreads[bin - 2], smem, st>>>(s, bin, flag);
    return cudaGetLastError();
}

cudaError_t launch_sweep_block(const DevState& s, int mode, int bin, int blocks, cudaStream_t st) {
    const bool async = mode == MODE_ASYNC;
    const int flag = mode != MODE_SYNC_FULL;
    const bool batch = s.G > 1;
#define LPA_BLOCK_W(A, B)                                                             \
    switch (s.weight_kind) {                                                          \
        case W_UNIT: return launch_block_t<A, W_UNIT, B>(s, bin, flag, blocks, st);   \
        case W_U32: return launch_block_t<A, W_U32, B>(s, bin, flag, blocks, st);     \
        default: return launch_block_t<A, W_F32, B>(s, bin, flag, blocks, st);        \
    }
    if (async) {
        if (batch) { LPA_BLOCK_W(true, true) } else { LPA_BLOCK_W(true, false) }
    } else {
        if (batch) { LPA_BLOCK_W(false, true) } else { LPA_BLOCK_W(false, false) }
    }
#undef LPA_BLOCK_W
}

}  // namespace lpa
