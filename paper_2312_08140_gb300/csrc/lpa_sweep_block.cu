// lpa_sweep_block.cu -- sweep for vertices with degree above warp_max: one
// thread block per frontier vertex, the block size growing with the degree
// bin (128 threads up to mid_max, 256 up to large_max, 512 above) so that the
// shared table (2^ceil(log2(2d)) slots) per warp stays about constant and the
// SM keeps enough warps in flight.
//
// Warps read the row in 32-entry chunks and group equal labels with
// __match_any_sync as in the warp kernel; group leaders add their sums into a
// shared-memory open-addressing table; the block then reduces (sum, smallest
// label) to the winner (Eq. 2; Section 4.1.5) and, on change, marks the
// neighbours unprocessed (Section 4.1.4).
//
// Last bin (d > large_max): the table has kLargeSlots slots.  Rows longer than
// kLargeSlots / 2 may carry more distinct labels than it holds; their inserts
// probe a bounded number of slots and, if one fails, the block stops and
// appends the row to an overflow list.  A second kernel (k_sweep_parts) then
// rescans each overflowed row with parts = ceil(2d / kLargeSlots) blocks:
// block p aggregates only the labels whose hash lands in partition p (about
// d / parts distinct labels at most, half of the table, so an insert always
// finds a slot), folds its winner into a 64-bit atomicMax of
// (sum << 32 | ~label) -- larger sum first, then smaller label -- and the
// block that completes the row applies the result.  No block waits on another.
#include "lpa_device.cuh"

namespace lpa {

constexpr int kSharedProbes = 16;
constexpr int kUnroll = 4;          // chunks of 32 entries in flight per warp

// Block-wide argmax of one (key, label) candidate per thread; returns the
// winner (or -1) to every thread.  Uses red_key/red_lab (32 entries) and
// `winner` in shared memory.
__device__ __forceinline__ int32_t block_argmax(uint32_t key, int32_t label, uint32_t* red_key, int32_t* red_lab,
                                                int32_t* winner) {
    const unsigned lane = lane_id();
    const int wib = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const uint32_t m = __reduce_max_sync(kFull, key);
    const uint32_t c = __reduce_min_sync(kFull, (m != 0 && key == m) ? (uint32_t)label : 0xffffffffu);
    if (lane == 0) {
        red_key[wib] = m;
        red_lab[wib] = (int32_t)c;
    }
    __syncthreads();
    if (wib == 0) {
        const uint32_t kk = (int)lane < nw ? red_key[lane] : 0u;
        const int32_t ll = (int)lane < nw ? red_lab[lane] : 0;
        const int32_t w = warp_argmax(kk, ll);
        if (lane == 0) *winner = w;
    }
    __syncthreads();
    return *winner;
}

// Scans table slots [0, slots) for this thread's best candidate and clears
// the slots it visits.
template <typename T>
__device__ __forceinline__ void scan_table(int32_t* keys, T* vals, int slots, uint32_t& key, int32_t& cand) {
    bool any = false;
    T best_w = 0;
    int32_t best = 0x7fffffff;
    for (int q = threadIdx.x; q < slots; q += blockDim.x) {
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
    key = any ? sum_key(best_w) : 0u;
    cand = best;
}

__device__ __forceinline__ void mark_neighbours(const DevState& s, int32_t v, int64_t st, int64_t en) {
    for (int64_t e = st + threadIdx.x; e < en; e += blockDim.x) {
        const int32_t j = s.idx[e];
        if (j != v) mark_unprocessed(s.flags, j);
    }
}

// U: chunks in flight per warp (4 for the last bin, whose rows span many
// chunks per warp; 1 for the middle bins, where the SM's 64 warps already
// overlap the few chunks of each row).
template <bool ASYNC, int WK, bool BATCH, int U>
__global__ void k_sweep_block(DevState s, int bin, int flag_neighbours) {
    using T = typename Acc<WK>::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int S = s.block_slots[bin - 2];
    int32_t* keys = reinterpret_cast<int32_t*>(smem_raw);
    T* vals = reinterpret_cast<T*>(keys + S);
    __shared__ uint32_t red_key[32];
    __shared__ int32_t red_lab[32];
    __shared__ int overflow;
    __shared__ int32_t winner;

    const unsigned lane = lane_id();
    const int wib = threadIdx.x >> 5;
    const int nw = blockDim.x >> 5;
    for (int q = threadIdx.x; q < S; q += blockDim.x) {
        keys[q] = kEmptyKey;
        vals[q] = (T)0;
    }
    if (threadIdx.x == 0) overflow = 0;
    __syncthreads();

    const BinView bv = bin_view(s, bin);
    const Labels L = labels_of(s);
    const bool marks = marks_on(s, flag_neighbours);
    const unsigned cnt = bv.cnt;
    const int log_S = ceil_log2((unsigned)S);
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
        const int64_t en = s.off_end[v];
        const int64_t d = en - st;
        const int log_full = ceil_log2((unsigned)(2 * d));
        const bool fits = log_full <= log_S;
        const int log_s = fits ? log_full : log_S;
        // Each warp takes U chunks per step (chunk c = wib + (u + U*it)*nw):
        // their index loads, then their label gathers and weights, are issued
        // together so the latencies overlap; then the chunks are aggregated.
        const int64_t step = (int64_t)nw * 32;
        for (int64_t e0 = st + (int64_t)wib * 32; e0 < en; e0 += step * U) {
            if (!fits && *(volatile int*)&overflow) break;     // warp-uniform
            int32_t jj[U], lab[U];
            T ww[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int64_t e = e0 + u * step + lane;
                jj[u] = e < en ? load_index_keep(s.idx, e) : v;
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int64_t e = e0 + u * step + lane;
                const bool ok = jj[u] != v;                      // also false past the row end
                lab[u] = ok ? load_label<ASYNC>(L.C, jj[u]) : kEmptyKey;
                ww[u] = ok ? load_weight<WK>(s.w, e) : (T)0;
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                if (e0 + u * step >= en) break;                 // warp-uniform
                const bool ok = jj[u] != v;
                T w = ww[u];
                bool lead = ok;
                if constexpr (WK != W_F32) {
                    const unsigned peers = __match_any_sync(kFull, lab[u]);
                    if constexpr (WK == W_UNIT) {
                        w = (T)__popc(peers);
                    } else {
                        w = __reduce_add_sync(peers, w);
                    }
                    lead = ok && lane == (unsigned)(__ffs(peers) - 1);
                }
                if (lead) {
                    if (fits) {
                        if (!table_add<T>(keys, vals, log_s, lab[u], w)) atomicExch(&s.ctrl->error, 3);
                    } else if (!table_add_bounded<T>(keys, vals, log_s, lab[u], w, kSharedProbes)) {
                        overflow = 1;
                    }
                }
            }
        }
        __syncthreads();
        uint32_t key;
        int32_t cand;
        scan_table<T>(keys, vals, 1 << log_s, key, cand);     // also clears the table
        const int ovf = overflow;
        const int32_t best_lab = block_argmax(key, cand, red_key, red_lab, &winner);
        if (ovf) {
            // hand the row to the partitioned rescan
            if (threadIdx.x == 0) {
                const uint32_t parts = (uint32_t)((2 * d + S - 1) / S);
                const unsigned long long old =
                    atomicAdd(&s.ctrl->ovf_packed, (1ull << 40) | (unsigned long long)parts);
                Overflow& o = s.ovf[old >> 40];
                o.v = v;
                o.slot = k;
                o.st = st;
                o.d = (int32_t)d;
                o.own = own;
                o.item_base = (uint32_t)(old & ((1ull << 40) - 1));
                o.parts = parts;
                o.best = 0ull;
                o.done = 0u;
                overflow = 0;
            }
            __syncthreads();
            continue;
        }
        const bool changed = best_lab >= 0 && best_lab != own;   // block-uniform
        if (threadIdx.x == 0) record_label<ASYNC>(L, bv.chg + k, v, own, best_lab, changed);
        if (changed) {
            if (threadIdx.x == 0) {
                ++my_changed;
                my_changed_entries += (unsigned long long)d;
                if constexpr (BATCH) atomicAdd(&s.dN[s.gid[v]], 1ull);
            }
            if (marks) mark_neighbours(s, v, st, en);
        }
        __syncthreads();    // `winner` consumed before the next vertex
    }
    flush_bin_counts(s, bin, my_changed, my_changed_entries);
}

__device__ __forceinline__ uint32_t part_of(int32_t label, uint32_t parts) {
    uint32_t h = (uint32_t)label;            // murmur3 finaliser, then multiply-shift into [0, parts)
    h ^= h >> 16;
    h *= 0x85ebca6bu;
    h ^= h >> 13;
    h *= 0xc2b2ae35u;
    h ^= h >> 16;
    return (uint32_t)(((unsigned long long)h * parts) >> 32);
}

template <bool ASYNC, int WK, bool BATCH>
__global__ void k_sweep_parts(DevState s, int flag_neighbours) {
    using T = typename Acc<WK>::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int S = kLargeSlots;
    int32_t* keys = reinterpret_cast<int32_t*>(smem_raw);
    T* vals = reinterpret_cast<T*>(keys + S);
    __shared__ uint32_t red_key[32];
    __shared__ int32_t red_lab[32];
    __shared__ int32_t winner;
    __shared__ int resolver;
    __shared__ unsigned long long best_packed;

    const unsigned lane = lane_id();
    const int wib = threadIdx.x >> 5;
    const int nw = blockDim.x >> 5;
    for (int q = threadIdx.x; q < S; q += blockDim.x) {
        keys[q] = kEmptyKey;
        vals[q] = (T)0;
    }
    __syncthreads();

    const unsigned long long packed = s.ctrl->ovf_packed;
    const uint32_t nent = (uint32_t)(packed >> 40);
    const uint32_t items = (uint32_t)(packed & ((1ull << 40) - 1));
    const BinView bv = bin_view(s, kBins - 1);
    const Labels L = labels_of(s);
    const bool marks = marks_on(s, flag_neighbours);
    const int log_S = ceil_log2((unsigned)S);
    unsigned long long my_changed = 0, my_changed_entries = 0;
    for (uint32_t item = blockIdx.x; item < items; item += gridDim.x) {
        // entry owning this item: largest e with item_base <= item (bases ascend with e)
        uint32_t lo = 0, hi = nent;
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            if (s.ovf[mid].item_base <= item) lo = mid;
            else hi = mid;
        }
        Overflow& o = s.ovf[lo];
        const int32_t v = o.v;
        const int64_t st = o.st, en = o.st + o.d;
        const uint32_t parts = o.parts, p = item - o.item_base;
        const int64_t step = (int64_t)nw * 32;
        for (int64_t e0 = st + (int64_t)wib * 32; e0 < en; e0 += step * kUnroll) {
            int32_t jj[kUnroll], lab[kUnroll];
            T ww[kUnroll];
#pragma unroll
            for (int u = 0; u < kUnroll; ++u) {
                const int64_t e = e0 + u * step + lane;
                jj[u] = e < en ? load_index(s.idx, e) : v;
            }
#pragma unroll
            for (int u = 0; u < kUnroll; ++u) {
                const int64_t e = e0 + u * step + lane;
                bool ok = jj[u] != v;
                int32_t l = ok ? load_label<ASYNC>(L.C, jj[u]) : kEmptyKey;
                ok = ok && part_of(l, parts) == p;
                lab[u] = ok ? l : kEmptyKey;
                ww[u] = ok ? load_weight<WK>(s.w, e) : (T)0;
            }
#pragma unroll
            for (int u = 0; u < kUnroll; ++u) {
                if (e0 + u * step >= en) break;                 // warp-uniform
                const bool ok = lab[u] != kEmptyKey;
                T w = ww[u];
                bool lead = ok;
                if constexpr (WK != W_F32) {
                    const unsigned peers = __match_any_sync(kFull, lab[u]);
                    if constexpr (WK == W_UNIT) {
                        w = (T)__popc(peers);
                    } else {
                        w = __reduce_add_sync(peers, w);
                    }
                    lead = ok && lane == (unsigned)(__ffs(peers) - 1);
                }
                if (lead && !table_add<T>(keys, vals, log_S, lab[u], w)) atomicExch(&s.ctrl->error, 4);
            }
        }
        __syncthreads();
        uint32_t key;
        int32_t cand;
        scan_table<T>(keys, vals, S, key, cand);
        const int32_t part_best = block_argmax(key, cand, red_key, red_lab, &winner);
        if (threadIdx.x == 0) {
            // winner's key again: every thread holding the winning label reports it
            resolver = 0;
        }
        __syncthreads();
        if (part_best >= 0 && key != 0 && cand == part_best) {
            const unsigned long long pk = ((unsigned long long)key << 32) | (unsigned long long)(~(uint32_t)part_best);
            atomicMax(&o.best, pk);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            const unsigned t = atomicAdd(&o.done, 1u);
            if (t == parts - 1) {
                __threadfence();
                best_packed = atomicAdd(&o.best, 0ull);
                resolver = 1;
            }
        }
        __syncthreads();
        if (resolver) {
            const unsigned long long bp = best_packed;
            const int32_t best_lab = (bp >> 32) ? (int32_t)(~(uint32_t)(bp & 0xffffffffull)) : -1;
            const int32_t own = o.own;
            const bool changed = best_lab >= 0 && best_lab != own;
            if (threadIdx.x == 0) {
                record_label<ASYNC>(L, bv.chg + o.slot, v, own, best_lab, changed);
                if (changed) {
                    ++my_changed;
                    my_changed_entries += (unsigned long long)o.d;
                    if constexpr (BATCH) atomicAdd(&s.dN[s.gid[v]], 1ull);
                }
            }
            if (changed && marks) mark_neighbours(s, v, st, en);
        }
        __syncthreads();
    }
    flush_bin_counts(s, kBins - 1, my_changed, my_changed_entries);
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
    auto kern = bin == kBins - 1 ? k_sweep_block<ASYNC, WK, BATCH, kUnroll> : k_sweep_block<ASYNC, WK, BATCH, 1>;
    cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    kern<<<blocks, kBlockThreads[bin - 2], smem, st>>>(s, bin, flag);
    err = cudaGetLastError();
    if (err != cudaSuccess || bin != kBins - 1) return err;
    const size_t psmem = (size_t)kLargeSlots * 8;
    auto pk = k_sweep_parts<ASYNC, WK, BATCH>;
    err = cudaFuncSetAttribute(pk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)psmem);
    if (err != cudaSuccess) return err;
    pk<<<blocks, kBlockThreads[kBlockBins - 1], psmem, st>>>(s, flag);
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
        case W_U8: return launch_block_t<A, W_U8, B>(s, bin, flag, blocks, st);       \
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
