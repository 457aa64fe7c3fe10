// lpa_sweep_block.cu -- the rows of the last degree bin whose distinct labels
// overflow the shared table of the block-per-row kernel (lpa_sweep_rows.cu),
// and the launcher of the block bins.
//
// An overflowing row's labels are split over parts = ceil(2d / kLargeSlots)
// hash partitions (about d / parts distinct labels each at most, half of the
// table, so an insert always finds a slot): the row is read once in slices
// grouped by partition (k_ovf_slices) and aggregated by one block per
// partition (k_ovf_parts); rows beyond that path's limits are rescanned by one
// block per partition (k_sweep_parts).  Each partition's winner is folded
// into a 64-bit atomicMax of (sum << 32 | ~tie key) -- larger sum first, then
// the tie-break (Eq. 2; Section 4.1.5) -- and the block that completes the
// row applies the result and marks the neighbours (Section 4.1.4).  No block
// waits on another.
#include "lpa_device.cuh"

namespace lpa {

constexpr int kUnroll = 4;          // chunks of 32 entries in flight per warp
constexpr int kSliceThreads = 512;  // blocks of the sliced overflow path

// Block-wide argmax of one (sum key, tie key) candidate per thread: the
// largest sum key, then the smallest tie key.  Returns the winning tie key
// (0xffffffff when no thread holds a candidate) to every thread.  Uses
// red_key/red_tie (32 entries) and `winner` in shared memory.
__device__ __forceinline__ uint32_t block_argmax(uint32_t key, uint32_t tie, uint32_t* red_key, uint32_t* red_tie,
                                                 uint32_t* winner) {
    const unsigned lane = lane_id();
    const int wib = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const uint32_t m = __reduce_max_sync(kFull, key);
    const uint32_t c = __reduce_min_sync(kFull, (m != 0 && key == m) ? tie : 0xffffffffu);
    if (lane == 0) {
        red_key[wib] = m;
        red_tie[wib] = c;
    }
    __syncthreads();
    if (wib == 0) {
        const uint32_t kk = (int)lane < nw ? red_key[lane] : 0u;
        const uint32_t tt = (int)lane < nw ? red_tie[lane] : 0xffffffffu;
        const uint32_t w = warp_argmax_tie(kk, tt);
        if (lane == 0) *winner = w;
    }
    __syncthreads();
    return *winner;
}

// This thread's best candidate of the row's table under the row's tie rule
// (sum key, tie key); clears the slots it visits.  With `lists` the slots the
// row filled are read from the warps' segments (wcnt[w] entries of segment w,
// seg_cap each; wpre holds their prefix sums); without, or when a segment
// overflowed, all `slots` slots are scanned.
template <typename T>
__device__ __forceinline__ void scan_table(int32_t* keys, T* vals, int slots, bool lists, const uint16_t* segs,
                                           unsigned seg_cap, const unsigned* wpre, int nw, const TieRule& tr,
                                           uint32_t& key, uint32_t& tie) {
    bool any = false;
    T best_w = 0;
    uint32_t best_k = 0xffffffffu;
    auto visit = [&](int q) {
        const int32_t kq = keys[q];
        if (kq != kEmptyKey) {
            const T vq = vals[q];
            const uint32_t tq = tr.key(kq);
            if (!any || vq > best_w || (vq == best_w && tq < best_k)) {
                any = true;
                best_w = vq;
                best_k = tq;
            }
            keys[q] = kEmptyKey;
            vals[q] = (T)0;
        }
    };
    if (lists) {
        const unsigned total = wpre[nw];
        for (unsigned f = threadIdx.x; f < total; f += blockDim.x) {
            int w = 0;
            while (w + 1 < nw && wpre[w + 1] <= f) ++w;
            visit(segs[(size_t)w * seg_cap + (f - wpre[w])]);
        }
    } else {
        for (int q = threadIdx.x; q < slots; q += blockDim.x) visit(q);
    }
    key = any ? sum_key(best_w) : 0u;
    tie = best_k;
}

// Marks v's neighbours unprocessed (Section 4.1.4); with FLPA's rule (po)
// only those whose label is not v's new label `best`.
template <bool ASYNC>
__device__ __forceinline__ void mark_neighbours(const DevState& s, int32_t v, int64_t st, int64_t en, bool po,
                                                int32_t best, const int32_t* C) {
    for (int64_t e = st + threadIdx.x; e < en; e += blockDim.x) {
        const int32_t j = s.idx[e];
        if (j != v && !(po && load_label<ASYNC>(C, j) == best)) mark_unprocessed(s.flags, j);
    }
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

// ------------------------------------------------------ overflowing rows --
// Owner of a work item: the largest e with base(e) <= item (bases ascend with
// e; rows contributing no items on a path have the next row's base, so they
// are never the largest such e for an item they do not own).
template <uint32_t Overflow::*F>
__device__ __forceinline__ uint32_t owner_of(const Overflow* ovf, uint32_t n, uint32_t item) {
    uint32_t lo = 0, hi = n;
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (ovf[mid].*F <= item) lo = mid;
        else hi = mid;
    }
    return lo;
}

static_assert(2 * kMaxParts * sizeof(uint32_t) <= kLargeSlots * 8, "slice counters fit the table's memory");

// Block-wide exclusive scan of K 64-bit values (blockDim.x a multiple of 32,
// at most 1024).  Returns the block totals in `total`.
template <int K>
__device__ __forceinline__ void block_exclusive_scan(const unsigned long long (&v)[K], unsigned long long (&ex)[K],
                                                     unsigned long long (&total)[K]) {
    __shared__ unsigned long long ws[32][K];
    __shared__ unsigned long long tot[K];
    const unsigned lane = lane_id();
    const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        unsigned long long incl = v[k];
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(kFull, incl, o);
            if ((int)lane >= o) incl += y;
        }
        ex[k] = incl - v[k];
        if (lane == 31) ws[w][k] = incl;
    }
    __syncthreads();
    if (w == 0) {
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const unsigned long long x = (int)lane < nw ? ws[lane][k] : 0ull;
            unsigned long long incl = x;
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned long long y = __shfl_up_sync(kFull, incl, o);
                if ((int)lane >= o) incl += y;
            }
            if ((int)lane < nw) ws[lane][k] = incl - x;
            if (lane == 31) tot[k] = incl;
        }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < K; ++k) {
        ex[k] += ws[w][k];
        total[k] = tot[k];
    }
    __syncthreads();
}

// One block: work-item bases of the rows that overflowed in this pass.  Rows
// whose partition and slice counts qualify take the sliced path while their
// scratch (d pairs, Q x P counts, in row order) fits; the others take the
// rescan path.
__global__ void __launch_bounds__(1024) k_ovf_plan(DevState s) {
    Ctrl* c = s.ctrl;
    const unsigned n = (unsigned)c->ovf_count;
    unsigned long long run[4] = {0, 0, 0, 0};   // pairs, counts, slices, parts over eligible rows
    unsigned long long rrun = 0;                // rescan parts
    unsigned long long sl_items = 0, pt_items = 0;
    for (unsigned c0 = 0; c0 < n; c0 += blockDim.x) {
        const unsigned e = c0 + threadIdx.x;
        unsigned long long v[4] = {0, 0, 0, 0};
        uint32_t P = 0, Q = 0;
        if (e < n) {
            const Overflow& o = s.ovf[e];
            P = o.parts;
            Q = (uint32_t)((o.d + kSliceLen - 1) / kSliceLen);
            if (P >= (uint32_t)kSliceMinParts && P <= (uint32_t)kMaxParts && Q <= (uint32_t)kMaxSlices) {
                v[0] = (unsigned long long)o.d;
                v[1] = (unsigned long long)Q * P;
                v[2] = Q;
                v[3] = P;
            }
        }
        unsigned long long ex[4], tot[4];
        block_exclusive_scan<4>(v, ex, tot);
        bool sliced = false;
        if (e < n && v[0] > 0) {
            const unsigned long long pairs_end = run[0] + ex[0] + v[0];
            const unsigned long long cnt_end = run[1] + ex[1] + v[1];
            sliced = pairs_end <= (unsigned long long)s.ovf_pairs_cap && cnt_end <= (unsigned long long)s.ovf_cnt_cap &&
                     run[2] + ex[2] + v[2] < (1ull << 32) && run[3] + ex[3] + v[3] < (1ull << 32);
        }
        unsigned long long rv[1] = {(e < n && !sliced) ? (unsigned long long)P : 0ull}, rex[1], rtot[1];
        block_exclusive_scan<1>(rv, rex, rtot);
        if (e < n) {
            Overflow& o = s.ovf[e];
            o.pair_base = (int64_t)(run[0] + ex[0]);
            o.cnt_base = (int64_t)(run[1] + ex[1]);
            o.slice_base = (uint32_t)(run[2] + ex[2]);
            o.part_base = (uint32_t)(run[3] + ex[3]);
            o.slices = sliced ? Q : 0u;
            o.rescan_base = (uint32_t)(rrun + rex[0]);
            o.rescan_parts = sliced ? 0u : P;
        }
        // sliced rows are a prefix of the eligible ones: item totals are the
        // slice and part prefixes at the last sliced row
        unsigned long long ls[2] = {sliced ? run[2] + ex[2] + v[2] : 0ull, sliced ? run[3] + ex[3] + v[3] : 0ull};
        for (int o2 = 16; o2 > 0; o2 >>= 1) {
            ls[0] = max(ls[0], __shfl_xor_sync(kFull, ls[0], o2));
            ls[1] = max(ls[1], __shfl_xor_sync(kFull, ls[1], o2));
        }
        __shared__ unsigned long long wmax[32][2];
        if (lane_id() == 0) {
            wmax[threadIdx.x >> 5][0] = ls[0];
            wmax[threadIdx.x >> 5][1] = ls[1];
        }
        __syncthreads();
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            sl_items = max(sl_items, wmax[w][0]);
            pt_items = max(pt_items, wmax[w][1]);
        }
        __syncthreads();
        for (int k = 0; k < 4; ++k) run[k] += tot[k];
        rrun += rtot[0];
    }
    if (threadIdx.x == 0) {
        c->ovf_slice_items = (unsigned)sl_items;
        c->ovf_part_items = (unsigned)pt_items;
        c->ovf_rescan_items = (unsigned)rrun;
    }
}

template <int WK>
__device__ __forceinline__ uint32_t sum_bits(typename Acc<WK>::T x) {
    if constexpr (WK == W_F32) return __float_as_uint(x);
    else return (uint32_t)x;
}

template <int WK>
__device__ __forceinline__ typename Acc<WK>::T sum_from_bits(uint32_t b) {
    if constexpr (WK == W_F32) return __uint_as_float(b);
    else return (typename Acc<WK>::T)b;
}

// Sliced path, step 1: a block per kSliceLen-entry slice of an overflowing
// row reads the slice once, groups equal labels per 32-entry chunk, and
// writes the groups as (label, partial sum) pairs ordered by label partition
// (counting sort in shared memory), with the count and offset of every
// partition's run.
template <bool ASYNC, int WK, bool BATCH>
__global__ void __launch_bounds__(kSliceThreads, 2) k_ovf_slices(DevState s) {
    using T = typename Acc<WK>::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint32_t* cnt = reinterpret_cast<uint32_t*>(smem_raw);   // [kMaxParts] counts, then cursors
    uint32_t* off = cnt + kMaxParts;                          // [kMaxParts] offsets
    const Labels L = labels_of(s);
    const unsigned n = (unsigned)s.ctrl->ovf_count;
    const unsigned items = s.ctrl->ovf_slice_items;
    const unsigned lane = lane_id();
    const int wib = threadIdx.x >> 5;
    constexpr int kChunks = kSliceLen / 32 / (kSliceThreads / 32);   // chunks per warp
    for (unsigned item = blockIdx.x; item < items; item += gridDim.x) {
        const Overflow& o = s.ovf[owner_of<&Overflow::slice_base>(s.ovf, n, item)];
        const uint32_t P = o.parts;
        const uint32_t q = item - o.slice_base;
        const int32_t v = o.v;
        const int64_t e_lo = o.st + (int64_t)q * kSliceLen;
        const int64_t e_hi = min(e_lo + (int64_t)kSliceLen, o.st + (int64_t)o.d);
        for (uint32_t b = threadIdx.x; b < P; b += blockDim.x) cnt[b] = 0;
        __syncthreads();
        int32_t glab[kChunks];
        T gsum[kChunks];
        uint32_t gb[kChunks];
#pragma unroll
        for (int u = 0; u < kChunks; ++u) {
            const int64_t e = e_lo + (int64_t)(wib + u * (kSliceThreads / 32)) * 32 + lane;
            const bool in = e < e_hi;
            const int32_t j = in ? load_index(s.idx, e) : v;
            const bool ok = in && j != v;
            const int32_t lab = ok ? load_label<ASYNC>(L.C, j) : kEmptyKey;
            T w = ok ? load_weight<WK>(s.w, e) : (T)0;
            bool lead = ok;
            if constexpr (WK != W_F32) {
                const unsigned peers = __match_any_sync(kFull, lab);
                if constexpr (WK == W_UNIT) w = (T)__popc(peers);
                else w = __reduce_add_sync(peers, w);
                lead = ok && lane == (unsigned)(__ffs(peers) - 1);
            }
            glab[u] = lead ? lab : kEmptyKey;
            gsum[u] = w;
            gb[u] = lead ? part_of(lab, P) : 0u;
            if (lead) atomicAdd(&cnt[gb[u]], 1u);
        }
        __syncthreads();
        // exclusive scan of cnt[0, P): each thread a run of consecutive partitions
        const uint32_t per = (P + blockDim.x - 1) / blockDim.x;
        const uint32_t b0 = min(P, threadIdx.x * per), b1 = min(P, b0 + per);
        unsigned long long mine[1] = {0}, ex[1], tot[1];
        for (uint32_t b = b0; b < b1; ++b) mine[0] += cnt[b];
        block_exclusive_scan<1>(mine, ex, tot);
        uint32_t r = (uint32_t)ex[0];
        for (uint32_t b = b0; b < b1; ++b) {
            off[b] = r;
            r += cnt[b];
        }
        __syncthreads();
        const int64_t cb = o.cnt_base + (int64_t)q * P;
        for (uint32_t b = threadIdx.x; b < P; b += blockDim.x) {
            s.ovf_cnt[cb + b] = cnt[b];
            s.ovf_off[cb + b] = off[b];
        }
        __syncthreads();
        for (uint32_t b = threadIdx.x; b < P; b += blockDim.x) cnt[b] = off[b];
        __syncthreads();
        const int64_t pb = o.pair_base + (int64_t)q * kSliceLen;
#pragma unroll
        for (int u = 0; u < kChunks; ++u) {
            if (glab[u] != kEmptyKey) {
                const uint32_t pos = atomicAdd(&cnt[gb[u]], 1u);
                s.ovf_pairs[pb + pos] = make_uint2((uint32_t)glab[u], sum_bits<WK>(gsum[u]));
            }
        }
        __syncthreads();
    }
}

// Folds a partition's winner (held by the thread whose candidate it is) into
// the row's 64-bit atomicMax of (sum key << 32 | ~tie key): larger sum first,
// then smaller tie key -- the smallest label when strict (Eq. 2; Section
// 4.1.5); the row's tie rule maps the key back to its label.  The block completing the row's
// last partition applies the result and marks the neighbours.  All threads
// of the block must call.
template <bool ASYNC, bool BATCH>
__device__ __forceinline__ void fold_partition(const DevState& s, const Labels& L, const BinView& bv, Overflow& o,
                                               const TieRule& tr, bool marks, uint32_t key, uint32_t tie,
                                               uint32_t part_best, unsigned long long& my_changed,
                                               unsigned long long& my_changed_entries) {
    __shared__ int resolver;
    __shared__ unsigned long long best_packed;
    const bool po = ASYNC && s.ctrl->prune_other != 0;               // FLPA's pruning rule
    if (threadIdx.x == 0) resolver = 0;
    __syncthreads();
    if (part_best != 0xffffffffu && key != 0 && tie == part_best) {
        const unsigned long long pk = ((unsigned long long)key << 32) | (unsigned long long)(~part_best);
        atomicMax(&o.best, pk);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned t = atomicAdd(&o.done, 1u);
        if (t == o.parts - 1) {
            __threadfence();
            best_packed = atomicAdd(&o.best, 0ull);
            resolver = 1;
        }
    }
    __syncthreads();
    if (resolver) {
        const unsigned long long bp = best_packed;
        const int32_t best_lab = (bp >> 32) ? tr.label(~(uint32_t)(bp & 0xffffffffull)) : -1;
        const int32_t own = o.own;
        const int32_t v = o.v;
        const bool changed = best_lab >= 0 && best_lab != own;
        if (threadIdx.x == 0) {
            record_label<ASYNC>(L, bv.chg + o.slot, v, own, best_lab, changed);
            if (changed) {
                ++my_changed;
                my_changed_entries += (unsigned long long)o.d;
                if constexpr (BATCH) atomicAdd(&s.dN[s.gid[v]], 1ull);
            }
        }
        if (changed && marks) mark_neighbours<ASYNC>(s, v, o.st, o.st + o.d, po, best_lab, L.C);
    }
    __syncthreads();
}

// Sliced path, step 2: a block per (row, partition p) reads partition p's run
// of every slice, aggregates it in the shared table and folds its winner.
template <bool ASYNC, int WK, bool BATCH, bool NS>
__global__ void __launch_bounds__(kSliceThreads, 2) k_ovf_parts(DevState s, int flag_neighbours) {
    using T = typename Acc<WK>::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int S = kLargeSlots;
    int32_t* keys = reinterpret_cast<int32_t*>(smem_raw);
    T* vals = reinterpret_cast<T*>(keys + S);
    uint32_t* qpre = reinterpret_cast<uint32_t*>(vals + S);      // [kMaxSlices + 1]
    uint32_t* qstart = qpre + kMaxSlices + 1;                    // [kMaxSlices]
    __shared__ uint32_t red_key[32];
    __shared__ uint32_t red_tie[32];
    __shared__ uint32_t winner;
    for (int q = threadIdx.x; q < S; q += blockDim.x) {
        keys[q] = kEmptyKey;
        vals[q] = (T)0;
    }
    __syncthreads();
    const unsigned n = (unsigned)s.ctrl->ovf_count;
    const unsigned items = s.ctrl->ovf_part_items;
    const BinView bv = bin_view(s, kBins - 1);
    const Labels L = labels_of(s);
    const bool marks = marks_on(s, flag_neighbours);
    const uint32_t sweep = NS ? (uint32_t)s.ctrl->iter + 1u : 0u;   // non-strict tie-break (Section 4.1.5)
    const int log_S = ceil_log2((unsigned)S);
    const unsigned lane = lane_id();
    const int wib = threadIdx.x >> 5, nw = blockDim.x >> 5;
    unsigned long long my_changed = 0, my_changed_entries = 0;
    for (unsigned item = blockIdx.x; item < items; item += gridDim.x) {
        Overflow& o = s.ovf[owner_of<&Overflow::part_base>(s.ovf, n, item)];
        const uint32_t P = o.parts, p = item - o.part_base, Q = o.slices;
        // partition p's run of every slice: its start (relative to the row's
        // pairs) and the prefix of run lengths, so the warps share all pairs
        for (uint32_t q0 = 0; q0 < Q; q0 += blockDim.x) {
            const uint32_t q = q0 + threadIdx.x;
            unsigned long long c[1] = {0}, ex[1], tot[1];
            if (q < Q) {
                const int64_t cb = o.cnt_base + (int64_t)q * P + p;
                c[0] = s.ovf_cnt[cb];
                qstart[q] = q * (uint32_t)kSliceLen + s.ovf_off[cb];
            }
            block_exclusive_scan<1>(c, ex, tot);
            const uint32_t carry = q0 ? qpre[q0] : 0u;
            if (q < Q) qpre[q] = carry + (uint32_t)ex[0];
            if (threadIdx.x == 0) qpre[min(q0 + blockDim.x, Q)] = carry + (uint32_t)tot[0];
            __syncthreads();
        }
        const uint32_t total = Q ? qpre[Q] : 0u;
        for (uint32_t f0 = (uint32_t)wib * 32; f0 < total; f0 += (uint32_t)nw * 32) {
            const uint32_t f = f0 + lane;
            const bool ok = f < total;
            int32_t lab = kEmptyKey;
            T w = (T)0;
            if (ok) {
                uint32_t lo = 0, hi = Q;                        // slice: largest q with qpre[q] <= f
                while (hi - lo > 1) {
                    const uint32_t mid = (lo + hi) >> 1;
                    if (qpre[mid] <= f) lo = mid;
                    else hi = mid;
                }
                const uint2 pr = s.ovf_pairs[o.pair_base + qstart[lo] + (f - qpre[lo])];
                lab = (int32_t)pr.x;
                w = sum_from_bits<WK>(pr.y);
            }
            bool lead = ok;
            if constexpr (WK != W_F32) {
                const unsigned peers = __match_any_sync(kFull, lab);
                w = __reduce_add_sync(peers, w);
                lead = ok && lane == (unsigned)(__ffs(peers) - 1);
            }
            if (lead && !table_add<T>(keys, vals, log_S, lab, w)) atomicExch(&s.ctrl->error, 4);
        }
        __syncthreads();
        const TieRule tr = tie_rule(s, NS, sweep, o.v);
        uint32_t key, tie;
        scan_table<T>(keys, vals, S, false, nullptr, 0u, nullptr, 0, tr, key, tie);     // the whole table
        const uint32_t part_best = block_argmax(key, tie, red_key, red_tie, &winner);
        fold_partition<ASYNC, BATCH>(s, L, bv, o, tr, marks, key, tie, part_best, my_changed, my_changed_entries);
    }
    flush_bin_counts(s, kBins - 1, my_changed, my_changed_entries);
}

// Rescan path (rows of fewer than kSliceMinParts or more than kMaxParts
// partitions, or beyond the scratch): a block per (row, partition p) scans the
// whole row keeping only the labels whose hash lands in partition p.
template <bool ASYNC, int WK, bool BATCH, bool NS>
__global__ void k_sweep_parts(DevState s, int flag_neighbours) {
    using T = typename Acc<WK>::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int S = kLargeSlots;
    int32_t* keys = reinterpret_cast<int32_t*>(smem_raw);
    T* vals = reinterpret_cast<T*>(keys + S);
    __shared__ uint32_t red_key[32];
    __shared__ uint32_t red_tie[32];
    __shared__ uint32_t winner;

    const unsigned lane = lane_id();
    const int wib = threadIdx.x >> 5;
    const int nw = blockDim.x >> 5;
    for (int q = threadIdx.x; q < S; q += blockDim.x) {
        keys[q] = kEmptyKey;
        vals[q] = (T)0;
    }
    __syncthreads();

    const unsigned n = (unsigned)s.ctrl->ovf_count;
    const unsigned items = s.ctrl->ovf_rescan_items;
    const BinView bv = bin_view(s, kBins - 1);
    const Labels L = labels_of(s);
    const bool marks = marks_on(s, flag_neighbours);
    const uint32_t sweep = NS ? (uint32_t)s.ctrl->iter + 1u : 0u;   // non-strict tie-break (Section 4.1.5)
    const int log_S = ceil_log2((unsigned)S);
    unsigned long long my_changed = 0, my_changed_entries = 0;
    for (unsigned item = blockIdx.x; item < items; item += gridDim.x) {
        Overflow& o = s.ovf[owner_of<&Overflow::rescan_base>(s.ovf, n, item)];
        const int32_t v = o.v;
        const int64_t st = o.st, en = o.st + o.d;
        const uint32_t parts = o.parts, p = item - o.rescan_base;
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
        const TieRule tr = tie_rule(s, NS, sweep, o.v);
        uint32_t key, tie;
        scan_table<T>(keys, vals, S, false, nullptr, 0u, nullptr, 0, tr, key, tie);     // the whole table
        const uint32_t part_best = block_argmax(key, tie, red_key, red_tie, &winner);
        fold_partition<ASYNC, BATCH>(s, L, bv, o, tr, marks, key, tie, part_best, my_changed, my_changed_entries);
    }
    flush_bin_counts(s, kBins - 1, my_changed, my_changed_entries);
}

// Scratch the sliced path may need: over last-bin rows longer than
// kLargeSlots / 2 (the only ones that can overflow) whose partition count
// qualifies for it, their entries (pairs) and Q x P (counts); and how many
// rows can overflow at all.
__global__ void k_ovf_capacity(DevState s, unsigned long long* out) {
    const int32_t* list = s.slist + s.bin_base[kBins - 1];
    const unsigned cnt = s.bin_static[kBins - 1];
    unsigned long long pairs = 0, counts = 0, rows = 0;
    for (unsigned k = blockIdx.x * blockDim.x + threadIdx.x; k < cnt; k += gridDim.x * blockDim.x) {
        const int32_t v = list[k];
        const int64_t d = s.off_end[v] - s.off[v];
        if (2 * d > kLargeSlots) {
            ++rows;
            const int64_t P = (2 * d + kLargeSlots - 1) / kLargeSlots;
            if (P >= kSliceMinParts && P <= kMaxParts && (d + kSliceLen - 1) / kSliceLen <= kMaxSlices) {
                pairs += (unsigned long long)d;
                counts += (unsigned long long)((d + kSliceLen - 1) / kSliceLen) * (unsigned long long)P;
            }
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        pairs += __shfl_xor_sync(kFull, pairs, o);
        counts += __shfl_xor_sync(kFull, counts, o);
        rows += __shfl_xor_sync(kFull, rows, o);
    }
    if (lane_id() == 0 && (pairs | counts | rows)) {
        atomicAdd(out, pairs);
        atomicAdd(out + 1, counts);
        atomicAdd(out + 2, rows);
    }
}

cudaError_t ovf_capacity(const DevState& s, cudaStream_t st, int sms, int64_t* pairs, int64_t* counts,
                         int64_t* rows, unsigned long long* scratch3) {
    cudaError_t e = cudaMemsetAsync(scratch3, 0, 3 * sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    if (s.bin_static[kBins - 1] > 0) {
        k_ovf_capacity<<<sms * 4, 256, 0, st>>>(s, scratch3);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    unsigned long long h[3];
    if ((e = cudaMemcpyAsync(h, scratch3, sizeof(h), cudaMemcpyDeviceToHost, st)) != cudaSuccess) return e;
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
    *pairs = (int64_t)h[0];
    *counts = (int64_t)h[1];
    *rows = (int64_t)h[2];
    return cudaSuccess;
}

template <bool ASYNC, int WK, bool BATCH, bool NS>
static cudaError_t launch_block_t(const DevState& s, int bin, int flag, int sms, cudaStream_t st) {
    // one resident wave: blocks stream the bin's rows (lpa_sweep_rows.cu)
    int blocks = sms;
    cudaError_t err = launch_rows<ASYNC, WK, BATCH, NS>(s, bin, flag, sms, st, &blocks);
    if (err != cudaSuccess || bin != kBins - 1 || !s.ovf_possible) return err;
    // overflowing rows: plan, sliced path (slices, then partitions), rescan path
    k_ovf_plan<<<1, 1024, 0, st>>>(s);
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
    const size_t tsmem = (size_t)kLargeSlots * 8;     // also the slices' 2 x kMaxParts counters
    auto k1 = k_ovf_slices<ASYNC, WK, BATCH>;
    if ((err = cudaFuncSetAttribute(k1, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tsmem)) != cudaSuccess)
        return err;
    k1<<<blocks, kSliceThreads, tsmem, st>>>(s);
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
    auto k3 = k_ovf_parts<ASYNC, WK, BATCH, NS>;
    const size_t psmem = tsmem + (size_t)(2 * kMaxSlices + 1) * sizeof(uint32_t);
    if ((err = cudaFuncSetAttribute(k3, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)psmem)) != cudaSuccess)
        return err;
    k3<<<blocks, kSliceThreads, psmem, st>>>(s, flag);
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
    auto pk = k_sweep_parts<ASYNC, WK, BATCH, NS>;
    if ((err = cudaFuncSetAttribute(pk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tsmem)) != cudaSuccess)
        return err;
    pk<<<blocks, kBlockThreads[kBlockBins - 1], tsmem, st>>>(s, flag);
    return cudaGetLastError();
}

template <bool ASYNC, bool BATCH, bool NS>
static cudaError_t launch_block_w(const DevState& s, int bin, int flag, int sms, cudaStream_t st) {
    switch (s.weight_kind) {
        case W_UNIT: return launch_block_t<ASYNC, W_UNIT, BATCH, NS>(s, bin, flag, sms, st);
        case W_U32: return launch_block_t<ASYNC, W_U32, BATCH, NS>(s, bin, flag, sms, st);
        case W_U8: return launch_block_t<ASYNC, W_U8, BATCH, NS>(s, bin, flag, sms, st);
        default: return launch_block_t<ASYNC, W_F32, BATCH, NS>(s, bin, flag, sms, st);
    }
}

template <bool NS>
static cudaError_t launch_block_ns(const DevState& s, bool async, int bin, int flag, int sms, cudaStream_t st) {
    const bool batch = s.G > 1;
    if (async)
        return batch ? launch_block_w<true, true, NS>(s, bin, flag, sms, st)
                     : launch_block_w<true, false, NS>(s, bin, flag, sms, st);
    return batch ? launch_block_w<false, true, NS>(s, bin, flag, sms, st)
                 : launch_block_w<false, false, NS>(s, bin, flag, sms, st);
}

cudaError_t launch_sweep_block(const DevState& s, int mode, int bin, int sms, cudaStream_t st) {
    const bool ns = (mode & kModeNonstrict) != 0;
    mode &= ~kModeNonstrict;
    const bool async = mode == MODE_ASYNC;
    const int flag = mode != MODE_SYNC_FULL;
    return ns ? launch_block_ns<true>(s, async, bin, flag, sms, st)
              : launch_block_ns<false>(s, async, bin, flag, sms, st);
}

}  // namespace lpa
