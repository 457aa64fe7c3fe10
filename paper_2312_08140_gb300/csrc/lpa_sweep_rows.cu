// lpa_sweep_rows.cu -- sweep for vertices with degree above warp_max: one
// thread block per frontier row (128 threads up to mid_max, 256 up to
// large_max, 512 above), rows streamed through a block-wide pipeline.
//
// Per row the work is Eq. 2 (Section 3.3): gather the label of every
// neighbour, sum the weights per label, take the most weighted label (ties:
// Section 4.1.5) and, on change, mark the neighbours unprocessed (Section
// 4.1.4).  The gathers are random 4-byte reads, so the kernel is bound by how
// many of them are in flight.  It keeps them in flight across the whole pass:
//
//   * a row is cut into tiles of TILE = NC x P entries, NC the aggregating
//     threads.  One warp produces the tile sequence of the block (rows taken
//     from a per-bin counter in batches of 32, their metadata loaded by the
//     32 lanes in parallel) up to kStages tiles ahead, and copies each tile's
//     neighbour ids into one of kStages shared-memory buffers with one bulk
//     asynchronous copy (cp.async.bulk, completion counted on an mbarrier).
//     In the 256- and 512-thread kernels the last warp only produces: it
//     refills a buffer once the other warps have signalled (a second
//     mbarrier per buffer) that they read it, and those warps synchronise on
//     a named barrier of their own, so the producer's work never holds up a
//     step.  In the 128-thread kernel warp 0 produces between its own
//     aggregation steps;
//   * in step k every thread reads its P ids of tile k+1 from shared memory
//     and issues their label gathers into registers, then aggregates tile k
//     (whose labels arrived during step k-1): lanes holding the same label
//     are grouped with __match_any_sync and the group leader adds the group's
//     weight into a shared-memory open-addressing table, listing the slots it
//     fills;
//   * after a row's last tile each warp scans the slots it listed and
//     reduces (sum, tie key) to its candidate, a shared 64-bit maximum gives
//     the block's winner, which is recorded, and the neighbours are marked.
//     The next row's gathers are already in flight at that point.
//
// Rows whose distinct labels overflow the last bin's table (bounded probing
// fails) are appended to the overflow list and finished by the partitioned
// kernels of lpa_sweep_block.cu.  The first synchronous sweep of a
// repeat-free graph, and the last bin of the first asynchronous sweep, take
// the max-over-row pass instead (every label is still its vertex's id): no
// gathers, so each warp streams whole rows with 16-byte loads and reduces
// them to the max of (weight key, tie key); under the strict tie-break the
// tie key is the entry's position (rows list their neighbours in increasing
// caller id), and with unit weights the pick is the row's first entry other
// than the vertex itself.
//
// Every wait on an mbarrier is bounded (2 s of GPU time); a wait that gives
// up sets error code 5 in the control block and the abort flag, the
// aggregating warps leave together at their next barrier, and the producing
// warp leaves after its copies in flight have landed (again waited for with
// a bound).  lpa_graph_debug_stall makes one copy go missing, to test this.
#include "lpa_device.cuh"

namespace lpa {

constexpr int kRowBatch = 32;                  // rows taken from the counter at a time
constexpr int kStages = 4;                     // index buffers: a tile's copy starts three steps ahead
constexpr int kSharedProbes = 16;              // probe bound of rows that may overflow the table
constexpr unsigned long long kWaitNs = 2000000000ull;

// ---- PTX wrappers: mbarrier and bulk asynchronous copy --------------------
__device__ __forceinline__ unsigned smem_u32(const void* p) {
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Orders this thread's earlier generic-proxy accesses of shared memory before
// later async-proxy (bulk copy) writes to it.
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// dst (shared, 16-byte aligned) <- src (global, 16-byte aligned), bytes a
// multiple of 16; completion adds `bytes` to the mbarrier's transaction count.
// The row indices are read once per sweep: L2 evict-first.
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
    const uint64_t pol = l2_policy_evict_first();
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], "
        "%4;" ::"r"(smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(pol)
        : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Named barrier 1 over the first `count` threads of the block (a multiple
// of 32): the consumer warps of the row kernels with a producer warp.
__device__ __forceinline__ void named_sync(unsigned count) {
    asm volatile("bar.sync 1, %0;" ::"r"(count) : "memory");
}

__device__ __forceinline__ int named_sync_or(unsigned count, bool pred) {
    unsigned r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 p, %1, 0;\n\t"
        "bar.red.or.pred q, 1, %2, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"((unsigned)pred), "r"(count)
        : "memory");
    return (int)r;
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Waits until phase `parity` of the mbarrier has completed, for at most
// kWaitNs.  Returns false if it gave up.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    for (unsigned polls = 1;; ++polls) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((polls & 63u) == 0 && global_ns() - t0 > kWaitNs) return false;
    }
}

// The same wait, also giving up once *stop is set.
__device__ __forceinline__ bool mbar_wait_bounded_or(uint64_t* bar, unsigned parity, const volatile int* stop) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    for (unsigned polls = 1;; ++polls) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((polls & 63u) == 0 && (*stop || global_ns() - t0 > kWaitNs)) return false;
    }
}

// Entries [e, e + 4) of idx (e a multiple of 4, e < en; idx starts at a
// 16-byte aligned address): one 16-byte load where the vector lies inside the
// row [st, en), else entry by entry; entries outside the row read as `fill`.
__device__ __forceinline__ void load_idx4(const int32_t* idx, int64_t e, int64_t st, int64_t en, int32_t fill,
                                          int32_t (&j)[4]) {
    if (e >= st && e + 4 <= en) {
        const int4 x = __ldg(reinterpret_cast<const int4*>(idx + e));
        j[0] = x.x;
        j[1] = x.y;
        j[2] = x.z;
        j[3] = x.w;
    } else {
        // the first or last vector of the row
#pragma unroll
        for (int c = 0; c < 4; ++c) j[c] = (e + c >= st && e + c < en) ? __ldg(idx + e + c) : fill;
    }
}

// Marks the neighbours of changed vertex v unprocessed (Section 4.1.4): the
// GROUP threads of rank 0..GROUP-1 walk row [st, en) in 4-entry vectors,
// VEC vectors per thread in flight (their ids, then their flags, then the
// stores).  FLPA's rule (po) leaves a neighbour already carrying `best`.
template <bool ASYNC, int GROUP, int VEC>
__device__ __forceinline__ void mark_row(const DevState& s, const Labels& L, int64_t st, int64_t en, int32_t v,
                                         unsigned rank, bool po, int32_t best) {
    for (int64_t e0 = (st & ~(int64_t)3) + 4 * (int64_t)rank; e0 < en; e0 += 4 * GROUP * VEC) {
        int32_t j[VEC][4];
        uint8_t f[VEC][4];
#pragma unroll
        for (int u = 0; u < VEC; ++u) {
            const int64_t e = e0 + 4 * GROUP * u;
            if (e < en) {
                load_idx4(s.idx, e, st, en, v, j[u]);
            } else {
#pragma unroll
                for (int c = 0; c < 4; ++c) j[u][c] = v;
            }
        }
#pragma unroll
        for (int u = 0; u < VEC; ++u)
#pragma unroll
            for (int c = 0; c < 4; ++c) f[u][c] = j[u][c] != v ? __ldcg(s.flags + j[u][c]) : (uint8_t)1;
#pragma unroll
        for (int u = 0; u < VEC; ++u)
#pragma unroll
            for (int c = 0; c < 4; ++c)
                if (f[u][c] == 0 && !(po && load_label<ASYNC>(L.C, j[u][c]) == best)) s.flags[j[u][c]] = 1;
    }
}

// ---- per-block shared state -----------------------------------------------
// One tile: entries [e0, e1) of one row.  Written by warp 0 kStages steps
// before it is aggregated.
struct Tile {
    int64_t e0, e1;        // entry range of the tile
    int64_t a0;            // first entry held by the tile's buffer (e0 rounded down to 4)
    int64_t st, en;        // the row
    int32_t v;             // vertex (-1: no tile, the pass is over for this block)
    int32_t own;           // its label before the sweep
    uint32_t k;            // its slot in the bin's frontier list
    int32_t last;          // last tile of the row
    int32_t skip;          // batches: the vertex's graph is done; the row is left as it is
    int32_t pad;
};

// Entries per thread per tile, tiles of gathers in flight ahead of the one
// being aggregated, entries per tile, and one index buffer.  The unit-weight
// kernels of the wider blocks keep 8 gathers per thread in flight (1 block of
// 512 or 2 of 256 threads per SM, no register spills); a second tile of
// gathers in flight (LA = 2) measured no faster on R-MAT 27.
template <int NT, int WK>
struct RowsShape {
    static constexpr bool SPEC = NT >= 256;        // the last warp only produces tiles
    static constexpr int NC = SPEC ? NT - 32 : NT; // threads that aggregate
    static constexpr int P = (NT >= 256 && WK == W_UNIT) ? 8 : 4;
    static constexpr int LA = 1;                   // tiles whose gathers run ahead of the aggregated one
    static constexpr int TILE = NC * P;
    static constexpr int BUF = TILE + 8;       // + up to 3 entries of alignment slack on each side
};

// Blocks of NT threads the launch bounds ask to fit on one SM (registers per
// thread follow from it).  Measured on R-MAT 27: one 512-thread block per SM
// for the last bin and two 256-thread blocks for the bin before it ran the
// run in 107 ms; two and four blocks (64 registers, 4 gathers per thread)
// took 154 ms, and with 8 gathers per thread (spilling) 136 ms.
template <int NT>
struct RowsOccupancy {
    static constexpr int kBlocks = NT >= 512 ? 1 : NT >= 256 ? 2 : 8;
};

// Metadata of one row of the current batch.
struct RowMeta {
    int64_t st, en;        // the row
    int32_t v;             // vertex (-1: past the end of the bin)
    int32_t own;           // its label before the sweep
    int32_t skip;          // batches: the vertex's graph is done
    uint32_t k;            // its slot in the bin's frontier list
};

// Production cursor of warp 0.
struct ProdState {
    int64_t pe, pen;       // next entry of the row being cut into tiles, and its end
    int32_t bpos;          // next row of the batch
    int32_t prow;          // the row being cut into tiles
    int32_t exhausted;     // no rows left for this block
    int32_t pad;
};

template <bool ASYNC, int WK, bool BATCH, bool NS, int NT>
__global__ void __launch_bounds__(NT, RowsOccupancy<NT>::kBlocks) k_sweep_rows(DevState s, int bin,
                                                                            int flag_neighbours) {
    using T = typename Acc<WK>::T;
    using Sh = RowsShape<NT, WK>;
    constexpr int P = Sh::P;
    constexpr int NW = NT / 32;
    constexpr bool SPEC = Sh::SPEC;            // the last warp produces, the others aggregate
    constexpr int NC = Sh::NC;                 // aggregating threads
    constexpr int NWC = NC / 32;
    constexpr int PW = SPEC ? NW - 1 : 0;      // the producing warp
    extern __shared__ __align__(16) unsigned char smem_raw[];
    // layout: kStages index buffers | table keys | table values | filled-slot lists
    int32_t* ibuf = reinterpret_cast<int32_t*>(smem_raw);                   // [kStages][BUF]
    const int S = s.block_slots[bin - 2];
    int32_t* keys = ibuf + kStages * Sh::BUF;
    T* vals = reinterpret_cast<T*>(keys + S);
    const unsigned seg_cap = (unsigned)S / 2u / NWC;
    uint16_t* segs = reinterpret_cast<uint16_t*>(vals + S);
    __shared__ __align__(8) uint64_t mbar[kStages];        // full: a tile's indices (and descriptor) landed
    __shared__ __align__(8) uint64_t mbar_empty[kStages];  // producer warp only: a buffer was read
    __shared__ Tile tiles[2 * kStages];
    __shared__ RowMeta batch[kRowBatch];
    __shared__ ProdState prod;
    __shared__ unsigned long long row_best[2];     // packed winner of the current row (rows alternate)
    __shared__ int overflow, abort_flag;

    const unsigned lane = lane_id();
    const int wib = threadIdx.x >> 5;
    uint16_t* my_seg = segs + (size_t)(wib < NWC ? wib : 0) * seg_cap;
    unsigned wfill = 0;
    unsigned rb = 0;                                // row_best slot of the current row
    for (int q = threadIdx.x; q < S; q += NT) {
        keys[q] = kEmptyKey;
        vals[q] = (T)0;
    }
    if (threadIdx.x == 0) {
        for (int b = 0; b < kStages; ++b) {
            mbar_init(&mbar[b], 1);
            mbar_init(&mbar_empty[b], 1);
        }
        fence_mbar_init();
        overflow = 0;
        abort_flag = 0;
        row_best[0] = row_best[1] = 0ull;
        prod.pe = prod.pen = 0;
        prod.bpos = kRowBatch;
        prod.prow = -1;
        prod.exhausted = 0;
    }

    const BinView bv = bin_view(s, bin);
    const Labels L = labels_of(s);
    const bool marks = marks_on(s, flag_neighbours);
    const uint32_t sweep = NS ? (uint32_t)s.ctrl->iter + 1u : 0u;   // non-strict tie-break (Section 4.1.5)
    bool ident = identity_sweep<ASYNC, BATCH>(s);
    if constexpr (ASYNC && !BATCH) ident = bin == kBins - 1 && s.rows_distinct && s.ctrl->iter == 0 && L.dense;
    const bool po = ASYNC && s.ctrl->prune_other != 0;               // FLPA's pruning rule
    const int log_S = ceil_log2((unsigned)S);
    const unsigned cnt = bv.cnt;
    const int64_t E_al = s.E & ~(int64_t)3;                          // end of the 16-byte aligned part of idx

    if (ident) {
        // ---- max-over-row pass: every label is still its vertex's id, so each
        // row's pick is the max of (weight key, tie key) over its entries.  No
        // gathers to hide, so no tiles: each warp takes whole rows from the
        // bin's counter (the largest first, as the list holds them) and
        // streams them with 16-byte loads, kIdentVec per lane in flight;
        // NW rows per block are in flight at once and no block barrier runs.
        constexpr int kIdentVec = NT >= 256 ? 4 : 2;    // 4-entry index vectors per lane in flight
        unsigned long long n_changed = 0, n_changed_entries = 0;
        unsigned k = 0;
        if (lane == 0) k = atomicAdd(&s.ctrl->row_next[bin], 1u);
        k = __shfl_sync(kFull, k, 0);
        while (k < cnt) {
            // the warp's next row is claimed now and read after this one
            unsigned k_next = 0;
            if (lane == 0) k_next = atomicAdd(&s.ctrl->row_next[bin], 1u);
            const int32_t v = bv.list[k];
            const int64_t st = s.off[v], en = s.off_end[v];
            const int32_t own = ASYNC ? __ldcg(L.C + v) : L.C[v];
            int32_t best_lab = -1;
            if constexpr (!NS && WK == W_UNIT) {
                // strict tie-break, unit weights: every label's sum is 1, so
                // the pick is the smallest neighbour id; the row lists its
                // neighbours in increasing caller id (the storage orders keep
                // each row's entry order), so it is the first entry other
                // than v itself
                for (int64_t e0 = st; e0 < en; e0 += 32) {
                    const int64_t e = e0 + lane;
                    const int32_t j = e < en ? __ldg(s.idx + e) : v;
                    const unsigned okm = __ballot_sync(kFull, j != v);
                    if (okm != 0u) {
                        best_lab = initial_label(s, __shfl_sync(kFull, j, __ffs(okm) - 1));
                        break;
                    }
                }
            } else {
                // max of (weight key, tie key); with the strict tie-break the
                // tie key is the entry's position in the row (positions
                // increase with the caller's neighbour ids), so no label is
                // read but the winner's
                const TieRule tr = tie_rule(s, NS, sweep, v);
                unsigned long long bp = 0ull;
                for (int64_t e0 = (st & ~(int64_t)3) + 4 * (int64_t)lane; e0 < en; e0 += 128 * kIdentVec) {
                    int32_t jj[kIdentVec][4];
                    T ww[kIdentVec][4];
#pragma unroll
                    for (int u = 0; u < kIdentVec; ++u) {
                        const int64_t e = e0 + 128 * u;
                        if (e < en) {
                            load_idx4(s.idx, e, st, en, v, jj[u]);
                        } else {
#pragma unroll
                            for (int c = 0; c < 4; ++c) jj[u][c] = v;
                        }
#pragma unroll
                        for (int c = 0; c < 4; ++c) {
                            if constexpr (WK == W_UNIT) ww[u][c] = (T)1;
                            else ww[u][c] = jj[u][c] != v ? load_weight<WK>(s.w, e + c) : (T)0;
                        }
                    }
#pragma unroll
                    for (int u = 0; u < kIdentVec; ++u)
#pragma unroll
                        for (int c = 0; c < 4; ++c) {
                            if (jj[u][c] != v) {
                                const uint32_t tie = NS ? tr.key(initial_label(s, jj[u][c]))
                                                        : (uint32_t)(e0 + 128 * u + c - st);
                                const unsigned long long cc = pack_candidate(sum_key(ww[u][c]), tie);
                                bp = cc > bp ? cc : bp;
                            }
                        }
                }
                bp = warp_max_u64(bp);
                if (bp != 0ull) {
                    const uint32_t tie = ~(uint32_t)bp;
                    best_lab = NS ? tr.label(tie) : initial_label(s, __ldg(s.idx + st + tie));
                }
            }
            const bool changed = best_lab >= 0 && best_lab != own;   // warp-uniform
            if (lane == 0) record_label<ASYNC>(L, bv.chg + k, v, own, best_lab, changed);
            if (changed) {
                if (lane == 0) {
                    ++n_changed;
                    n_changed_entries += (unsigned long long)(en - st);
                }
                if (marks) mark_row<ASYNC, 32, (NT >= 256 ? 2 : 1)>(s, L, st, en, v, lane, po, best_lab);
            }
            k = __shfl_sync(kFull, k_next, 0);
        }
        flush_bin_counts(s, bin, n_changed, n_changed_entries);
        return;
    }

    // ---- producer (warp 0) -----------------------------------------------------
    // Rows come from the bin's counter in batches of kRowBatch.  The list
    // entries of the next batch (nxt_v, one per lane) and the counter value of
    // the one after (nn_base, lane 0) are fetched a batch ahead; when a batch
    // starts, its rows' offsets and labels are loaded into `batch`.
    int32_t nxt_v = -1;
    unsigned nxt_base = 0, nn_base = 0;
    unsigned produced = 0;          // tiles produced by this block (index of the next one)

    auto list_at = [&](unsigned base) -> int32_t {
        const unsigned k = base + lane;
        return (base < cnt && k < cnt) ? bv.list[k] : -1;
    };
    auto start_batch = [&]() {      // warp 0: the batch at nxt_base becomes current
        RowMeta m;
        m.v = nxt_v;
        m.k = nxt_base + lane;
        m.st = m.en = 0;
        m.own = 0;
        m.skip = 0;
        if (m.v >= 0) {
            m.st = s.off[m.v];
            m.en = s.off_end[m.v];
            m.own = ASYNC ? __ldcg(L.C + m.v) : L.C[m.v];
            if constexpr (BATCH) m.skip = s.done[s.gid[m.v]] ? 1 : 0;
        }
        batch[lane] = m;
        nxt_base = __shfl_sync(kFull, nn_base, 0);
        nxt_v = list_at(nxt_base);
        if (lane == 0) nn_base = atomicAdd(&s.ctrl->row_next[bin], (unsigned)kRowBatch);
        __syncwarp();
        if (lane == 0) {
            prod.bpos = 0;
            if (batch[0].v < 0) prod.exhausted = 1;
        }
        __syncwarp();
    };
    // The producing warp: writes the descriptor of the next tile into
    // tiles[produced % 8] and starts its copy into buffer produced % kStages.
    // All 32 lanes call.
    auto produce = [&]() {
        for (;;) {                                     // warp-uniform: every lane reads the same state
            if (prod.exhausted || prod.pe < prod.pen) break;
            if (prod.bpos >= kRowBatch) {
                start_batch();
                if (prod.exhausted) break;
            }
            if (lane == 0) {
                const RowMeta& r = batch[prod.bpos];
                if (r.v < 0) {
                    prod.exhausted = 1;
                } else {
                    prod.prow = prod.bpos;
                    prod.pe = r.st;
                    prod.pen = r.en;
                }
                ++prod.bpos;
            }
            __syncwarp();
        }
        if (lane == 0) {
            Tile t;
            t.v = -1;
            const int b = (int)(produced % kStages);
            if (!prod.exhausted) {
                const RowMeta& r = batch[prod.prow];
                t.v = r.v;
                t.own = r.own;
                t.skip = r.skip;
                t.k = r.k;
                t.st = r.st;
                t.en = r.en;
                t.e0 = prod.pe;
                t.e1 = min(prod.pe + (int64_t)Sh::TILE, prod.pen);
                t.last = t.e1 >= prod.pen ? 1 : 0;
                t.a0 = t.e0 & ~(int64_t)3;
                prod.pe = t.e1;
            }
            tiles[produced % (2 * kStages)] = t;
            // test hook: the first block of the kernel named by
            // ctrl->stall_copy to produce a tile leaves that tile's copy
            // unissued (once), so the waits on it run out
            const bool stall = t.v >= 0 && produced == 0 && s.ctrl->stall_copy == NT &&
                               atomicCAS(&s.ctrl->stall_copy, NT, 0) == NT;
            if (stall) {
                // neither the copy nor the arrival that would complete it
            } else if (t.v >= 0) {
                int64_t a1 = (t.e1 + 3) & ~(int64_t)3;
                if (a1 > E_al) a1 = E_al;
                const int64_t bytes = a1 > t.a0 ? (a1 - t.a0) * 4 : 0;
                int32_t* dst = ibuf + b * Sh::BUF;
                // entries past the aligned end of idx (at most 3, at the end of
                // the array) are copied with plain loads
                for (int64_t e = a1 > t.a0 ? a1 : t.a0; e < t.e1; ++e) dst[e - t.a0] = s.idx[e];
                fence_proxy_async_smem();
                mbar_arrive_expect_tx(&mbar[b], (unsigned)bytes);
                if (bytes > 0) bulk_copy_g2s(dst, s.idx + t.a0, (unsigned)bytes, &mbar[b]);
            } else if (SPEC) {
                mbar_arrive(&mbar[b]);                 // the end of the sequence, for the waiting consumers
            }
        }
        ++produced;
        __syncwarp();
    };

    if (wib == PW) {
        unsigned b0 = 0;
        if (lane == 0) b0 = atomicAdd(&s.ctrl->row_next[bin], (unsigned)kRowBatch);
        nxt_base = __shfl_sync(kFull, b0, 0);
        nxt_v = list_at(nxt_base);
        if (lane == 0) nn_base = atomicAdd(&s.ctrl->row_next[bin], (unsigned)kRowBatch);
    }
    __syncthreads();                                   // mbarriers initialised, table clear
    __shared__ unsigned long long blk_changed, blk_changed_entries;   // this block's changes (thread 0)
    if (threadIdx.x == 0) blk_changed = blk_changed_entries = 0ull;
    if constexpr (!SPEC) {
        if (wib == 0) {
            for (int q = 0; q < kStages; ++q) produce();
        }
        __syncthreads();
    } else if (wib == PW) {
        // ---- the producing warp: tile t goes into buffer t % kStages once the
        // aggregating warps have read tile t - kStages from it (mbar_empty),
        // up to and including the end of the sequence (v = -1)
        for (unsigned t = 0;; ++t) {
            const unsigned b = t % kStages;
            if (t >= kStages) {
                bool ok = true;
                if (lane == 0) ok = mbar_wait_bounded_or(&mbar_empty[b], ((t / kStages) - 1u) & 1u, &abort_flag);
                ok = __shfl_sync(kFull, ok, 0) != 0;
                if (!ok) {
                    if (lane == 0 && !abort_flag) {
                        atomicExch(&s.ctrl->error, 5);
                        abort_flag = 1;
                    }
                    break;
                }
            }
            produce();
            if (tiles[t % (2 * kStages)].v < 0) break;
        }
        // after an abort, let the copies still in flight land before the
        // block can leave
        if (lane == 0 && abort_flag)
            for (unsigned q = produced >= kStages ? produced - kStages : 0; q < produced; ++q)
                if (tiles[q % (2 * kStages)].v >= 0) (void)mbar_wait_bounded(&mbar[q % kStages], (q / kStages) & 1u);
    }
    if (!(SPEC && wib == PW)) {

    // ---- consumer state ------------------------------------------------------
    // lab_q[0]: the tile being aggregated; lab_q[1..LA]: the next LA tiles,
    // whose gathers are in flight
    constexpr int LA = Sh::LA;
    int32_t lab_q[LA + 1][P];
    T w_q[LA + 1][P];
    int32_t (&lab_cur)[P] = lab_q[0];
    T (&w_cur)[P] = w_q[0];

    // Waits for tile t (buffer t % kStages, phase (t / kStages) & 1; with a
    // producing warp, its descriptor lands with it), then reads the tile's
    // ids and issues their gathers.  Returns false if the wait gave up.
    auto load_tile = [&](unsigned t_idx, int32_t (&lab)[P], T (&w)[P]) -> bool {
        const int b = (int)(t_idx % kStages);
        const Tile& t = tiles[t_idx % (2 * kStages)];
        if (!SPEC && t.v < 0) return true;               // no copy: nothing to wait for
        if (!mbar_wait_bounded(&mbar[b], (t_idx / kStages) & 1u)) return false;
        if (t.v < 0) return true;
        const int64_t e0 = t.e0;
        const int32_t n = (int32_t)(t.e1 - e0);
        const int32_t* src = ibuf + b * Sh::BUF + (int32_t)(e0 - t.a0);
        const int32_t v = t.v;
        const bool on = !t.skip;
#pragma unroll
        for (int p = 0; p < P; ++p) {
            const int r = p * NC + (int)threadIdx.x;
            const bool in = on && r < n;
            const int32_t j = in ? src[r] : v;
            const bool ok = in && j != v;
            lab[p] = ok ? load_label<ASYNC>(L.C, j) : kEmptyKey;
            if constexpr (WK == W_UNIT) w[p] = ok ? (T)1 : (T)0;
            else w[p] = ok ? load_weight<WK>(s.w, e0 + r) : (T)0;
        }
        return true;
    };

    bool alive = true;
#pragma unroll
    for (int a = 0; a < LA; ++a) {
        if (!load_tile((unsigned)a, lab_q[a], w_q[a])) {
            atomicExch(&s.ctrl->error, 5);
            abort_flag = 1;
        }
    }

    for (unsigned k = 0;; ++k) {
        // step k-1 done: buffer k % kStages is free
        int stop;
        if constexpr (SPEC) {
            stop = named_sync_or(NC, abort_flag != 0);   // the producer may set the flag at any time
            if (threadIdx.x == 0) mbar_arrive(&mbar_empty[k % kStages]);
        } else {
            __syncthreads();
            stop = abort_flag;
        }
        if (stop) {
            alive = false;
            break;
        }
        const Tile& tk = tiles[k % (2 * kStages)];
        if (tk.v < 0) break;
        if (!SPEC && wib == 0) produce();              // tile k + kStages into buffer k % kStages
        if (!load_tile(k + LA, lab_q[LA], w_q[LA])) {
            atomicExch(&s.ctrl->error, 5);
            abort_flag = 1;
        }

        // aggregate tile k into the table (its descriptor read once)
        const int32_t v = tk.v;
        const int32_t k_n = (int32_t)(tk.e1 - tk.e0);
        const bool k_skip = tk.skip != 0;
        const int64_t d = tk.en - tk.st;
        const int log_full = ceil_log2((unsigned)(2 * d < ((int64_t)1 << 30) ? 2 * d : ((int64_t)1 << 30)));
        const bool fits = log_full <= log_S;
        const int log_s = fits ? log_full : log_S;
        // one (label, weight) into the table; returns the slot it filled, or -1
        auto insert = [&](int32_t label, T wsum) -> int {
            int created = -1;
            if (fits) {
                if (!table_insert<T>(keys, vals, log_s, label, wsum, 1u << log_s, created))
                    atomicExch(&s.ctrl->error, 3);
            } else if (!overflow && !table_insert<T>(keys, vals, log_s, label, wsum, kSharedProbes, created)) {
                overflow = 1;
            }
            return created;
        };
        auto list_created = [&](int created) {
            const unsigned nm = __ballot_sync(kFull, created >= 0);
            if (created >= 0) {
                const unsigned pos = wfill + __popc(nm & lanes_below());
                if (pos < seg_cap) my_seg[pos] = (uint16_t)created;
            }
            wfill += __popc(nm);
        };
        if (!k_skip && (int)(wib * 32) < k_n) {
            // Fast path: every entry this warp holds in the tile carries one
            // label (after the first sweeps nearly every neighbour of a hub
            // does) -- one reduction and one insert for the warp's share.
            int32_t mine = kEmptyKey;
            bool uni = true;
            T tw = (T)0;
#pragma unroll
            for (int p = 0; p < P; ++p) {
                if (lab_cur[p] != kEmptyKey) {
                    uni = uni && (mine == kEmptyKey || mine == lab_cur[p]);
                    mine = lab_cur[p];
                    tw += w_cur[p];
                }
            }
            const int32_t wl = __reduce_max_sync(kFull, mine);
            if (__all_sync(kFull, uni && (mine == kEmptyKey || mine == wl))) {
                if (wl != kEmptyKey) {
                    T tot;
                    if constexpr (WK == W_F32) {
                        tot = tw;
                        for (int o = 16; o > 0; o >>= 1) tot += __shfl_xor_sync(kFull, tot, o);
                    } else {
                        tot = __reduce_add_sync(kFull, tw);
                    }
                    list_created(lane == 0 ? insert(wl, tot) : -1);
                }
            } else {
#pragma unroll
                for (int p = 0; p < P; ++p) {
                    if (p * NC + (int)(wib * 32) >= k_n) break;       // warp-uniform
                    const bool ok = lab_cur[p] != kEmptyKey;
                    T wsum = w_cur[p];
                    bool lead = ok;
                    if constexpr (WK != W_F32) {
                        const unsigned peers = __match_any_sync(kFull, lab_cur[p]);
                        if constexpr (WK == W_UNIT) {
                            wsum = (T)__popc(peers);
                        } else {
                            wsum = __reduce_add_sync(peers, wsum);
                        }
                        lead = ok && lane == (unsigned)(__ffs(peers) - 1);
                    }
                    list_created(lead ? insert(lab_cur[p], wsum) : -1);
                }
            }
        }

        if (tk.last) {
            // ---- the row is complete: pick, record, mark --------------------
            const TieRule tr = tie_rule(s, NS, sweep, v);
            int32_t best_lab = -1;
            int ovf = 0;
            if (tk.skip) {
                // a done graph's vertex keeps its label (batches)
            } else {
                // two barriers per row.  The first completes the table and the
                // slot lists, and tells every thread whether some warp's list
                // overflowed (then the whole table is scanned).  Each warp
                // scans the slots it created, reduces its candidates, and its
                // lane 0 folds (sum key, ~tie key) into one packed 64-bit
                // shared maximum; after the second barrier every thread reads
                // the winner.  The two maxima alternate between rows, so the
                // one for the next row is cleared here.
                int full_scan;
                if constexpr (SPEC) full_scan = named_sync_or(NC, wfill > seg_cap);
                else full_scan = __syncthreads_or(wfill > seg_cap);
                ovf = overflow;
                // this thread's best candidate among the row's slots; clears them
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
                if (!full_scan) {
                    for (unsigned f = lane; f < wfill; f += 32) visit(my_seg[f]);
                } else {
                    for (int q = threadIdx.x; q < (1 << log_s); q += NC) visit(q);
                }
                wfill = 0;
                const uint32_t key = any ? sum_key(best_w) : 0u;
                const uint32_t m = __reduce_max_sync(kFull, key);
                const uint32_t c = __reduce_min_sync(kFull, (m != 0 && key == m) ? best_k : 0xffffffffu);
                if (lane == 0 && m != 0u) atomicMax(&row_best[rb], pack_candidate(m, c));
                if constexpr (SPEC) named_sync(NC);
                else __syncthreads();
                const unsigned long long bp = row_best[rb];
                if (threadIdx.x == 0) row_best[rb ^ 1] = 0ull;
                rb ^= 1;
                best_lab = bp == 0ull ? -1 : tr.label(~(uint32_t)bp);
            }
            if (ovf) {
                // hand the row to the partitioned kernels (last bin only)
                if (threadIdx.x == 0) {
                    Overflow& o = s.ovf[atomicAdd(&s.ctrl->ovf_count, 1ull)];
                    o.v = v;
                    o.slot = tk.k;
                    o.st = tk.st;
                    o.d = (int32_t)d;
                    o.own = tk.own;
                    o.parts = (uint32_t)((2 * d + S - 1) / S);
                    o.best = 0ull;
                    o.done = 0u;
                    overflow = 0;
                }
            } else {
                const bool changed = best_lab >= 0 && best_lab != tk.own;     // block-uniform
                if (threadIdx.x == 0) record_label<ASYNC>(L, bv.chg + tk.k, v, tk.own, tk.skip ? tk.own : best_lab,
                                                          changed);
                if (changed) {
                    if (threadIdx.x == 0) {
                        ++blk_changed;
                        blk_changed_entries += (unsigned long long)d;
                        if constexpr (BATCH) atomicAdd(&s.dN[s.gid[v]], 1ull);
                    }
                    if (marks) mark_row<ASYNC, NC, (NT >= 256 ? 2 : 1)>(s, L, tk.st, tk.en, v, threadIdx.x, po, best_lab);
                }
            }
        }
#pragma unroll
        for (int a = 0; a < LA; ++a)
#pragma unroll
            for (int p = 0; p < P; ++p) {
                lab_q[a][p] = lab_q[a + 1][p];
                w_q[a][p] = w_q[a + 1][p];
            }

    }
    if (!SPEC && !alive && threadIdx.x == 0) {
        // let the copies this block started land before it leaves
        for (unsigned q = produced >= kStages ? produced - kStages : 0; q < produced; ++q)
            if (tiles[q % (2 * kStages)].v >= 0) (void)mbar_wait_bounded(&mbar[q % kStages], (q / kStages) & 1u);
    }
    }  // the aggregating warps
    __syncthreads();
    flush_bin_counts(s, bin, threadIdx.x == 0 ? blk_changed : 0ull, threadIdx.x == 0 ? blk_changed_entries : 0ull);
}

// Dynamic shared memory: kStages index buffers, the table (S keys, S values)
// and the filled-slot lists (S / 2 two-byte entries).
template <int NT, int WK>
static size_t rows_smem(int S) {
    return (size_t)kStages * RowsShape<NT, WK>::BUF * 4 + (size_t)S * 8 + (size_t)S;
}

template <bool ASYNC, int WK, bool BATCH, bool NS, int NT>
static cudaError_t launch_rows_nt(const DevState& s, int bin, int flag, int sms, cudaStream_t st, int* blocks_out) {
    const size_t smem = rows_smem<NT, WK>(s.block_slots[bin - 2]);
    auto kern = k_sweep_rows<ASYNC, WK, BATCH, NS, NT>;
    cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    int per_sm = 0;
    err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, smem);
    if (err != cudaSuccess) return err;
    const int blocks = sms * (per_sm > 0 ? per_sm : 1);
    *blocks_out = blocks;
    kern<<<blocks, NT, smem, st>>>(s, bin, flag);
    return cudaGetLastError();
}

template <bool ASYNC, int WK, bool BATCH, bool NS>
cudaError_t launch_rows(const DevState& s, int bin, int flag, int sms, cudaStream_t st, int* blocks_out) {
    switch (bin) {
        case 2: return launch_rows_nt<ASYNC, WK, BATCH, NS, 128>(s, bin, flag, sms, st, blocks_out);
        case 3: return launch_rows_nt<ASYNC, WK, BATCH, NS, 256>(s, bin, flag, sms, st, blocks_out);
        default: return launch_rows_nt<ASYNC, WK, BATCH, NS, 512>(s, bin, flag, sms, st, blocks_out);
    }
}

#define LPA_ROWS_INST(A, W, B, N) \
    template cudaError_t launch_rows<A, W, B, N>(const DevState&, int, int, int, cudaStream_t, int*);
#define LPA_ROWS_INST_W(A, B, N) \
    LPA_ROWS_INST(A, W_UNIT, B, N) LPA_ROWS_INST(A, W_U32, B, N) LPA_ROWS_INST(A, W_U8, B, N) LPA_ROWS_INST(A, W_F32, B, N)
LPA_ROWS_INST_W(false, false, false)
LPA_ROWS_INST_W(false, false, true)
LPA_ROWS_INST_W(false, true, false)
LPA_ROWS_INST_W(false, true, true)
LPA_ROWS_INST_W(true, false, false)
LPA_ROWS_INST_W(true, false, true)
LPA_ROWS_INST_W(true, true, false)
LPA_ROWS_INST_W(true, true, true)
#undef LPA_ROWS_INST_W
#undef LPA_ROWS_INST

}  // namespace lpa
