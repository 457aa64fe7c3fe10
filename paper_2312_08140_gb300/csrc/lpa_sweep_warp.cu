// lpa_sweep_warp.cu -- sweep for mid-degree vertices (small_max < d <= warp_max):
// one warp per frontier vertex.
//
// The warp reads the row 32 entries at a time (coalesced index and weight
// loads, one label gather per lane).  Within each 32-entry chunk, lanes that
// hold the same label are grouped with __match_any_sync and their weights
// combined (a popcount for unit weights, a group reduction for integer
// weights), so each distinct label of the chunk costs one table update.
//   d <= 32: the grouped sums are already the per-label totals K_{i->c}
//            (Eq. 2) and the warp takes the argmax directly.
//   d  > 32: group leaders add their sums into a per-warp open-addressing
//            table in shared memory sized 2^ceil(log2(2d)) slots (so it can
//            never fill) and list the slots they fill; the warp then scans
//            the listed slots for the argmax and clears them.
// A chunk whose labels all agree (after the first sweeps nearly every chunk)
// skips the grouping: a row of one chunk takes that label's total directly,
// and in a longer row such chunks extend a run of one label held in
// registers, which reaches the table once.
// Ties go to the smallest label id (Section 4.1.5); self-loops are skipped
// (Algorithm 1).  On change, the warp re-reads the row and marks the
// neighbours unprocessed (Section 4.1.4).
#include "lpa_device.cuh"

namespace lpa {

constexpr int kWarpThreads = 256;
constexpr int kWarpsPerBlock = kWarpThreads / 32;
constexpr int kWarpUnroll = 3;      // chunks of 32 entries in flight per warp beyond the first
constexpr unsigned kAsyncMinBatch = 16;       // async: at least this many consecutive visits per warp batch
constexpr unsigned kAsyncMaxRunBatches = 8;   // async: batches a warp walks in one run
constexpr unsigned kAsyncSmallRunBatches = 2;  // async, a bin of one wave of batches: batches per run
constexpr unsigned kScatterWindow = 4096;   // batches per scattered window (a power of two)

// Combined weight of the lanes in `peers` (all hold the same label).
template <int WK>
__device__ __forceinline__ typename Acc<WK>::T group_sum(unsigned peers, typename Acc<WK>::T w,
                                                         int32_t lab, bool ok) {
    if constexpr (WK == W_UNIT) {
        return (typename Acc<WK>::T)__popc(peers);
    } else if constexpr (WK == W_U32 || WK == W_U8) {
        return __reduce_add_sync(peers, w);
    } else {
        // fp32: every lane of a group adds the group's weights in lane order,
        // so all of them obtain the same value.
        float sum = 0.f;
        for (int q = 0; q < 32; ++q) {
            float wq = __shfl_sync(kFull, w, q);
            int32_t lq = __shfl_sync(kFull, lab, q);
            if (ok && lq == lab) sum += wq;
        }
        (void)peers;
        return sum;
    }
}

template <bool ASYNC, int WK, bool BATCH, bool NS>
__global__ void __launch_bounds__(kWarpThreads, 4) k_sweep_warp(DevState s, int flag_neighbours) {
    using T = typename Acc<WK>::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int wslots = s.warp_slots;
    const unsigned lane = lane_id();
    const int wib = threadIdx.x >> 5;
    int32_t* keys = reinterpret_cast<int32_t*>(smem_raw) + (size_t)wib * wslots * 2;
    T* vals = reinterpret_cast<T*>(keys + wslots);
    // slots the current row filled (a row has at most wslots / 2 labels);
    // `filled` counts them, the same value in every lane
    uint16_t* filled_slots =
        reinterpret_cast<uint16_t*>(reinterpret_cast<int32_t*>(smem_raw) + (size_t)kWarpsPerBlock * wslots * 2) +
        (size_t)wib * (wslots / 2);
    unsigned filled = 0;
    for (int q = lane; q < wslots; q += 32) {
        keys[q] = kEmptyKey;
        vals[q] = (T)0;
    }
    __syncwarp();

    const BinView bv = bin_view(s, 1);
    const Labels L = labels_of(s);
    const bool marks = marks_on(s, flag_neighbours);
    const uint32_t sweep = NS ? (uint32_t)s.ctrl->iter + 1u : 0u;   // non-strict tie-break (Section 4.1.5)
    const bool ident = identity_sweep<ASYNC, BATCH>(s);
    const bool po = ASYNC && s.ctrl->prune_other != 0;               // FLPA's pruning rule
    const unsigned cnt = bv.cnt;
    const unsigned nwarps = gridDim.x * kWarpsPerBlock;
    // each warp takes batches of B consecutive frontier entries (B <= 32) and
    // visits them one after another, B shrinking when the bin is too small to
    // give every warp a full batch.  In the asynchronous mode B stays at least
    // kAsyncMinBatch, so that a small graph is not scanned all at once (which
    // would make the pass synchronous).  On the 4313-vertex planted partition
    // of the tests, runs of 8 gave Q 0.731 where serial random orders reach
    // 0.753 (a lockstep model of the kernel, every batch advancing one vertex
    // per round on the labels before the round, predicts the same); runs of
    // 16 stay within 0.02 of the serial median on every test graph in that
    // model, runs of 32 do not (ascending runs flood two of them).
    unsigned B = (cnt + nwarps - 1) / nwarps;
    if (ASYNC && B < kAsyncMinBatch) B = kAsyncMinBatch;
    B = B < 1u ? 1u : (B > 32u ? 32u : B);
    // In the asynchronous mode the batches are visited in a scattered order
    // within windows of kScatterWindow batches (an odd multiplier modulo the
    // window's power-of-two size; the last, partial window in order).  In id
    // order, a graph spanning several waves of warps would have its low ids
    // updated before its high ids -- a coarse ascending sweep that, with the
    // smallest-id tie-break, lets the smallest labels flood through id-ordered
    // blocks.  The windows keep the labels being gathered at a time to a few
    // graphs' worth (L2-resident) in large batches.
    const unsigned nbatch = (cnt + B - 1) / B;
    // Asynchronous mode: a warp walks K consecutive batches in order (a run
    // of K x B vertices), K as large as 8 while the bin still gives every
    // warp at least two runs; fewer runs in flight at once means fewer
    // vertices reading labels their neighbours are about to change (a
    // 140K-vertex planted partition inside a 4096-graph batch: median Q 0.645
    // with single batches, 0.750 with runs of 8, serial runs 0.745).
    unsigned K = 1;
    if (ASYNC)
        while (K < kAsyncMaxRunBatches && (unsigned long long)nbatch >= 2ull * (2u * K) * nwarps) K *= 2u;
    // A bin of one wave (a small graph) has every batch in flight at once;
    // runs of two batches halve that (the twenty 100-5000-vertex test graphs,
    // 20 runs each on fresh handles: one run in 400 fell 0.02 below the
    // lowest of 16 serial orders with single batches, none with runs of two).
    if (ASYNC && nbatch <= nwarps) K = kAsyncSmallRunBatches;
    const unsigned nruns = (nbatch + K - 1) / K;
    const unsigned full_windows = nruns / kScatterWindow;
    // Graphs kept in the caller's order inside a batch (the serving arena,
    // LPA_KEEP_ORDER): their vertices come in id order, and on id-ordered
    // communities a run of consecutive vertices acts as a short ascending
    // sweep, so the entries of a run are drawn at pseudo-random positions of
    // the frontier instead (a Feistel permutation, redrawn every sweep) --
    // what the shuffled storage order of batches gives the others.
    const bool scatter_entries = ASYNC && BATCH && s.orig == nullptr;
    const uint64_t visit_seed = 0x2312081405ull + 0x9E3779B97F4A7C15ull * (uint64_t)s.ctrl->iter;
    unsigned long long my_changed = 0, my_changed_entries = 0;
    for (unsigned ri = blockIdx.x * kWarpsPerBlock + wib; ri < nruns; ri += nwarps) {
        unsigned pr = ri;
        if (ASYNC && ri / kScatterWindow < full_windows)
            pr = (ri & ~(kScatterWindow - 1u)) | ((ri * 0x9E3779B1u) & (kScatterWindow - 1u));
      for (unsigned pb = pr * K; pb < pr * K + K && pb < nbatch; ++pb) {
        const unsigned base = pb * B;
        // Metadata of up to B consecutive frontier entries, one per lane, loaded
        // together so their latencies overlap.
        const unsigned kl = base + lane;
        const bool okl = lane < B && kl < cnt;
        const unsigned pl = (scatter_entries && okl) ? shuffle_pos(kl, cnt, visit_seed) : kl;   // frontier slot
        const int32_t vl = okl ? bv.list[pl] : 0;
        int64_t stl = 0, enl = 0;
        int32_t ownl = 0;
        int actl = okl;
        if (okl) {
            stl = s.off[vl];
            enl = s.off_end[vl];
            ownl = ASYNC ? __ldcg(L.C + vl) : L.C[vl];
            if constexpr (BATCH) {
                if (s.done[s.gid[vl]]) actl = 0;
            }
        }
        const unsigned nv = min(B, cnt - base);
        // Two-stage pipeline over the batch: while vertex i is aggregated, the
        // first-chunk labels and weights of vertex i+1 and the first-chunk
        // indices of vertex i+2 are in flight.
        auto first_index = [&](unsigned i) -> int32_t {
            const unsigned q = i & 31u;
            const int64_t sq = __shfl_sync(kFull, stl, q), eq = __shfl_sync(kFull, enl, q);
            const int aq = __shfl_sync(kFull, actl, q) && (i < nv);
            return (aq && sq + lane < eq) ? load_index_keep(s.idx, sq + lane) : kEmptyKey;
        };
        auto first_label = [&](unsigned i, int32_t j, int32_t& lab, T& w) {
            const unsigned q = i & 31u;
            const int32_t vq = __shfl_sync(kFull, vl, q);
            const int64_t sq = __shfl_sync(kFull, stl, q);
            const bool ok = j != kEmptyKey && j != vq;
            lab = ok ? (ident ? initial_label(s, j) : load_label<ASYNC>(L.C, j)) : kEmptyKey;
            w = ok ? load_weight<WK>(s.w, sq + lane) : (T)0;
        };
        int32_t j_cur = first_index(0), j_nxt = first_index(1);
        int32_t lab_cur;
        T w_cur;
        first_label(0, j_cur, lab_cur, w_cur);
        for (unsigned i = 0; i < nv; ++i) {
            const int32_t v = __shfl_sync(kFull, vl, i);
            const int64_t st = __shfl_sync(kFull, stl, i);
            const int64_t en = __shfl_sync(kFull, enl, i);
            const int32_t own = __shfl_sync(kFull, ownl, i);
            const int act = __shfl_sync(kFull, actl, i);
            const int d = (int)(en - st);
            const TieRule tr = tie_rule(s, NS && act, sweep, v);
            const int32_t j = j_cur;
            const int32_t lab_row = lab_cur;        // this row's first-chunk labels
            const int32_t j_nn = first_index(i + 2);
            int32_t lab_nxt;
            T w_nxt;
            first_label(i + 1, j_nxt, lab_nxt, w_nxt);
            uint32_t key = 0;
            int32_t cand = 0;
            if (act && d <= 32) {
                const bool ok = lab_cur != kEmptyKey;
                // all of the row's labels agree (after the first sweeps the
                // usual case): the row's total weight is that label's sum
                const int32_t lmax = __reduce_max_sync(kFull, lab_cur);
                if (__all_sync(kFull, !ok || lab_cur == lmax)) {
                    T sum;
                    if constexpr (WK == W_UNIT) {
                        sum = (T)__popc(__ballot_sync(kFull, ok));
                    } else if constexpr (WK == W_F32) {
                        sum = group_sum<WK>(kFull, w_cur, lab_cur, ok);
                    } else {
                        sum = __reduce_add_sync(kFull, w_cur);
                    }
                    if (lane == 0 && lmax != kEmptyKey) {
                        key = sum_key(sum);
                        cand = lmax;
                    }
                } else {
                    const unsigned peers = __match_any_sync(kFull, lab_cur);
                    const T sum = group_sum<WK>(peers, w_cur, lab_cur, ok);
                    if (ok && lane == (unsigned)(__ffs(peers) - 1)) {
                        key = sum_key(sum);
                        cand = lab_cur;
                    }
                }
            } else if (act && ident) {
                // labels are the neighbour ids and occur once: a max over the row
                unsigned long long bp = lab_cur != kEmptyKey ? pack_candidate(sum_key(w_cur), tr.key(lab_cur)) : 0ull;
#pragma unroll 4
                for (int64_t e = st + 32 + lane; e < en; e += 32) {
                    const int32_t jj = load_index_keep(s.idx, e);
                    if (jj != v) {
                        const unsigned long long c =
                            pack_candidate(sum_key(load_weight<WK>(s.w, e)), tr.key(initial_label(s, jj)));
                        bp = c > bp ? c : bp;
                    }
                }
                bp = warp_max_u64(bp);
                if (lane == 0 && bp != 0ull) {
                    key = (uint32_t)(bp >> 32);
                    cand = tr.label(~(uint32_t)bp);
                }
            } else if (act) {
                const int log_slots = ceil_log2(2u * (unsigned)d);
                // one (label, weight) into the warp's table by `lane`, its
                // newly filled slot listed
                auto insert_listed = [&](bool ins, int32_t lab, T add) {
                    int created = -1;
                    if (ins && !table_insert<T>(keys, vals, log_slots, lab, add, 1u << log_slots, created))
                        atomicExch(&s.ctrl->error, 2);
                    const unsigned nm = __ballot_sync(kFull, created >= 0);
                    if (created >= 0) filled_slots[filled + __popc(nm & lanes_below())] = (uint16_t)created;
                    filled += __popc(nm);
                };
                // Chunks whose labels all agree extend a run held in registers
                // (same value in every lane); the run reaches the table once,
                // when a chunk with another label or mixed labels ends it, or
                // at the end of the row.
                int32_t run_lab = kEmptyKey;
                T run_w = (T)0;
                auto flush_run = [&]() {
                    if (run_lab != kEmptyKey) insert_listed(lane == 0, run_lab, run_w);
                    run_lab = kEmptyKey;
                    run_w = (T)0;
                };
                auto add_chunk = [&](int32_t lab, T w) {
                    const bool ok = lab != kEmptyKey;
                    const int32_t lmax = __reduce_max_sync(kFull, lab);
                    if (__all_sync(kFull, !ok || lab == lmax)) {
                        if (lmax == kEmptyKey) return;
                        T sum;
                        if constexpr (WK == W_UNIT) {
                            sum = (T)__popc(__ballot_sync(kFull, ok));
                        } else if constexpr (WK == W_F32) {
                            sum = group_sum<WK>(kFull, w, lab, ok);
                        } else {
                            sum = __reduce_add_sync(kFull, w);
                        }
                        if (lmax != run_lab) {
                            flush_run();
                            run_lab = lmax;
                        }
                        run_w += sum;
                        return;
                    }
                    flush_run();
                    bool ins = ok;
                    T add = w;
                    if constexpr (WK != W_F32) {
                        const unsigned peers = __match_any_sync(kFull, lab);
                        add = group_sum<WK>(peers, w, lab, ok);
                        ins = ok && lane == (unsigned)(__ffs(peers) - 1);
                    }
                    insert_listed(ins, lab, add);
                };
                add_chunk(lab_cur, w_cur);                 // first chunk, prefetched
                for (int64_t e0 = st + 32; e0 < en; e0 += 32 * kWarpUnroll) {
                    int32_t jj[kWarpUnroll], ll[kWarpUnroll];
                    T wq[kWarpUnroll];
#pragma unroll
                    for (int u = 0; u < kWarpUnroll; ++u) {
                        const int64_t e = e0 + 32 * u + lane;
                        jj[u] = e < en ? load_index_keep(s.idx, e) : v;
                    }
#pragma unroll
                    for (int u = 0; u < kWarpUnroll; ++u) {
                        const bool ok = jj[u] != v;
                        ll[u] = ok ? load_label<ASYNC>(L.C, jj[u]) : kEmptyKey;
                        wq[u] = ok ? load_weight<WK>(s.w, e0 + 32 * u + lane) : (T)0;
                    }
#pragma unroll
                    for (int u = 0; u < kWarpUnroll; ++u) {
                        if (e0 + 32 * u >= en) break;      // warp-uniform
                        add_chunk(ll[u], wq[u]);
                    }
                }
                flush_run();
                __syncwarp();
                bool any = false;
                T best_w = 0;
                uint32_t best_k = 0xffffffffu;
                for (unsigned f = lane; f < filled; f += 32) {
                    const int q = filled_slots[f];
                    const int32_t kq = keys[q];
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
                filled = 0;
                __syncwarp();
                if (any) {
                    key = sum_key(best_w);
                    cand = tr.label(best_k);
                }
            }
            j_cur = j_nxt;
            j_nxt = j_nn;
            lab_cur = lab_nxt;
            w_cur = w_nxt;
            const uint32_t best_key = warp_argmax_tie(key, key ? tr.key(cand) : 0xffffffffu);
            const int32_t best = best_key == 0xffffffffu ? -1 : tr.label(best_key);
            const bool changed = act && best >= 0 && best != own;   // warp-uniform
            const unsigned slot = __shfl_sync(kFull, pl, i);
            if (lane == 0) record_label<ASYNC>(L, bv.chg + slot, v, own, best, changed);
            if constexpr (ASYNC) {
                // the next vertex's first-chunk labels were read before this
                // update: lanes holding v as neighbour take its new label
                if (changed && j_cur == v) lab_cur = best;
            }
            if (changed) {
                if (marks) {
                    // FLPA's rule: a neighbour already carrying `best` stays unmarked
                    if (d <= 32) {                   // this row's indices are still in j
                        if ((int)lane < d && j != v && !(po && lab_row == best)) mark_unprocessed(s.flags, j);
                    } else {
                        // up to four chunks of the row in flight: ids, then flags
                        for (int64_t e0 = st + lane; e0 < en; e0 += 128) {
                            int32_t jj[4];
                            uint8_t f[4];
#pragma unroll
                            for (int u = 0; u < 4; ++u) jj[u] = e0 + 32 * u < en ? s.idx[e0 + 32 * u] : v;
#pragma unroll
                            for (int u = 0; u < 4; ++u) f[u] = jj[u] != v ? __ldcg(s.flags + jj[u]) : (uint8_t)1;
#pragma unroll
                            for (int u = 0; u < 4; ++u)
                                if (f[u] == 0 && !(po && load_label<ASYNC>(L.C, jj[u]) == best)) s.flags[jj[u]] = 1;
                        }
                    }
                }
                if (lane == 0) {
                    ++my_changed;
                    my_changed_entries += (unsigned)d;
                    if constexpr (BATCH) atomicAdd(&s.dN[s.gid[v]], 1ull);
                }
            }
        }
      }
    }
    flush_bin_counts(s, 1, my_changed, my_changed_entries);
}

template <bool ASYNC, int WK, bool BATCH, bool NS>
static cudaError_t launch_warp_t(const DevState& s, int flag, cudaStream_t st, int sms) {
    const size_t smem = (size_t)kWarpsPerBlock * s.warp_slots * 9;     // table + list of filled slots
    auto kern = k_sweep_warp<ASYNC, WK, BATCH, NS>;
    cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    int per_sm = 0;
    err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kWarpThreads, smem);
    if (err != cudaSuccess) return err;
    if (per_sm < 1) per_sm = 1;
    kern<<<sms * per_sm, kWarpThreads, smem, st>>>(s, flag);
    return cudaGetLastError();
}

template <bool ASYNC, bool BATCH, bool NS>
static cudaError_t launch_warp_w(const DevState& s, int flag, cudaStream_t st, int sms) {
    switch (s.weight_kind) {
        case W_UNIT: return launch_warp_t<ASYNC, W_UNIT, BATCH, NS>(s, flag, st, sms);
        case W_U32: return launch_warp_t<ASYNC, W_U32, BATCH, NS>(s, flag, st, sms);
        case W_U8: return launch_warp_t<ASYNC, W_U8, BATCH, NS>(s, flag, st, sms);
        default: return launch_warp_t<ASYNC, W_F32, BATCH, NS>(s, flag, st, sms);
    }
}

template <bool NS>
static cudaError_t launch_warp_ns(const DevState& s, bool async, int flag, cudaStream_t st, int sms) {
    const bool batch = s.G > 1;
    if (async) return batch ? launch_warp_w<true, true, NS>(s, flag, st, sms) : launch_warp_w<true, false, NS>(s, flag, st, sms);
    return batch ? launch_warp_w<false, true, NS>(s, flag, st, sms) : launch_warp_w<false, false, NS>(s, flag, st, sms);
}

cudaError_t launch_sweep_warp(const DevState& s, int mode, cudaStream_t st, int sms) {
    const bool ns = (mode & kModeNonstrict) != 0;
    mode &= ~kModeNonstrict;
    const bool async = mode == MODE_ASYNC;
    const int flag = mode != MODE_SYNC_FULL;
    return ns ? launch_warp_ns<true>(s, async, flag, st, sms) : launch_warp_ns<false>(s, async, flag, st, sms);
}

}  // namespace lpa
