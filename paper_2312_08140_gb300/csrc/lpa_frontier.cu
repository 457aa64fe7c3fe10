// lpa_frontier.cu -- everything around the sweep kernels:
//   k_set_params   run parameters into the control block
//   k_init         C <- [0..N), every vertex with an entry marked unprocessed
//                  (Algorithm 1, lpa(): initialisation)
//   k_finish       after a sweep: apply sync-mode changes, compact the flags
//                  of unprocessed vertices into per-degree-bin frontier lists,
//                  and, in the last block, the per-graph convergence test
//                  dN/N <= tau or the sweep cap (Algorithm 1; Sections 4.1.2,
//                  4.1.3), which also sets the device-side loop condition
//   k_finalize     labels out (optionally as graph-local ids)
//   k_validate     CSR checks at graph creation, weight exactness
//   k_mod_*        modularity, Eq. 1 (Section 3.2), in fp64
#include <vector>

#include "lpa_device.cuh"

namespace lpa {

constexpr int kFrontThreads = 256;
constexpr int kVertsPerThread = 16;

__global__ void k_set_params(Ctrl* ctrl, double tau, int max_iters, int mode, int nonstrict, int prune_other,
                             int32_t* labels_out, int local_ids) {
    ctrl->tau = tau;
    ctrl->max_iters = max_iters;
    ctrl->mode = mode;
    ctrl->nonstrict = nonstrict;
    ctrl->prune_other = prune_other;
    ctrl->labels_out = labels_out;
    ctrl->local_ids = local_ids;
}

cudaError_t launch_set_params(Ctrl* ctrl, double tau, int max_iters, int mode, int nonstrict, int prune_other,
                              int32_t* labels_out, int local_ids, cudaStream_t st) {
    k_set_params<<<1, 1, 0, st>>>(ctrl, tau, max_iters, mode, nonstrict, prune_other, labels_out, local_ids);
    return cudaGetLastError();
}

__global__ void k_init(DevState s) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (int64_t i = tid; i < s.N; i += stride) {
        const int32_t c0 = initial_label(s, (int32_t)i);   // C <- [0 .. |V|) (Algorithm 1), in both buffers
        s.lab[0][i] = c0;
        s.lab[1][i] = c0;
        s.flags[i] = 0;
    }
    Ctrl* c = s.ctrl;
    const int max_iters = c->max_iters;
    for (int64_t g = tid; g < s.G; g += stride) {
        const int64_t ng = s.g_end[g] - s.g_begin[g];
        const bool nothing = ng == 0 || max_iters == 0;
        s.dN[g] = 0;
        s.done[g] = nothing ? 1 : 0;
        s.iters[g] = 0;
        s.exit_reason[g] = nothing ? 2 : 0;
    }
    for (int64_t q = tid; q < kMaxHist; q += stride) {
        c->hist_active[q] = 0;
        c->hist_scanned[q] = 0;
        c->hist_changed_entries[q] = 0;
        for (int b = 0; b < kBins; ++b) {
            c->hist_bin_vertices[q][b] = 0;
            c->hist_bin_entries[q][b] = 0;
            c->hist_bin_changed[q][b] = 0;
            c->hist_bin_changed_entries[q][b] = 0;
        }
    }
    if (tid == 0) {
        // Algorithm 1 marks every vertex unprocessed: the first sweep is dense
        c->iter = 0;
        c->error = 0;
        c->ticket = 0;
        c->cbuf = 0;
        c->rd = 0;
        c->allow_dense = 1;
        c->skip_marks = 1;          // the first pass changes nearly every label
        c->last_pass_high = 0;
        c->dense[0] = 1;
        c->dense[1] = 0;
        c->pass_changed_entries = 0;
        c->ovf_count = 0;
        for (int b = 0; b < kBins; ++b) {
            c->row_next[b] = 0;
            c->bin_cnt[0][b] = s.bin_static[b];
            c->bin_entries[0][b] = s.bin_static_entries[b];
            c->bin_cnt[1][b] = 0;
            c->bin_entries[1][b] = 0;
            c->bin_changed[b] = 0;
            c->bin_changed_entries[b] = 0;
            c->sweep_bin_vertices[b] = 0;
            c->sweep_bin_entries[b] = 0;
        }
    }
}

// Separate 1-thread kernel: the only writer of the loop condition before the
// loop starts (concurrent writers of a conditional handle are not allowed).
__global__ void k_init_cond(DevState s, cudaGraphConditionalHandle h, int in_graph) {
    const bool run = s.ctrl->max_iters > 0 && s.N > 0;
    s.ctrl->any_active = run ? 1 : 0;
    if (in_graph) cudaGraphSetConditional(h, run ? 1u : 0u);
}

cudaError_t launch_init(const DevState& s, cudaStream_t st, int sms) {
    k_init<<<sms * 4, kFrontThreads, 0, st>>>(s);
    return cudaGetLastError();
}

cudaError_t launch_init_cond(const DevState& s, cudaGraphConditionalHandle h, int in_graph, cudaStream_t st) {
    k_init_cond<<<1, 1, 0, st>>>(s, h, in_graph);
    return cudaGetLastError();
}

__device__ __forceinline__ int bin_of(const DevState& s, int64_t d) {
    return d <= s.small_max ? 0 : d <= s.warp_max ? 1 : d <= s.mid_max ? 2 : d <= s.large_max ? 3 : 4;
}

// A thread's chunk of kVertsPerThread consecutive vertices v0 + q, each
// either left out or given a degree bin: the bins packed 4 bits per vertex
// (0 = left out, else bin + 1) and the entries (degree sum) per bin.  Kept this
// compact so the compaction kernels stay at a few dozen registers.
struct Chunk {
    int64_t v0;
    uint64_t code;
    unsigned long long ent[kBins];
};

__device__ __forceinline__ void chunk_reset(Chunk& c, int64_t v0) {
    c.v0 = v0;
    c.code = 0;
#pragma unroll
    for (int b = 0; b < kBins; ++b) c.ent[b] = 0;
}

__device__ __forceinline__ void chunk_add(Chunk& c, int q, int bin, int64_t d) {
    c.code |= (uint64_t)(bin + 1) << (4 * q);
#pragma unroll
    for (int b = 0; b < kBins; ++b) c.ent[b] += bin == b ? (unsigned long long)d : 0ull;
}

// Number of 4-bit fields of `code` equal to `val` (exact: no borrow between fields).
__device__ __forceinline__ unsigned nibbles_equal(uint64_t code, unsigned val) {
    const uint64_t x = code ^ (0x1111111111111111ull * val);
    const uint64_t lo = 0x7777777777777777ull;
    return (unsigned)__popcll(~(((x & lo) + lo) | x | lo));
}

// Bin of vertex v0 + q of the chunk, or -1.
__device__ __forceinline__ int chunk_bin(const Chunk& c, int q) { return (int)((c.code >> (4 * q)) & 0xf) - 1; }

// Block-wide ordered append of every thread's chunk into the kBins bin
// regions of `list`; `cursor[b]` is the running length of bin b (device
// counter when ATOMIC, otherwise a running offset owned by the caller).
// Entries keep ascending thread order.  The block's ids are grouped by bin in
// shared memory first, so each bin's run is written with coalesced stores.
// All threads of the block must call.
template <bool ATOMIC>
__device__ __forceinline__ void block_append(const int64_t (&base)[kBins], int32_t* list, unsigned* cursor,
                                             unsigned long long* entries, const Chunk& c) {
    __shared__ unsigned wcnt[kBins][32];
    __shared__ unsigned long long went[kBins][32];
    __shared__ unsigned bbase[kBins], brun[kBins], boff[kBins];
    __shared__ int32_t stage[kFrontThreads * kVertsPerThread];   // the block's ids, grouped by bin
    const unsigned lane = lane_id();
    const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    unsigned excl[kBins];
#pragma unroll
    for (int b = 0; b < kBins; ++b) {
        const unsigned cnt = nibbles_equal(c.code, (unsigned)b + 1u);
        unsigned incl = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned y = __shfl_up_sync(kFull, incl, o);
            if ((int)lane >= o) incl += y;
        }
        unsigned long long ent = c.ent[b];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) ent += __shfl_xor_sync(kFull, ent, o);
        excl[b] = incl - cnt;
        if (lane == 31) {
            wcnt[b][w] = incl;
            went[b][w] = ent;
        }
    }
    __syncthreads();
    if (threadIdx.x < kBins) {
        const int b = threadIdx.x;
        unsigned run = 0;
        unsigned long long ent = 0;
        for (int q = 0; q < nw; ++q) {
            const unsigned x = wcnt[b][q];
            wcnt[b][q] = run;
            run += x;
            ent += went[b][q];
        }
        brun[b] = run;
        if (ATOMIC) {
            bbase[b] = run ? atomicAdd(&cursor[b], run) : 0u;
            if (run) atomicAdd(&entries[b], ent);
        } else {
            bbase[b] = cursor[b];
            cursor[b] += run;
            entries[b] += ent;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned o = 0;
#pragma unroll
        for (int b = 0; b < kBins; ++b) {
            boff[b] = o;
            o += brun[b];
        }
    }
    __syncthreads();
    if (c.code) {
        unsigned pos[kBins];
#pragma unroll
        for (int b = 0; b < kBins; ++b) pos[b] = boff[b] + wcnt[b][w] + excl[b];
#pragma unroll
        for (int q = 0; q < kVertsPerThread; ++q) {
            const int b = chunk_bin(c, q);
#pragma unroll
            for (int k = 0; k < kBins; ++k)
                if (b == k) stage[pos[k]++] = (int32_t)(c.v0 + q);
        }
    }
    __syncthreads();
    // coalesced copy of each bin's run to its place in the list
#pragma unroll
    for (int b = 0; b < kBins; ++b) {
        int32_t* out = list + base[b] + bbase[b];
        const int32_t* in = stage + boff[b];
        for (unsigned i = threadIdx.x; i < brun[b]; i += blockDim.x) out[i] = in[i];
    }
    __syncthreads();
}

// Loads the flags of vertices [v0, v0 + kVertsPerThread) (zeros past N), one
// byte per vertex in `raw`, and clears them when `clear`.  Returns true if any
// is set.
__device__ __forceinline__ bool load_flags(uint8_t* flags, int64_t N, int64_t v0, bool clear, uint4& raw) {
    if (v0 + kVertsPerThread <= N) {
        raw = *reinterpret_cast<const uint4*>(flags + v0);
        const bool anyf = (raw.x | raw.y | raw.z | raw.w) != 0;
        if (anyf && clear) *reinterpret_cast<uint4*>(flags + v0) = make_uint4(0, 0, 0, 0);
        return anyf;
    }
    uint32_t wd[4] = {0, 0, 0, 0};
    for (int q = 0; q < kVertsPerThread; ++q)
        if (v0 + q < N) wd[q >> 2] |= (uint32_t)flags[v0 + q] << (8 * (q & 3));
    raw = make_uint4(wd[0], wd[1], wd[2], wd[3]);
    const bool anyf = (raw.x | raw.y | raw.z | raw.w) != 0;
    if (anyf && clear)
        for (int q = 0; q < kVertsPerThread; ++q)
            if (v0 + q < N) flags[v0 + q] = 0;
    return anyf;
}

__device__ __forceinline__ bool flag_at(const uint4& raw, int q) {
    const uint32_t wd = q < 4 ? raw.x : q < 8 ? raw.y : q < 12 ? raw.z : raw.w;
    return ((wd >> (8 * (q & 3))) & 0xffu) != 0;
}

// Bit q set <=> flag byte q of the chunk is non-zero.
__device__ __forceinline__ uint32_t flag_mask(const uint4& raw) {
    const uint32_t wd[4] = {raw.x, raw.y, raw.z, raw.w};
    uint32_t m = 0;
#pragma unroll
    for (int q = 0; q < kVertsPerThread; ++q) m |= (((wd[q >> 2] >> (8 * (q & 3))) & 0xffu) != 0 ? 1u : 0u) << q;
    return m;
}

// Clears the flag bytes of the chunk at v0 selected by `mask` (bit q = byte q).
__device__ __forceinline__ void clear_flags(uint8_t* flags, int64_t N, int64_t v0, uint4 raw, uint32_t mask) {
    if (v0 + kVertsPerThread <= N) {
        uint32_t wd[4] = {raw.x, raw.y, raw.z, raw.w};
#pragma unroll
        for (int q = 0; q < kVertsPerThread; ++q)
            if ((mask >> q) & 1u) wd[q >> 2] &= ~(0xffu << (8 * (q & 3)));
        *reinterpret_cast<uint4*>(flags + v0) = make_uint4(wd[0], wd[1], wd[2], wd[3]);
    } else {
        for (int q = 0; q < kVertsPerThread && v0 + q < N; ++q)
            if ((mask >> q) & 1u) flags[v0 + q] = 0;
    }
}

// ------------------------------------------------------------ static lists --
// Every vertex with at least one entry, grouped by degree bin, ascending.
// Two passes over blocks of 4096 vertices: count, then ordered scatter from
// per-block bases computed on the host.
constexpr int kStaticChunk = kFrontThreads * kVertsPerThread;

__device__ __forceinline__ void static_chunk(const DevState& s, int64_t v0, Chunk& c) {
    chunk_reset(c, v0);
#pragma unroll
    for (int q = 0; q < kVertsPerThread; ++q) {
        const int64_t v = v0 + q;
        if (v < s.N) {
            const int64_t d = s.off_end[v] - s.off[v];
            if (d > 0) chunk_add(c, q, bin_of(s, d), d);
        }
    }
}

__global__ void __launch_bounds__(kFrontThreads) k_static_count(DevState s, unsigned* counts,
                                                                 unsigned long long* ents) {
    const int64_t v0 = (int64_t)blockIdx.x * kStaticChunk + (int64_t)threadIdx.x * kVertsPerThread;
    Chunk c;
    static_chunk(s, v0, c);
    __shared__ unsigned sc[kBins];
    __shared__ unsigned long long se[kBins];
    if (threadIdx.x < kBins) {
        sc[threadIdx.x] = 0;
        se[threadIdx.x] = 0;
    }
    __syncthreads();
    // one shared atomic per warp and bin
    const unsigned lane = lane_id();
#pragma unroll
    for (int b = 0; b < kBins; ++b) {
        const unsigned cw = __reduce_add_sync(kFull, nibbles_equal(c.code, (unsigned)b + 1u));
        unsigned long long ew = c.ent[b];
        for (int o = 16; o > 0; o >>= 1) ew += __shfl_xor_sync(kFull, ew, o);
        if (lane == 0 && cw) {
            atomicAdd(&sc[b], cw);
            atomicAdd(&se[b], ew);
        }
    }
    __syncthreads();
    if (threadIdx.x < kBins) {
        counts[(size_t)threadIdx.x * gridDim.x + blockIdx.x] = sc[threadIdx.x];
        ents[(size_t)threadIdx.x * gridDim.x + blockIdx.x] = se[threadIdx.x];
    }
}

__global__ void __launch_bounds__(kFrontThreads) k_static_scatter(DevState s, const unsigned* block_base) {
    const int64_t v0 = (int64_t)blockIdx.x * kStaticChunk + (int64_t)threadIdx.x * kVertsPerThread;
    Chunk c;
    static_chunk(s, v0, c);
    __shared__ unsigned cursor[kBins];
    __shared__ unsigned long long ent[kBins];
    if (threadIdx.x < kBins) {
        cursor[threadIdx.x] = block_base[(size_t)threadIdx.x * gridDim.x + blockIdx.x];
        ent[threadIdx.x] = 0;
    }
    __syncthreads();
    block_append<false>(s.bin_base, s.slist, cursor, ent, c);
}

int64_t static_scratch_blocks(int64_t N) { return (N + kStaticChunk - 1) / kStaticChunk; }

cudaError_t build_static_lists(DevState& s, cudaStream_t st, unsigned* counts, unsigned long long* ents) {
    const int64_t nblk = static_scratch_blocks(s.N);
    for (int b = 0; b < kBins; ++b) {
        s.bin_base[b] = 0;
        s.bin_static[b] = 0;
        s.bin_static_entries[b] = 0;
    }
    s.active_entries = 0;
    s.small_iota = 0;
    if (nblk == 0) return cudaSuccess;
    std::vector<unsigned> hc((size_t)nblk * kBins);
    std::vector<unsigned long long> he((size_t)nblk * kBins);
    k_static_count<<<(unsigned)nblk, kFrontThreads, 0, st>>>(s, counts, ents);
    cudaError_t err = cudaGetLastError();
    if (err == cudaSuccess) err = cudaMemcpyAsync(hc.data(), counts, hc.size() * 4, cudaMemcpyDeviceToHost, st);
    if (err == cudaSuccess) err = cudaMemcpyAsync(he.data(), ents, he.size() * 8, cudaMemcpyDeviceToHost, st);
    if (err == cudaSuccess) err = cudaStreamSynchronize(st);
    if (err == cudaSuccess) {
        int64_t base = 0;
        for (int b = 0; b < kBins; ++b) {
            s.bin_base[b] = base;
            unsigned run = 0;
            unsigned long long e = 0;
            for (int64_t k = 0; k < nblk; ++k) {
                const unsigned x = hc[(size_t)b * nblk + k];
                hc[(size_t)b * nblk + k] = run;
                run += x;
                e += he[(size_t)b * nblk + k];
            }
            s.bin_static[b] = run;
            s.bin_static_entries[b] = e;
            s.active_entries += (int64_t)e;
            base += run;
        }
        s.small_iota = (int64_t)s.bin_static[0] * 4 >= s.N * 3 ? 1 : 0;
        err = cudaMemcpyAsync(counts, hc.data(), hc.size() * 4, cudaMemcpyHostToDevice, st);
    }
    if (err == cudaSuccess) {
        k_static_scatter<<<(unsigned)nblk, kFrontThreads, 0, st>>>(s, counts);
        err = cudaGetLastError();
    }
    if (err == cudaSuccess) err = cudaStreamSynchronize(st);
    return err;
}

// Run by the last block of k_finish once every block is done.  `rd` is the
// buffer the pass just consumed; `wr` = rd ^ 1 received the next frontier
// (or is dense; kRoleControl compacts nothing and keeps rd).  At the end of
// sweep t (kRoleEndSweep, kRoleControl) it also runs the per-graph
// convergence test of Algorithm 1 and sets the loop condition.
__device__ void control_step(const DevState& s, int mode, int role, int dense_next, cudaGraphConditionalHandle h,
                             int in_graph) {
    Ctrl* c = s.ctrl;
    volatile Ctrl* vc = c;
    const int t = vc->iter;
    const int rd = vc->rd, wr = rd ^ 1;
    int any = 0;
    const bool ends_sweep = role == kRoleEndSweep || role == kRoleControl;
    const bool compacted = role != kRoleControl;
    if (ends_sweep) {
        const double tau = vc->tau;
        const int max_iters = vc->max_iters;
        unsigned long long changed_total = 0;
        for (int b = 0; b < kBins; ++b) changed_total += vc->bin_changed[b];
        for (int64_t g = threadIdx.x; g < s.G; g += blockDim.x) {
            if (!s.done[g]) {
                const unsigned long long dn =
                    (s.G == 1) ? changed_total : ((volatile unsigned long long*)s.dN)[g];
                const int it = s.iters[g] + 1;          // sweeps of graph g so far
                if (it <= kMaxHist) s.hist_changed[g * kMaxHist + it - 1] = (long long)dn;
                s.iters[g] = it;
                const int64_t ng = s.g_end[g] - s.g_begin[g];
                if ((long long)dn <= dn_threshold(tau, ng)) {     // Algorithm 1: dN / N <= tau
                    s.done[g] = 1;
                    s.exit_reason[g] = 0;
                } else if (it >= max_iters) {
                    s.done[g] = 1;
                    s.exit_reason[g] = 1;
                }
                s.dN[g] = 0;
            }
            any |= !s.done[g];
        }
        any = __syncthreads_or(any);
    }
    if (threadIdx.x != 0) return;
    // the pass that just ended scanned buffer rd
    for (int b = 0; b < kBins; ++b) {
        c->sweep_bin_vertices[b] += vc->bin_cnt[rd][b];
        c->sweep_bin_entries[b] += (long long)vc->bin_entries[rd][b];
    }
    if (ends_sweep) {
        long long act = 0, scn = 0, che = 0;
        for (int b = 0; b < kBins; ++b) {
            act += vc->sweep_bin_vertices[b];
            scn += vc->sweep_bin_entries[b];
            che += (long long)vc->bin_changed_entries[b];
        }
        if (t < kMaxHist) {
            for (int b = 0; b < kBins; ++b) {
                c->hist_bin_vertices[t][b] = vc->sweep_bin_vertices[b];
                c->hist_bin_entries[t][b] = vc->sweep_bin_entries[b];
                c->hist_bin_changed[t][b] = (long long)vc->bin_changed[b];
                c->hist_bin_changed_entries[t][b] = (long long)vc->bin_changed_entries[b];
            }
            c->hist_active[t] = act;
            c->hist_scanned[t] = scn;
            c->hist_changed_entries[t] = che;
        }
        c->total_sweeps += 1;
        c->total_scanned += scn;
        // per pass: one launch per statically non-empty bin (the last bin adds
        // the partitioned rescan), then the finish kernel
        int per_pass = 1;
        for (int b = 0; b < kBins; ++b) per_pass += s.bin_static[b] ? 1 : 0;
        if (s.bin_static[kBins - 1] && s.ovf_possible) per_pass += 4;   // plan, slices, partitions, rescan
        c->total_sweep_launches += mode == MODE_ASYNC ? 2 * per_pass : per_pass;
        for (int b = 0; b < kBins; ++b) {
            c->bin_changed[b] = 0;
            c->bin_changed_entries[b] = 0;
            c->sweep_bin_vertices[b] = 0;
            c->sweep_bin_entries[b] = 0;
        }
        // a dense sync sweep wrote every scanned vertex into the other buffer
        if (mode != MODE_ASYNC && vc->dense[rd]) c->cbuf ^= 1;
        c->iter = t + 1;
        c->any_active = any;
    }
    for (int b = 0; b < kBins; ++b) {
        if (dense_next && compacted) {
            c->bin_cnt[wr][b] = s.bin_static[b];
            c->bin_entries[wr][b] = s.bin_static_entries[b];
        }
        c->bin_cnt[rd][b] = 0;
        c->bin_entries[rd][b] = 0;
        c->row_next[b] = 0;
    }
    if (ends_sweep) {
        // Marks are useless when the next pass is dense anyway.  After two
        // sweeps in a row that changed almost every vertex, the next sweep
        // skips them and the one after it is dense.  An asynchronous sweep's
        // two passes count as one (its catch-up pass marks like its main pass).
        const bool high =
            (double)vc->pass_changed_entries * 1000.0 >= (double)kHighPermille * (double)s.active_entries;
        c->skip_marks = (high && vc->last_pass_high && vc->allow_dense) ? 1 : 0;
        c->last_pass_high = high ? 1 : 0;
        c->pass_changed_entries = 0;
    }
    if (compacted) {
        c->dense[wr] = dense_next;
        c->rd = wr;
    }
    c->ovf_count = 0;
    c->ticket = 0;
    __threadfence();
    if (ends_sweep && in_graph) cudaGraphSetConditional(h, any ? 1u : 0u);
}

// After a pass over buffer rd: (1) at the end of a sparse sync sweep, apply
// the marked changes (current label buffer <- next buffer at the marked
// vertices; after a dense sync sweep the control step flips the buffers
// instead); (2) the next pass is dense (static lists, every vertex) when the
// vertices changed since the last compaction hold at least dense_permille of
// all entries -- then the flags are only cleared -- else the flags are
// compacted into the per-bin frontier lists of buffer rd ^ 1 (the catch-up
// compaction of an asynchronous sweep takes only marked vertices outside the
// sweep's main frontier and is never dense); (3) the last block runs the
// control step.
__global__ void __launch_bounds__(kFrontThreads) k_finish(DevState s, int mode, int role,
                                                           cudaGraphConditionalHandle h, int in_graph) {
    const int rd = s.ctrl->rd, wr = rd ^ 1;
    const unsigned gtid = blockIdx.x * blockDim.x + threadIdx.x;
    const unsigned gstride = gridDim.x * blockDim.x;

    if ((role == kRoleEndSweep || role == kRoleControl) && mode != MODE_ASYNC && !s.ctrl->dense[rd]) {
        const int cb = s.ctrl->cbuf;
        int32_t* C = s.lab[cb];
        const int32_t* Cn = s.lab[cb ^ 1];
        for (int b = 0; b < kBins; ++b) {
            const unsigned cnt = s.ctrl->bin_cnt[rd][b];
            const int32_t* chg = s.chg + s.bin_base[b];
            for (unsigned k0 = gtid * 4u; k0 < cnt; k0 += gstride * 4u) {
                int32_t v[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) v[q] = (k0 + q < cnt) ? chg[k0 + q] : -1;
                int32_t c[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) c[q] = v[q] >= 0 ? Cn[v[q]] : 0;
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    if (v[q] >= 0) C[v[q]] = c[q];
            }
        }
    }

    const bool catch_up = role == kRoleCatchUp;
    const unsigned long long che = ((volatile Ctrl*)s.ctrl)->pass_changed_entries;
    const int dense = !catch_up && s.ctrl->allow_dense &&
                      (mode == MODE_SYNC_FULL || s.ctrl->skip_marks ||
                       (double)che * 1000.0 >= (double)s.dense_permille * (double)s.active_entries);

    const int64_t nchunks = (s.N + kVertsPerThread - 1) / kVertsPerThread;
    if (role == kRoleControl) {
        // serving cycles leave the marks for the next cycle's compaction
    } else if (catch_up && (s.ctrl->dense[rd] || s.ctrl->skip_marks)) {
        // the main pass scanned every vertex (or recorded no marks): nothing
        // is left to reach in this sweep; the marks wait for the next one
    } else if (dense) {
        if (mode != MODE_SYNC_FULL) {
            for (int64_t ch = gtid; ch < nchunks; ch += gstride) {
                const int64_t v0 = ch * kVertsPerThread;
                if (v0 + kVertsPerThread <= s.N) {
                    *reinterpret_cast<uint4*>(s.flags + v0) = make_uint4(0, 0, 0, 0);
                } else {
                    for (int64_t v = v0; v < s.N; ++v) s.flags[v] = 0;
                }
            }
        }
    } else {
        // the compaction that starts an asynchronous sweep records its frontier
        const bool record = mode == MODE_ASYNC && !catch_up;
        for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < nchunks; base += gstride) {
            const int64_t ch = base + threadIdx.x;
            const int64_t v0 = ch * kVertsPerThread;
            uint4 raw = make_uint4(0, 0, 0, 0);
            uint32_t pick = 0;
            if (ch < nchunks && load_flags(s.flags, s.N, v0, !catch_up, raw)) {
                pick = flag_mask(raw);
                if (catch_up) {
                    pick &= ~(uint32_t)s.fr_bits[ch];       // scanned this sweep: keep the mark
                    if (pick) clear_flags(s.flags, s.N, v0, raw, pick);
                }
            }
            Chunk c;
            chunk_reset(c, v0);
            if (pick) {
#pragma unroll
                for (int q = 0; q < kVertsPerThread; ++q) {
                    if ((pick >> q) & 1u) {
                        const int64_t d = s.off_end[v0 + q] - s.off[v0 + q];
                        if (d > 0) chunk_add(c, q, bin_of(s, d), d);
                    }
                }
            }
            if (record && ch < nchunks) s.fr_bits[ch] = (uint16_t)pick;
            if (__syncthreads_or(pick != 0))
                block_append<true>(s.bin_base, s.flist, s.ctrl->bin_cnt[wr], s.ctrl->bin_entries[wr], c);
        }
    }

    // last block runs the control step
    __shared__ bool is_last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned tk = atomicAdd(&s.ctrl->ticket, 1u);
        is_last = tk == gridDim.x - 1;
    }
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    control_step(s, mode, role, dense, h, in_graph);
}

cudaError_t launch_finish(const DevState& s, int mode, int role, cudaGraphConditionalHandle h, int in_graph,
                          cudaStream_t st, int sms) {
    k_finish<<<sms * 4, kFrontThreads, 0, st>>>(s, mode, role, h, in_graph);
    return cudaGetLastError();
}

__global__ void k_finalize(DevState s) {
    int32_t* out = s.ctrl->labels_out;
    const int local = s.ctrl->local_ids;
    const int32_t* C = s.lab[s.ctrl->cbuf];
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < s.N; i += stride) {
        int32_t c = C[i];
        if (local && s.G > 1) c -= (int32_t)s.g_begin[s.gid[i]];
        out[initial_label(s, (int32_t)i)] = c;      // back to the caller's vertex order
    }
}

cudaError_t launch_finalize(const DevState& s, cudaStream_t st, int sms) {
    k_finalize<<<sms * 4, kFrontThreads, 0, st>>>(s);
    return cudaGetLastError();
}

// ------------------------------------------------------------ validation --
// Two flat passes, each with per-thread counters, one shared-memory reduction
// per block and one global atomic per field per block.
//   entries: index range (graph-local for a batch, then rewritten to global
//            ids in idx_rw, the library's own copy), weights finite and
//            >= 0, integer-valued or not, and the largest weight;
//   rows:    offsets (in order, within [0, E], the first at 0, the last at E,
//            batch boundaries at edge_off), degree, and the weighted-degree
//            thresholds 2^24 (fp32 sums may round) and 2^31 (32-bit integer
//            sums may overflow).  A row's exact weighted sum is taken (by the
//            whole warp) only when degree x largest weight reaches 2^24.
constexpr int kValThreads = 256;

struct ValAcc {
    unsigned int c[6];          // bad_offsets, bad_index, bad_weight, non_integer, heavy_row, huge_row
    unsigned long long desc;    // non-increasing adjacent entry pairs (entries pass) / at row starts (rows pass)
    unsigned long long max_degree;
    unsigned int max_weight_bits;
};

__device__ __forceinline__ void val_flush(ValAcc& a, ValidateResult* res, unsigned long long* desc_out) {
    __shared__ unsigned int sc[6];
    __shared__ unsigned long long smax;
    __shared__ unsigned int swmax;
    if (threadIdx.x < 6) sc[threadIdx.x] = 0;
    if (threadIdx.x == 0) {
        smax = 0;
        swmax = 0;
    }
    __syncthreads();
    const unsigned lane = lane_id();
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        const unsigned v = __reduce_add_sync(kFull, a.c[k]);
        if (lane == 0 && v) atomicAdd(&sc[k], v);
    }
    unsigned long long m = a.max_degree;
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long x = __shfl_xor_sync(kFull, m, o);
        m = x > m ? x : m;
    }
    const unsigned wm = __reduce_max_sync(kFull, a.max_weight_bits);
    unsigned long long dsc = a.desc;
    for (int o = 16; o > 0; o >>= 1) dsc += __shfl_xor_sync(kFull, dsc, o);
    if (lane == 0) {
        if (m) atomicMax(&smax, m);
        if (wm) atomicMax(&swmax, wm);
        if (dsc) atomicAdd(desc_out, dsc);
    }
    __syncthreads();
    if (threadIdx.x < 6 && sc[threadIdx.x]) atomicAdd(&res->c[threadIdx.x], sc[threadIdx.x]);
    if (threadIdx.x == 0) {
        if (smax) atomicMax(&res->max_degree, smax);
        if (swmax) atomicMax(&res->max_weight_bits, swmax);
    }
}

// Entries: block b owns the contiguous chunk [e0 + b*chunk, e0 + (b+1)*chunk)
// of the range [e0, e1).
__global__ void __launch_bounds__(kValThreads) k_validate_entries(const int32_t* idx, const float* w, int64_t N,
                                                                  int64_t E, int64_t e0, int64_t e1,
                                                                  const int64_t* vtx_off, const int64_t* edge_off,
                                                                  int32_t G, int rewrite, int32_t* idx_rw,
                                                                  int64_t chunk, ValidateResult* res) {
    ValAcc a{};
    const int64_t beg = e0 + (int64_t)blockIdx.x * chunk;
    const int64_t end = beg + chunk < e1 ? beg + chunk : e1;
    int64_t ge_lo = 0, ge_hi = E, lo = 0, n_local = N;      // entry range, first vertex, size of the graph
    if (rewrite) ge_hi = -1;
    for (int64_t e = beg + threadIdx.x; e < end; e += kValThreads) {
        const int32_t j = idx[e];
        if (rewrite) {
            if (e < ge_lo || e >= ge_hi) {                      // graph g with edge_off[g] <= e < edge_off[g+1]
                int32_t l = 0, h = G;
                while (h - l > 1) {
                    const int32_t mid = (l + h) >> 1;
                    if (edge_off[mid] <= e) l = mid;
                    else h = mid;
                }
                ge_lo = edge_off[l];
                ge_hi = edge_off[l + 1];
                lo = vtx_off[l];
                n_local = vtx_off[l + 1] - lo;
            }
            if (j < 0 || j >= n_local) ++a.c[1];
            else idx_rw[e] = (int32_t)(j + lo);
        } else {
            if (j < 0 || j >= N) ++a.c[1];
            if (e > 0 && j <= idx[e - 1]) ++a.desc;           // no writes here: a single graph
        }
        if (w) {
            const float x = w[e];
            if (!isfinite(x) || x < 0.f) {
                ++a.c[2];
            } else {
                if (x != truncf(x)) ++a.c[3];
                const unsigned bits = __float_as_uint(x);     // x >= 0: bit order is value order
                a.max_weight_bits = bits > a.max_weight_bits ? bits : a.max_weight_bits;
            }
        }
    }
    val_flush(a, res, &res->desc_all);
}

// Rows: lane l of a warp takes row base + l; all lanes run the same trips.
__global__ void __launch_bounds__(kValThreads) k_validate_rows(const int64_t* off, const int32_t* idx, const float* w,
                                                               int64_t N, int64_t E, const int64_t* vtx_off,
                                                               const int64_t* edge_off, const int32_t* gid,
                                                               int32_t G, ValidateResult* res) {
    ValAcc a{};
    const unsigned lane = lane_id();
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const double wmax = w ? (double)__uint_as_float(res->max_weight_bits) : 1.0;   // entries pass ran first
    for (int64_t base = warp * 32; base < N; base += nwarps * 32) {
        const int64_t v = base + lane;
        int64_t st = 0, en = 0;
        bool need_sum = false;
        if (v < N) {
            st = off[v];
            en = off[v + 1];
            bool bad = st < 0 || en < st || en > E || (v == 0 && st != 0) || (v == N - 1 && en != E);
            if (G > 1) {
                const int32_t g = gid[v];
                if (v == vtx_off[g] && st != edge_off[g]) bad = true;
                if (v == vtx_off[g + 1] - 1 && en != edge_off[g + 1]) bad = true;
            }
            if (bad) {
                ++a.c[0];
            } else {
                const int64_t d = en - st;
                a.max_degree = (unsigned long long)d > a.max_degree ? (unsigned long long)d : a.max_degree;
                if (G == 1 && d > 0 && st > 0 && idx[st] <= idx[st - 1]) ++a.desc;
                if (!w) {
                    if (d >= 16777216) ++a.c[4];
                    if (d >= 2147483648LL) ++a.c[5];
                } else {
                    need_sum = (double)d * wmax >= 16777216.0;
                }
            }
        }
        unsigned m = __ballot_sync(kFull, need_sum);
        while (m) {                                             // exact weighted degree, whole warp
            const int l = __ffs(m) - 1;
            m &= m - 1;
            const int64_t rs = __shfl_sync(kFull, st, l), re = __shfl_sync(kFull, en, l);
            double sum = 0.0;
            for (int64_t e = rs + lane; e < re; e += 32) sum += (double)w[e];
            for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(kFull, sum, o);
            if (lane == 0) {
                if (sum >= 16777216.0) ++a.c[4];
                if (sum >= 2147483648.0) ++a.c[5];
            }
        }
    }
    val_flush(a, res, &res->desc_row_starts);
}

cudaError_t launch_validate_entries(const int32_t* idx, const float* w, int64_t N, int64_t E, int64_t e_begin,
                                    int64_t e_end, const int64_t* vtx_off, const int64_t* edge_off, int32_t G,
                                    int rewrite_local_ids, int32_t* idx_rw, ValidateResult* res, cudaStream_t st,
                                    int sms) {
    const int64_t cnt = e_end - e_begin;
    if (cnt <= 0) return cudaSuccess;
    const int64_t max_blocks = (int64_t)sms * 8;
    int64_t chunk = (cnt + max_blocks - 1) / max_blocks;
    chunk = std::max<int64_t>((chunk + kValThreads - 1) / kValThreads * kValThreads, kValThreads * 4);
    const int blocks = (int)((cnt + chunk - 1) / chunk);
    k_validate_entries<<<blocks, kValThreads, 0, st>>>(idx, w, N, E, e_begin, e_end, vtx_off, edge_off, G,
                                                       rewrite_local_ids, idx_rw, chunk, res);
    return cudaGetLastError();
}

cudaError_t launch_validate_rows(const int64_t* off, const int32_t* idx, const float* w, int64_t N, int64_t E,
                                 const int64_t* vtx_off, const int64_t* edge_off, const int32_t* gid, int32_t G,
                                 ValidateResult* res, cudaStream_t st, int sms) {
    const int64_t warps = (N + 31) / 32;
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((warps + 7) / 8, (int64_t)sms * 8));
    k_validate_rows<<<blocks, kValThreads, 0, st>>>(off, idx, w, N, E, vtx_off, edge_off, gid, G, res);
    return cudaGetLastError();
}

__global__ void k_fill_gid(const int64_t* vtx_off, int32_t G, int64_t N, int32_t* gid) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < N; v += stride) {
        int32_t lo = 0, hi = G;   // find g with vtx_off[g] <= v < vtx_off[g+1]
        while (hi - lo > 1) {
            const int32_t mid = (lo + hi) >> 1;
            if (vtx_off[mid] <= v) lo = mid;
            else hi = mid;
        }
        gid[v] = lo;
    }
}

cudaError_t launch_fill_gid(const int64_t* vtx_off, int32_t G, int64_t N, int32_t* gid, cudaStream_t st, int sms) {
    k_fill_gid<<<sms * 4, 256, 0, st>>>(vtx_off, G, N, gid);
    return cudaGetLastError();
}

__global__ void k_weights_to_u32(float* w, int64_t E) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    uint32_t* u = reinterpret_cast<uint32_t*>(w);
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < E; e += stride)
        u[e] = (uint32_t)w[e];
}

cudaError_t launch_weights_to_u32(float* w, int64_t E, cudaStream_t st, int sms) {
    k_weights_to_u32<<<sms * 8, 256, 0, st>>>(w, E);
    return cudaGetLastError();
}

__global__ void k_weights_to_u8(const float* w, unsigned char* out, int64_t E) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < E; e += stride)
        out[e] = (unsigned char)w[e];
}

cudaError_t launch_weights_to_u8(const float* w, unsigned char* out, int64_t E, cudaStream_t st, int sms) {
    k_weights_to_u8<<<sms * 8, 256, 0, st>>>(w, out, E);
    return cudaGetLastError();
}

// ------------------------------------------------------- degree histogram --
// Vertices and entries per degree bucket b = ceil(log2(d)) (d >= 1; b = 0 for
// d = 1), over vertices [0, N): hist[b] vertices, hist[kDegBuckets + b]
// entries.  With bin limits that are powers of two the bucket counts give the
// bin counts of any lpa_config exactly.
__global__ void k_degree_hist(const int64_t* off, const int64_t* off_end, int64_t N, unsigned long long* hist) {
    __shared__ unsigned long long sh[2 * kDegBuckets];
    for (int q = threadIdx.x; q < 2 * kDegBuckets; q += blockDim.x) sh[q] = 0ull;
    __syncthreads();
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < N; v += stride) {
        const int64_t d = off_end[v] - off[v];
        if (d > 0) {
            const int b = d <= 1 ? 0 : 64 - __clzll((unsigned long long)(d - 1));
            atomicAdd(&sh[b], 1ull);
            atomicAdd(&sh[kDegBuckets + b], (unsigned long long)d);
        }
    }
    __syncthreads();
    for (int q = threadIdx.x; q < 2 * kDegBuckets; q += blockDim.x)
        if (sh[q]) atomicAdd(&hist[q], sh[q]);
}

cudaError_t launch_degree_hist(const DevState& s, unsigned long long* hist, cudaStream_t st, int sms) {
    cudaError_t e = cudaMemsetAsync(hist, 0, 2 * kDegBuckets * sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    k_degree_hist<<<sms * 2, 256, 0, st>>>(s.off, s.off_end, s.N, hist);
    return cudaGetLastError();
}

// ------------------------------------------------------------ modularity --
__device__ __forceinline__ double weight_f64(const DevState& s, int64_t e) {
    if (s.weight_kind == W_UNIT) return 1.0;
    if (s.weight_kind == W_U32) return (double)static_cast<const uint32_t*>(s.w)[e];
    if (s.weight_kind == W_U8) return (double)static_cast<const unsigned char*>(s.w)[e];
    return (double)static_cast<const float*>(s.w)[e];
}

// One warp per vertex i of [v0, v1): K_i, and the weight of entries whose two
// ends share a label (sigma); Sigma_c += K_i.
__global__ void k_mod_rows(DevState s, int64_t v0, int64_t v1, const int32_t* labels, double* Sigma,
                           ModAccum* acc) {
    __shared__ double sh_two_m, sh_sigma;
    if (threadIdx.x == 0) {
        sh_two_m = 0.0;
        sh_sigma = 0.0;
    }
    __syncthreads();
    const unsigned lane = lane_id();
    const int64_t nloc = v1 - v0;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    double my_two_m = 0.0, my_sigma = 0.0;
    // labels are given in the caller's vertex order: stored vertex u holds
    // the label of its original id
    auto label_of = [&](int64_t u) -> int32_t { return labels[(int64_t)initial_label(s, (int32_t)u) - v0]; };
    for (int64_t i = warp; i < nloc; i += nwarps) {
        const int32_t ci = label_of(v0 + i);
        if (ci < 0 || ci >= nloc) {
            if (lane == 0) atomicAdd(&acc->bad_label, 1u);
            continue;
        }
        double K = 0.0, sg = 0.0;
        const int64_t st = s.off[v0 + i], en = s.off_end[v0 + i];
        for (int64_t e = st + lane; e < en; e += 32) {
            const double w = weight_f64(s, e);
            K += w;
            const int64_t j = (int64_t)s.idx[e] - v0;
            if (j >= 0 && j < nloc && label_of(v0 + j) == ci) sg += w;
        }
        for (int o = 16; o > 0; o >>= 1) {
            K += __shfl_xor_sync(kFull, K, o);
            sg += __shfl_xor_sync(kFull, sg, o);
        }
        if (lane == 0) {
            atomicAdd(&Sigma[ci], K);
            my_two_m += K;
            my_sigma += sg;
        }
    }
    if (lane == 0) {
        atomicAdd(&sh_two_m, my_two_m);
        atomicAdd(&sh_sigma, my_sigma);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        atomicAdd(&acc->two_m, sh_two_m);
        atomicAdd(&acc->sigma, sh_sigma);
    }
}

__global__ void k_mod_null(const double* Sigma, int64_t n, ModAccum* acc) {
    __shared__ double sh;
    if (threadIdx.x == 0) sh = 0.0;
    __syncthreads();
    double local = 0.0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += stride) local += Sigma[c] * Sigma[c];
    for (int o = 16; o > 0; o >>= 1) local += __shfl_xor_sync(kFull, local, o);
    if (lane_id() == 0) atomicAdd(&sh, local);
    __syncthreads();
    if (threadIdx.x == 0) atomicAdd(&acc->null_sum, sh);
}

cudaError_t launch_modularity(const DevState& s, int64_t v0, int64_t v1, const int32_t* labels, double* Sigma,
                              ModAccum* acc, cudaStream_t st, int sms) {
    k_mod_rows<<<sms * 8, 256, 0, st>>>(s, v0, v1, labels, Sigma, acc);
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return err;
    k_mod_null<<<sms * 4, 256, 0, st>>>(Sigma, v1 - v0, acc);
    return cudaGetLastError();
}

}  // namespace lpa
