// lpa_device.cuh -- device helpers shared by the sweep kernels.
//
// Weight sums: for graphs whose weights are integers (or unit) in the
// library's own copy, the per-label sums K_{i->c} are accumulated in uint32
// (exact in any order while every weighted degree is < 2^31, checked at graph
// creation).  Otherwise (non-integer or borrowed weights) they are
// accumulated in fp32, exact for integer weights while every weighted degree
// is < 2^24.
//
// Argmax with the strict tie-break (Section 4.1.5: smallest label id among the
// most weighted): a candidate is encoded as key = sum + 1 (uint32; 0 means "no
// candidate"), the warp takes the max key and then the min label among lanes
// holding that key.  fp32 sums are non-negative, so their bit patterns order
// like the values and the same encoding applies.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "lpa_internal.h"

namespace lpa {

constexpr unsigned kFull = 0xffffffffu;

template <int WK>
struct Acc {
    using T = uint32_t;
};
template <>
struct Acc<W_F32> {
    using T = float;
};

template <int WK>
__device__ __forceinline__ typename Acc<WK>::T load_weight(const void* w, int64_t e) {
    if constexpr (WK == W_UNIT) {
        return 1u;
    } else if constexpr (WK == W_U32) {
        return __ldcs(static_cast<const uint32_t*>(w) + e);
    } else if constexpr (WK == W_U8) {
        return (uint32_t)__ldcs(static_cast<const unsigned char*>(w) + e);
    } else {
        return __ldcs(static_cast<const float*>(w) + e);
    }
}

__device__ __forceinline__ int32_t load_index(const int32_t* idx, int64_t e) {
    return __ldcs(idx + e);   // streamed once per sweep: evict-first
}

// Row indices that are read again when the vertex changes (neighbour marks).
__device__ __forceinline__ int32_t load_index_keep(const int32_t* idx, int64_t e) {
    return __ldg(idx + e);
}

// Marks vertex j unprocessed (Section 4.1.4), for the rows of the warp and
// block kernels: their neighbours are marked by many rows each (hubs by
// thousands), so the flag is read first and the store issued only while it is
// still 0.  A flag only goes 0 -> 1 during a pass (the next compaction clears
// it), so a stale 0 costs one redundant store, never a lost mark.  The
// low-degree kernels store unconditionally: there the load would sit on each
// thread's sequential path and save few stores.
__device__ __forceinline__ void mark_unprocessed(uint8_t* flags, int32_t j) {
    if (__ldcg(flags + j) == 0) flags[j] = 1;
}

// First synchronous sweep of a single graph whose rows repeat no neighbour:
// every label is still its vertex's id, so neighbour j carries label j and the
// sum K_{i->c} of Eq. 2 for each label is one entry's weight.  The kernels
// then skip the label gathers (and the wider ones the hash table).
template <bool ASYNC, bool BATCH>
__device__ __forceinline__ bool identity_sweep(const DevState& s) {
    if constexpr (ASYNC || BATCH) {
        return false;
    } else {
        return s.rows_distinct && s.ctrl->iter == 0;
    }
}

// The label vertex v starts with (Algorithm 1: C_i = i): its original id.
// Vertices may be stored in another order (lpa_graph_create's storage
// orders); labels are original ids whatever the order.
__device__ __forceinline__ int32_t initial_label(const DevState& s, int32_t v) {
    return s.orig ? __ldg(s.orig + v) : v;
}

// One candidate packed for a 64-bit max: sum key above, complemented tie key
// below, so the larger sum wins and then the smaller tie key.  0 = none.
__device__ __forceinline__ unsigned long long pack_candidate(uint32_t key, uint32_t tie) {
    return ((unsigned long long)key << 32) | (unsigned long long)(~tie);
}

__device__ __forceinline__ unsigned long long warp_max_u64(unsigned long long x) {
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long y = __shfl_xor_sync(kFull, x, o);
        x = y > x ? y : x;
    }
    return x;
}

// Whether this pass writes neighbour marks (Section 4.1.4).
__device__ __forceinline__ bool marks_on(const DevState& s, int flag_neighbours) {
    return flag_neighbours && !s.ctrl->skip_marks;
}

// L2 policy for data read once per sweep (the row indices streamed by the
// block kernels' bulk copies): evict first, so the stream does not push the
// gathered labels out of L2 (on R-MAT 27 the row kernels ran 10-19% faster).
__device__ __forceinline__ uint64_t l2_policy_evict_first() {
    uint64_t pol;
    asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}

// Sync mode reads labels that no thread writes during the sweep (read-only
// path); async mode reads labels other SMs update in place, so it bypasses L1.
// A vertex's own label is written only by the thread that scans it, so it may
// be read at any point of the sweep.
template <bool ASYNC>
__device__ __forceinline__ int32_t load_label(const int32_t* C, int32_t j) {
    if constexpr (ASYNC) {
        return __ldcg(C + j);
    } else {
        return __ldg(C + j);
    }
}

template <typename T>
__device__ __forceinline__ uint32_t sum_key(T s) {
    if constexpr (std::is_same<T, float>::value) {
        return __float_as_uint(s) + 1u;
    } else {
        return s + 1u;
    }
}

// SplitMix64 (Steele, Lea & Flood, OOPSLA 2014): the generator's output
// function applied to state x, the counter-based draw of the non-strict
// tie-break.
__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// A Feistel network on 2m-bit values (four rounds of SplitMix64): a
// pseudo-random bijection of [0, 2^(2m)).
__device__ __forceinline__ uint32_t feistel(uint32_t x, int m, uint64_t seed) {
    const uint32_t mask = (m >= 32) ? 0xffffffffu : ((1u << m) - 1u);
    uint32_t L = x >> m, R = x & mask;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const uint32_t f = (uint32_t)splitmix64(seed + ((uint64_t)r << 40) + R) & mask;
        const uint32_t t = L ^ f;
        L = R;
        R = t;
    }
    return (L << m) | R;
}

// Position of i in a pseudo-random permutation of [0, n) (n >= 1).  The
// network permutes [0, 2^(2m)) with 2^(2m) < 4n, so the walk (apply the
// permutation until the value falls below n) ends after a few steps.
__device__ __forceinline__ uint32_t shuffle_pos(uint32_t i, uint32_t n, uint64_t seed) {
    if (n <= 1) return 0;
    int k = 32 - __clz(n - 1);                 // bits of n - 1
    if (k & 1) ++k;
    const int m = k / 2;
    uint32_t x = i;
    do {
        x = feistel(x, m, seed);
    } while (x >= n);
    return x;
}

// Tie-break among the most weighted labels of one vertex (Section 4.1.5).
// Strict: the smallest label id.  Non-strict (a pseudo-random choice through a
// modulo of the label id, read as a rotation of the label space):
// for vertex i (graph-local id) in its graph's sweep t, r = SplitMix64((t <<
// 32) | i) mod n, and the label c minimising (c_local - r) mod n wins.  key()
// maps a label to the value minimised (a bijection on the graph's labels, so
// it identifies the label); label() undoes it.
struct TieRule {
    uint32_t r;
    uint32_t n;
    int32_t v0;
    bool rot;
    __device__ __forceinline__ uint32_t key(int32_t c) const {
        if (!rot) return (uint32_t)c;
        const uint32_t k = (uint32_t)(c - v0);
        return k >= r ? k - r : k + (n - r);
    }
    __device__ __forceinline__ int32_t label(uint32_t k) const {
        if (!rot) return (int32_t)k;
        uint32_t x = k + r;
        if (x >= n) x -= n;
        return v0 + (int32_t)x;
    }
};

// Rule for (stored) vertex v, drawn with its original id; ns and sweep (the
// single graph's 1-based sweep) are read from the control block once per
// kernel.  In a batch each graph counts its own sweeps.
__device__ __forceinline__ TieRule tie_rule(const DevState& s, bool ns, uint32_t sweep, int32_t v) {
    TieRule t;
    t.r = 0;
    t.n = 0;
    t.v0 = 0;
    t.rot = ns;
    if (!ns) return t;
    int64_t v0 = 0, n = s.N;
    if (s.G > 1) {
        const int32_t g = s.gid[v];
        v0 = s.g_begin[g];
        n = s.g_end[g] - v0;
        sweep = (uint32_t)s.iters[g] + 1u;
    }
    t.v0 = (int32_t)v0;
    t.n = (uint32_t)n;
    const int32_t vid = initial_label(s, v);       // the vertex's original id
    t.r = (uint32_t)(splitmix64(((uint64_t)sweep << 32) | (uint64_t)(vid - v0)) % (uint64_t)n);
    return t;
}

// Warp-wide argmax over (sum key, tie key): the largest sum key, then the
// smallest tie key.  Returns the winning tie key, or 0xffffffff when no lane
// holds a candidate (sum key == 0).  All 32 lanes must call.
__device__ __forceinline__ uint32_t warp_argmax_tie(uint32_t key, uint32_t tie) {
    const uint32_t m = __reduce_max_sync(kFull, key);
    if (m == 0) return 0xffffffffu;
    return __reduce_min_sync(kFull, key == m ? tie : 0xffffffffu);
}

__device__ __forceinline__ int ceil_log2(uint32_t x) {  // x >= 1
    return x <= 1 ? 0 : 32 - __clz(x - 1);
}

__device__ __forceinline__ uint32_t slot_of(int32_t label, int log_slots) {
    return ((uint32_t)label * 0x9E3779B1u) >> (32 - log_slots);
}

// Open-addressing insert-or-add into a table with 2^log_slots slots whose
// free slots hold kEmptyKey, probing at most max_probes slots.  Returns false
// if the label is not in the probed slots and none of them was free.
// `created` receives the slot this call claimed for a new label, else -1, so
// callers can list the slots a row filled and scan only those.
template <typename T>
__device__ __forceinline__ bool table_insert(int32_t* keys, T* vals, int log_slots, int32_t label, T w,
                                             uint32_t max_probes, int& created) {
    const uint32_t mask = (1u << log_slots) - 1u;
    uint32_t h = slot_of(label, log_slots);
    volatile int32_t* vkeys = keys;
    created = -1;
    for (uint32_t p = 0; p < max_probes; ++p) {
        int32_t k = vkeys[h];
        if (k == label) {
            atomicAdd(vals + h, w);
            return true;
        }
        if (k == kEmptyKey) {
            int32_t old = atomicCAS(keys + h, kEmptyKey, label);
            if (old == kEmptyKey || old == label) {
                if (old == kEmptyKey) created = (int)h;
                atomicAdd(vals + h, w);
                return true;
            }
        }
        h = (h + 1u) & mask;
    }
    return false;
}

// Insert-or-add probing the whole table.  Callers size the table at >= 2 x
// the distinct labels it can receive, so a free slot always exists; the probe
// is still bounded by the table size and reports failure instead of looping.
template <typename T>
__device__ __forceinline__ bool table_add(int32_t* keys, T* vals, int log_slots, int32_t label, T w) {
    int created;
    return table_insert<T>(keys, vals, log_slots, label, w, 1u << log_slots, created);
}

// Bounded variant: gives up after max_probes occupied slots; returns false if
// the label is not in the table and could not be placed (the caller then
// treats the row as overflowing the table).
template <typename T>
__device__ __forceinline__ bool table_add_bounded(int32_t* keys, T* vals, int log_slots, int32_t label, T w,
                                                  int max_probes) {
    int created;
    return table_insert<T>(keys, vals, log_slots, label, w, (uint32_t)max_probes, created);
}

__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }

__device__ __forceinline__ unsigned lanes_below() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Batched runs: dN of each graph, aggregated over the lanes of a warp that
// changed a vertex of the same graph.  All 32 lanes must call.
template <bool BATCH>
__device__ __forceinline__ void count_graph_changes(const DevState& s, bool changed, int32_t v) {
    if constexpr (BATCH) {
        const unsigned m = __ballot_sync(kFull, changed);
        if (changed) {
            const int32_t g = s.gid[v];
            const unsigned peers = __match_any_sync(m, g);
            if (lane_id() == (unsigned)(__ffs(peers) - 1)) atomicAdd(&s.dN[g], (unsigned long long)__popc(peers));
        }
    }
}

// Per-thread counts of changed vertices (and their CSR entries) are summed
// over the block and added to the bin's counters with one atomic each.  All
// threads of the block must call, once, at the end of the kernel.
__device__ __forceinline__ void flush_bin_counts(const DevState& s, int bin, unsigned long long changed,
                                                 unsigned long long changed_entries) {
    __shared__ unsigned long long red[2][32];
    for (int o = 16; o > 0; o >>= 1) {
        changed += __shfl_xor_sync(kFull, changed, o);
        changed_entries += __shfl_xor_sync(kFull, changed_entries, o);
    }
    const int w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    if (lane_id() == 0) {
        red[0][w] = changed;
        red[1][w] = changed_entries;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long a = 0, b = 0;
        for (int q = 0; q < nw; ++q) {
            a += red[0][q];
            b += red[1][q];
        }
        if (a) {
            atomicAdd(&s.ctrl->bin_changed[bin], a);
            atomicAdd(&s.ctrl->bin_changed_entries[bin], b);
            atomicAdd(&s.ctrl->pass_changed_entries, b);
        }
    }
}

// Frontier of bin b for the current sweep: the static list when the sweep is
// dense, else the compacted list; both live in the bin's slot region.
struct BinView {
    const int32_t* list;   // already offset to the bin's region
    int32_t* chg;          // sync-mode change marks, same offset
    unsigned cnt;
};

__device__ __forceinline__ BinView bin_view(const DevState& s, int b) {
    const int buf = s.ctrl->rd;
    BinView bv;
    const int64_t base = s.bin_base[b];
    bv.list = (s.ctrl->dense[buf] ? s.slist : s.flist) + base;
    bv.chg = s.chg + base;
    bv.cnt = s.ctrl->bin_cnt[buf][b];
    return bv;
}

// Label buffers of the current sweep: C (read) and Cn (sync modes write it;
// async mode updates C in place).
struct Labels {
    int32_t* C;
    int32_t* Cn;
    bool dense;
};

__device__ __forceinline__ Labels labels_of(const DevState& s) {
    const int cb = s.ctrl->cbuf;
    Labels L;
    L.C = s.lab[cb];
    L.Cn = s.lab[cb ^ 1];
    L.dense = s.ctrl->dense[s.ctrl->rd] != 0;
    return L;
}

// Outcome of one scanned vertex.  Async: in-place write on change.  Sync,
// dense sweep: the next buffer receives every scanned vertex's label (the
// buffers flip after the sweep).  Sync, sparse sweep: only changed vertices
// are written and their list slot is marked for the apply step.
template <bool ASYNC>
__device__ __forceinline__ void record_label(const Labels& L, int32_t* chg_slot, int32_t v, int32_t own,
                                             int32_t best, bool changed) {
    if constexpr (ASYNC) {
        if (changed) L.C[v] = best;
    } else {
        if (L.dense) {
            L.Cn[v] = changed ? best : own;
        } else {
            if (changed) L.Cn[v] = best;
            *chg_slot = changed ? v : -1;
        }
    }
}

}  // namespace lpa
