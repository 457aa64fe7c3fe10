// lpa_device.cuh -- device helpers shared by the sweep kernels.
//
// Weight sums: for graphs whose weights are integers (or unit) the per-label
// sums K_{i->c} are accumulated in uint32 (exact, any order, as long as every
// weighted degree is < 2^24 -- checked at graph creation).  Otherwise they
// are accumulated in fp32.
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
    } else {
        return __ldcs(static_cast<const float*>(w) + e);
    }
}

__device__ __forceinline__ int32_t load_index(const int32_t* idx, int64_t e) {
    return __ldcs(idx + e);   // streamed once per sweep: evict-first
}

// Sync mode reads labels that no thread writes during the sweep (read-only
// path); async mode reads labels other SMs update in place, so it bypasses L1.
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

// Warp-wide argmax over (key, label): returns the winning label, or -1 when no
// lane holds a candidate (key == 0).  All 32 lanes must call.
__device__ __forceinline__ int32_t warp_argmax(uint32_t key, int32_t label) {
    uint32_t m = __reduce_max_sync(kFull, key);
    if (m == 0) return -1;
    uint32_t cand = (key == m) ? (uint32_t)label : 0xffffffffu;
    return (int32_t)__reduce_min_sync(kFull, cand);
}

__device__ __forceinline__ int ceil_log2(uint32_t x) {  // x >= 1
    return x <= 1 ? 0 : 32 - __clz(x - 1);
}

__device__ __forceinline__ uint32_t slot_of(int32_t label, int log_slots) {
    return ((uint32_t)label * 0x9E3779B1u) >> (32 - log_slots);
}

// Open-addressing insert-or-add into a table with 2^log_slots slots whose
// free slots hold kEmptyKey.  Callers size the table at >= 2 x the distinct
// labels it can receive, so a free slot always exists; the probe is still
// bounded by the table size and reports failure instead of looping.
template <typename T>
__device__ __forceinline__ bool table_add(int32_t* keys, T* vals, int log_slots, int32_t label, T w) {
    const uint32_t mask = (1u << log_slots) - 1u;
    uint32_t h = slot_of(label, log_slots);
    volatile int32_t* vkeys = keys;
    for (uint32_t p = 0; p <= mask; ++p) {
        int32_t k = vkeys[h];
        if (k == label) {
            atomicAdd(vals + h, w);
            return true;
        }
        if (k == kEmptyKey) {
            int32_t old = atomicCAS(keys + h, kEmptyKey, label);
            if (old == kEmptyKey || old == label) {
                atomicAdd(vals + h, w);
                return true;
            }
        }
        h = (h + 1u) & mask;
    }
    return false;
}

// Bounded variant: gives up after max_probes occupied slots; returns false if
// the label is not in the table and could not be placed.  Keys are never
// removed while a vertex is being scanned, so a label that failed once fails
// again: every label lives in exactly one of the shared and spill tables.
template <typename T>
__device__ __forceinline__ bool table_add_bounded(int32_t* keys, T* vals, int log_slots, int32_t label, T w,
                                                  int max_probes) {
    const uint32_t mask = (1u << log_slots) - 1u;
    uint32_t h = slot_of(label, log_slots);
    volatile int32_t* vkeys = keys;
    for (int p = 0; p < max_probes; ++p) {
        int32_t k = vkeys[h];
        if (k == label) {
            atomicAdd(vals + h, w);
            return true;
        }
        if (k == kEmptyKey) {
            int32_t old = atomicCAS(keys + h, kEmptyKey, label);
            if (old == kEmptyKey || old == label) {
                atomicAdd(vals + h, w);
                return true;
            }
        }
        h = (h + 1u) & mask;
    }
    return false;
}

__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }

// Per-warp bookkeeping of one processed slot per lane: dN (per graph when
// batched), per-bin changed counts and, in sync mode, the changed list.
// All 32 lanes must call.
template <bool ASYNC, bool BATCH>
__device__ __forceinline__ void account_changes(const DevState& s, int bin, bool changed, int32_t v,
                                                int64_t deg) {
    const unsigned lane = lane_id();
    const unsigned m = __ballot_sync(kFull, changed);
    if (m == 0) return;
    const unsigned leader = __ffs(m) - 1;
    unsigned long long deg_sum = __reduce_add_sync(kFull, changed ? (unsigned)deg : 0u);
    if (lane == leader) {
        atomicAdd(&s.ctrl->bin_changed[bin], (unsigned long long)__popc(m));
        atomicAdd(&s.ctrl->bin_changed_entries[bin], deg_sum);
    }
    if constexpr (BATCH) {
        if (changed) {
            int32_t g = s.gid[v];
            unsigned peers = __match_any_sync(m, g);
            if (lane == __ffs(peers) - 1) atomicAdd(&s.dN[g], (unsigned long long)__popc(peers));
        }
    }
    if constexpr (!ASYNC) {
        unsigned base = 0;
        if (lane == leader) base = atomicAdd(&s.ctrl->chg_cnt, (unsigned)__popc(m));
        base = __shfl_sync(kFull, base, leader);
        if (changed) s.chg_list[base + __popc(m & ((1u << lane) - 1u))] = v;
    }
}

// Result write for a vertex whose label changed.
template <bool ASYNC>
__device__ __forceinline__ void write_label(const DevState& s, int32_t v, int32_t c) {
    if constexpr (ASYNC) {
        s.C[v] = c;
    } else {
        s.Cnew[v] = c;
    }
}

}  // namespace lpa
