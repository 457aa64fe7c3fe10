// lpa_api.cu -- the C ABI of include/lpa.h: handle lifetime, validation,
// construction of the device-side loop (a CUDA graph whose WHILE node repeats
// one sweep of Algorithm 1 until the device sets the condition to 0), runs,
// modularity and the autotuner.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <chrono>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/lpa.h"
#include "lpa_internal.h"

using namespace lpa;

static_assert(LPA_MAX_RECORDED_ITERS == kMaxHist, "history depth mismatch");
static_assert(LPA_BINS == kBins, "bin count mismatch");

namespace {

thread_local std::string g_last_error;

lpa_status fail(lpa_status st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return st;
}

lpa_status cuda_fail(cudaError_t err, const char* where) {
    if (err == cudaErrorMemoryAllocation)
        return fail(LPA_ERR_OUT_OF_MEMORY, "%s: %s", where, cudaGetErrorString(err));
    return fail(LPA_ERR_CUDA, "%s: %s", where, cudaGetErrorString(err));
}

#define LPA_CUDA(call)                                        \
    do {                                                      \
        cudaError_t err__ = (call);                           \
        if (err__ != cudaSuccess) return cuda_fail(err__, #call); \
    } while (0)

int64_t pow2ceil(int64_t x) {
    int64_t p = 1;
    while (p < x) p <<= 1;
    return p;
}

// ------------------------------------------------------------ memory pool --
// Device memory of graphs and batches comes from one stream-ordered pool per
// device that keeps freed pages mapped (no release threshold): creating a
// graph after another was destroyed reuses those pages instead of mapping new
// ones and destroying one does not unmap.  lpa_release_cached_memory() hands
// the cached pages back to the driver.  Allocations and frees are issued on
// the pool's own stream and waited for, so memory is usable from any stream
// on return and a free never races a later allocation.
constexpr int kMaxPoolDevices = 64;
struct DevicePool {
    cudaMemPool_t pool = nullptr;
    cudaStream_t st = nullptr;
};
std::mutex g_pool_mu;
DevicePool g_pools[kMaxPoolDevices];

cudaError_t pool_of(int dev, DevicePool** out) {
    if (dev < 0 || dev >= kMaxPoolDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_pool_mu);
    DevicePool& P = g_pools[dev];
    if (!P.pool) {
        cudaMemPoolProps props{};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t pool = nullptr;
        cudaError_t e = cudaMemPoolCreate(&pool, &props);
        if (e != cudaSuccess) return e;
        uint64_t keep = ~0ull;
        e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        cudaStream_t st = nullptr;
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            cudaMemPoolDestroy(pool);
            return e;
        }
        P.pool = pool;
        P.st = st;
    }
    *out = &P;
    return cudaSuccess;
}

cudaError_t pool_alloc(int dev, void** p, size_t bytes) {
    DevicePool* P = nullptr;
    cudaError_t e = pool_of(dev, &P);
    if (e == cudaSuccess) e = cudaMallocFromPoolAsync(p, bytes, P->pool, P->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(P->st);
    return e;
}

// Frees a list of pool allocations once all work on the device is done (the
// same guarantee cudaFree gives).
void pool_free_all(int dev, std::vector<void*>& ptrs) {
    if (ptrs.empty()) return;
    int cur = 0;
    cudaGetDevice(&cur);
    if (cur != dev) cudaSetDevice(dev);
    DevicePool* P = nullptr;
    if (pool_of(dev, &P) == cudaSuccess) {
        cudaDeviceSynchronize();
        for (void* q : ptrs) cudaFreeAsync(q, P->st);
        cudaStreamSynchronize(P->st);
    }
    ptrs.clear();
    if (cur != dev) cudaSetDevice(cur);
}

struct Engine {
    int device = 0;
    int sms = 1;
    DevState s{};
    std::vector<void*> owned;        // pool allocations freed at destroy
    unsigned* static_counts = nullptr;             // static-list scratch
    unsigned long long* static_ents = nullptr;
    unsigned long long* cap_scratch = nullptr;     // [3] overflow capacity sums
    std::vector<void*> ovf_scratch;                // sliced overflow path: pairs, counts, offsets
    int32_t* idx_owned = nullptr;
    bool borrowed = false;
    bool weighted = false;
    bool exact = false;
    int64_t max_degree = 0;
    int64_t device_bytes = 0;
    lpa_config cfg{4, 128, 512, 2048, 500};
    Overflow* ovf = nullptr;
    cudaGraph_t graph[6] = {};         // per mode, strict (0..2) and non-strict (3..5)
    cudaGraphExec_t exec[6] = {};
    cudaStream_t cap_top = nullptr, cap_body = nullptr;
    // modularity scratch
    double* Sigma = nullptr;
    ModAccum* acc = nullptr;
    // host mirrors
    std::vector<int64_t> vtx_off_host;
    std::vector<int64_t> edge_off_host;
    unsigned long long* hist_d = nullptr;          // degree histogram scratch (autotuner)
    int order = kOrderCaller;                      // storage order of the vertices (StorageOrder)
    int32_t* tune_out = nullptr;                   // labels of the autotuner's timed runs
    int64_t runs_total = 0;          // lpa_run calls that launched the device loop
};

lpa_status dalloc(Engine& E, void** p, size_t bytes) {
    if (bytes == 0) bytes = 16;
    cudaError_t err = pool_alloc(E.device, p, bytes);
    if (err != cudaSuccess) {
        cudaGetLastError();
        return err == cudaErrorMemoryAllocation ? fail(LPA_ERR_OUT_OF_MEMORY, "device memory: %zu bytes", bytes)
                                                : cuda_fail(err, "cudaMallocFromPoolAsync");
    }
    E.owned.push_back(*p);
    E.device_bytes += (int64_t)bytes;
    return LPA_OK;
}

template <typename T>
lpa_status dalloc_t(Engine& E, T** p, size_t count) {
    return dalloc(E, reinterpret_cast<void**>(p), count * sizeof(T));
}

void destroy_graphs(Engine& E) {
    for (int m = 0; m < 6; ++m) {
        if (E.exec[m]) cudaGraphExecDestroy(E.exec[m]);
        if (E.graph[m]) cudaGraphDestroy(E.graph[m]);
        E.exec[m] = nullptr;
        E.graph[m] = nullptr;
    }
}

void engine_free(Engine& E) {
    destroy_graphs(E);
    if (E.cap_top) cudaStreamDestroy(E.cap_top);
    if (E.cap_body) cudaStreamDestroy(E.cap_body);
    if (E.ovf) E.owned.push_back(E.ovf);
    E.ovf = nullptr;
    for (void* p : E.ovf_scratch) E.owned.push_back(p);
    E.ovf_scratch.clear();
    pool_free_all(E.device, E.owned);
}

// Grid sizes of the block bins, and the overflow list of the last bin (one
// entry per vertex of that bin at most).
lpa_status setup_blocks(Engine& E, cudaStream_t st) {
    std::vector<void*> old;
    if (E.ovf) old.push_back(E.ovf);
    for (void* p : E.ovf_scratch) old.push_back(p);
    pool_free_all(E.device, old);
    E.ovf = nullptr;
    E.ovf_scratch.clear();
    const size_t n = std::max<size_t>(E.s.bin_static[kBins - 1], 1);
    void* p = nullptr;
    cudaError_t err = pool_alloc(E.device, &p, n * sizeof(Overflow));
    if (err != cudaSuccess) return cuda_fail(err, "overflow list");
    E.ovf = static_cast<Overflow*>(p);
    E.s.ovf = E.ovf;
    // sliced overflow path: scratch for every last-bin row that can overflow
    int64_t pairs = 0, counts = 0, rows = 0;
    err = ovf_capacity(E.s, st, E.sms, &pairs, &counts, &rows, E.cap_scratch);
    if (err != cudaSuccess) return cuda_fail(err, "overflow capacity");
    void* q[3] = {nullptr, nullptr, nullptr};
    const size_t bytes[3] = {(size_t)std::max<int64_t>(pairs, 1) * sizeof(uint2),
                             (size_t)std::max<int64_t>(counts, 1) * sizeof(uint32_t),
                             (size_t)std::max<int64_t>(counts, 1) * sizeof(uint32_t)};
    for (int k = 0; k < 3; ++k) {
        if ((err = pool_alloc(E.device, &q[k], bytes[k])) != cudaSuccess) {
            for (int j = 0; j < k; ++j) E.ovf_scratch.push_back(q[j]);
            cudaGetLastError();
            return fail(LPA_ERR_OUT_OF_MEMORY, "overflow scratch: %zu bytes", bytes[k]);
        }
        E.ovf_scratch.push_back(q[k]);
    }
    E.s.ovf_pairs = static_cast<uint2*>(q[0]);
    E.s.ovf_cnt = static_cast<uint32_t*>(q[1]);
    E.s.ovf_off = static_cast<uint32_t*>(q[2]);
    E.s.ovf_pairs_cap = pairs;
    E.s.ovf_cnt_cap = counts;
    E.s.ovf_possible = rows > 0 ? 1 : 0;
    return LPA_OK;
}

void apply_config_fields(Engine& E) {
    E.s.small_max = E.cfg.small_max;
    E.s.warp_max = E.cfg.warp_max;
    E.s.mid_max = E.cfg.mid_max;
    E.s.large_max = E.cfg.large_max;
    E.s.warp_slots = (int32_t)pow2ceil(2 * (int64_t)E.cfg.warp_max);
    E.s.block_slots[0] = (int32_t)pow2ceil(2 * (int64_t)E.cfg.mid_max);
    E.s.block_slots[1] = (int32_t)pow2ceil(2 * (int64_t)E.cfg.large_max);
    E.s.block_slots[2] = kLargeSlots;
    E.s.dense_permille = E.cfg.dense_permille;
}

lpa_status check_config(const lpa_config& c) {
    if (c.small_max < 1 || c.small_max > 8) return fail(LPA_ERR_INVALID_ARG, "small_max must be in [1, 8]");
    if (c.warp_max <= c.small_max || c.warp_max > 256)
        return fail(LPA_ERR_INVALID_ARG, "warp_max must be in (small_max, 256]");
    if (c.mid_max <= c.warp_max || c.mid_max > 2048)
        return fail(LPA_ERR_INVALID_ARG, "mid_max must be in (warp_max, 2048]");
    if (c.large_max <= c.mid_max || c.large_max > 4096)
        return fail(LPA_ERR_INVALID_ARG, "large_max must be in (mid_max, 4096]");
    if (c.dense_permille < 0 || c.dense_permille > 1001)
        return fail(LPA_ERR_INVALID_ARG, "dense_permille must be in [0, 1001]");
    return LPA_OK;
}

// Working state of an engine whose N, G and CSR fields are set: label
// buffers, flags, frontier bitmap and lists, change marks, control block and
// per-graph counters, and the static-list scratch.
lpa_status alloc_state(Engine& E, cudaStream_t st) {
    lpa_status rs;
    const int64_t n = E.s.N;
    const int32_t G = E.s.G;
    const size_t N1 = (size_t)std::max<int64_t>(n, 1);
    if ((rs = dalloc_t(E, &E.s.lab[0], N1)) != LPA_OK) return rs;
    if ((rs = dalloc_t(E, &E.s.lab[1], N1)) != LPA_OK) return rs;
    if ((rs = dalloc_t(E, &E.s.flags, N1 + 16)) != LPA_OK) return rs;
    if ((rs = dalloc_t(E, &E.s.fr_bits, N1 / 16 + 1)) != LPA_OK) return rs;
    if ((rs = dalloc_t(E, &E.s.slist, N1)) != LPA_OK) return rs;
    if ((rs = dalloc_t(E, &E.s.flist, N1)) != LPA_OK) return rs;
    if ((rs = dalloc_t(E, &E.s.chg, N1)) != LPA_OK) return rs;
    if ((rs = dalloc_t(E, &E.s.ctrl, 1)) != LPA_OK) return rs;
    if ((rs = dalloc_t(E, &E.s.dN, (size_t)G)) != LPA_OK) return rs;
    if ((rs = dalloc_t(E, &E.s.done, (size_t)G)) != LPA_OK) return rs;
    if ((rs = dalloc_t(E, &E.s.iters, (size_t)G)) != LPA_OK) return rs;
    if ((rs = dalloc_t(E, &E.s.exit_reason, (size_t)G)) != LPA_OK) return rs;
    if ((rs = dalloc_t(E, &E.s.hist_changed, (size_t)G * kMaxHist)) != LPA_OK) return rs;
    LPA_CUDA(cudaMemsetAsync(E.s.flags, 0, N1 + 16, st));
    LPA_CUDA(cudaMemsetAsync(E.s.ctrl, 0, sizeof(Ctrl), st));
    LPA_CUDA(cudaMemsetAsync(E.s.hist_changed, 0, (size_t)G * kMaxHist * 8, st));
    apply_config_fields(E);
    const size_t sblk = (size_t)std::max<int64_t>(static_scratch_blocks(n), 1) * kBins;
    if ((rs = dalloc_t(E, &E.static_counts, sblk)) != LPA_OK) return rs;
    if ((rs = dalloc_t(E, &E.static_ents, sblk)) != LPA_OK) return rs;
    if ((rs = dalloc_t(E, &E.cap_scratch, 3)) != LPA_OK) return rs;
    return LPA_OK;
}

// Frees one of the engine's own allocations before the engine is destroyed.
void release_owned(Engine& E, void* p, int64_t bytes) {
    auto it = std::find(E.owned.begin(), E.owned.end(), p);
    if (it == E.owned.end()) return;
    E.owned.erase(it);
    std::vector<void*> one{p};
    pool_free_all(E.device, one);
    E.device_bytes -= bytes;
}

// Stores the vertices in `kind` order (lpa_reorder.cu): orig, and the CSR
// rewritten in that order, replace the engine's arrays (the caller's arrays
// of a borrowed graph are left as they are); the static lists are rebuilt.
lpa_status apply_order(Engine& E, int kind, cudaStream_t st) {
    const int64_t n = E.s.N, nnz = E.s.E;
    lpa_status rs;
    int32_t *orig = nullptr, *inv = nullptr, *idx2 = nullptr;
    unsigned* scr = nullptr;
    int64_t* off2 = nullptr;
    void* w2 = nullptr;
    const int wbytes = E.s.weight_kind == W_UNIT ? 0 : E.s.weight_kind == W_U8 ? 1 : 4;
    const int64_t scr_words = reorder_scratch_words(n);
    if ((rs = dalloc_t(E, &orig, (size_t)n)) != LPA_OK) return rs;
    if ((rs = dalloc_t(E, &inv, (size_t)n)) != LPA_OK) return rs;
    if ((rs = dalloc_t(E, &scr, (size_t)scr_words)) != LPA_OK) return rs;
    LPA_CUDA(reorder_positions(kind, E.s.off, E.s.vtx_off, E.s.gid, E.s.G, n, 0x5EEDC0DE2312ull, orig, inv, scr, st,
                               E.sms));
    if ((rs = dalloc_t(E, &off2, (size_t)n + 1)) != LPA_OK) return rs;
    if ((rs = dalloc_t(E, &idx2, (size_t)std::max<int64_t>(nnz, 1))) != LPA_OK) return rs;
    if (wbytes && (rs = dalloc(E, &w2, (size_t)std::max<int64_t>(nnz, 1) * wbytes)) != LPA_OK) return rs;
    LPA_CUDA(reorder_rows(orig, inv, E.s.off, E.s.idx, E.s.w, wbytes, n, off2, idx2, w2,
                          reinterpret_cast<unsigned long long*>(scr), st, E.sms));
    release_owned(E, inv, n * 4);
    release_owned(E, scr, scr_words * 4);
    // the library's own copies of the caller's order (borrowed arrays are not
    // among the engine's allocations and stay untouched)
    release_owned(E, const_cast<int64_t*>(E.s.off), (n + 1) * 8);
    release_owned(E, const_cast<int32_t*>(E.s.idx), nnz * 4);
    if (E.s.w) release_owned(E, const_cast<void*>(E.s.w), nnz * wbytes);
    E.s.off = off2;
    E.s.off_end = off2 + 1;
    E.s.idx = idx2;
    E.s.w = w2;
    E.s.orig = orig;
    E.order = kind;
    LPA_CUDA(build_static_lists(E.s, st, E.static_counts, E.static_ents));
    return LPA_OK;
}

// Common creation path: G graphs (G == 1 for lpa_graph_create).
lpa_status engine_create(Engine& E, int32_t G, const int64_t* vtx_off_h, const int64_t* edge_off_h, int64_t n,
                         int64_t nnz, const int64_t* offsets, const int32_t* indices, const float* weights,
                         uint32_t flags, cudaStream_t st) {
    const bool dev = (flags & LPA_DEVICE_PTRS) != 0;
    const bool borrow = (flags & LPA_BORROW) != 0;
    const uint32_t known = LPA_DEVICE_PTRS | LPA_BORROW | LPA_REORDER_DEGREE | LPA_REORDER_SHUFFLE | LPA_KEEP_ORDER;
    if (flags & ~known) return fail(LPA_ERR_INVALID_ARG, "unknown flag bits");
    const int n_orders = ((flags & LPA_REORDER_DEGREE) ? 1 : 0) + ((flags & LPA_REORDER_SHUFFLE) ? 1 : 0) +
                         ((flags & LPA_KEEP_ORDER) ? 1 : 0);
    if (n_orders > 1) return fail(LPA_ERR_INVALID_ARG, "at most one storage-order flag");
    if ((flags & LPA_REORDER_DEGREE) && G > 1)
        return fail(LPA_ERR_INVALID_ARG, "LPA_REORDER_DEGREE is for single graphs");
    int order = kOrderCaller;
    if (flags & LPA_REORDER_DEGREE) order = kOrderDegree;
    else if ((flags & LPA_REORDER_SHUFFLE) || (G > 1 && !(flags & LPA_KEEP_ORDER))) order = kOrderShuffle;
    if (borrow && !dev) return fail(LPA_ERR_INVALID_ARG, "LPA_BORROW needs LPA_DEVICE_PTRS");
    if (borrow && G > 1) return fail(LPA_ERR_INVALID_ARG, "LPA_BORROW is not accepted for batches");
    if (n < 0 || n > 0x7fffffffLL) return fail(LPA_ERR_INVALID_ARG, "n out of range [0, 2^31-1]");
    if (nnz < 0) return fail(LPA_ERR_INVALID_ARG, "nnz < 0");
    if (!offsets) return fail(LPA_ERR_INVALID_ARG, "offsets is NULL");
    if (nnz > 0 && !indices) return fail(LPA_ERR_INVALID_ARG, "indices is NULL");

    LPA_CUDA(cudaGetDevice(&E.device));
    LPA_CUDA(cudaDeviceGetAttribute(&E.sms, cudaDevAttrMultiProcessorCount, E.device));
    E.s.N = n;
    E.s.E = nnz;
    E.s.G = G;
    E.weighted = weights != nullptr;
    E.borrowed = borrow;
    E.vtx_off_host.assign(vtx_off_h, vtx_off_h + G + 1);
    E.edge_off_host.assign(edge_off_h, edge_off_h + G + 1);
    const cudaMemcpyKind kind = dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    lpa_status rs;

    // The graph-capture streams double as the copy and helper streams here.
    LPA_CUDA(cudaStreamCreateWithFlags(&E.cap_top, cudaStreamNonBlocking));
    LPA_CUDA(cudaStreamCreateWithFlags(&E.cap_body, cudaStreamNonBlocking));

    // CSR.  Host arrays are copied in stages: the offsets first, then indices
    // and weights in chunks on the copy stream, each chunk's entries checked
    // as soon as it lands, while the static bin lists (which need only the
    // offsets) are built on the helper stream -- creation then costs about
    // the copy alone.
    // The sweep kernels copy index rows with 16-byte bulk copies: borrowed
    // indices that are not 16-byte aligned are copied like unborrowed ones.
    const bool idx_copy = borrow && nnz > 0 && (reinterpret_cast<uintptr_t>(indices) & 15u) != 0;
    const bool staged = !borrow && !dev && nnz > 0;
    int64_t* off_d = nullptr;
    int32_t* idx_d = nullptr;
    float* w_d = nullptr;
    if (borrow) {
        off_d = const_cast<int64_t*>(offsets);
        idx_d = const_cast<int32_t*>(indices);
        w_d = const_cast<float*>(weights);
        if (idx_copy) {
            if ((rs = dalloc_t(E, &idx_d, (size_t)nnz)) != LPA_OK) return rs;
            LPA_CUDA(cudaMemcpyAsync(idx_d, indices, (size_t)nnz * 4, cudaMemcpyDeviceToDevice, st));
        }
    } else {
        if ((rs = dalloc_t(E, &off_d, (size_t)n + 1)) != LPA_OK) return rs;
        if ((rs = dalloc_t(E, &idx_d, (size_t)nnz)) != LPA_OK) return rs;
        if (weights && (rs = dalloc_t(E, &w_d, (size_t)nnz)) != LPA_OK) return rs;
        LPA_CUDA(cudaMemcpyAsync(off_d, offsets, ((size_t)n + 1) * 8, kind, st));
        if (!staged && nnz) {
            LPA_CUDA(cudaMemcpyAsync(idx_d, indices, (size_t)nnz * 4, kind, st));
            if (weights) LPA_CUDA(cudaMemcpyAsync(w_d, weights, (size_t)nnz * 4, kind, st));
        }
    }
    int64_t* vo_d = nullptr;
    int64_t* eo_d = nullptr;
    if ((rs = dalloc_t(E, &vo_d, (size_t)G + 1)) != LPA_OK) return rs;
    if ((rs = dalloc_t(E, &eo_d, (size_t)G + 1)) != LPA_OK) return rs;
    LPA_CUDA(cudaMemcpyAsync(vo_d, vtx_off_h, ((size_t)G + 1) * 8, cudaMemcpyHostToDevice, st));
    LPA_CUDA(cudaMemcpyAsync(eo_d, edge_off_h, ((size_t)G + 1) * 8, cudaMemcpyHostToDevice, st));
    int32_t* gid_d = nullptr;
    if (G > 1) {
        if ((rs = dalloc_t(E, &gid_d, (size_t)std::max<int64_t>(n, 1))) != LPA_OK) return rs;
        LPA_CUDA(launch_fill_gid(vo_d, G, n, gid_d, st, E.sms));
    }
    E.s.off = off_d;
    E.s.off_end = off_d + 1;
    E.s.idx = idx_d;
    E.s.gid = gid_d;
    E.s.vtx_off = vo_d;
    E.s.g_begin = vo_d;
    E.s.g_end = vo_d + 1;

    if ((rs = alloc_state(E, st)) != LPA_OK) return rs;

    // validation (and, for batches, local -> global index rewrite in our copy)
    ValidateResult* vr_d = nullptr;
    if ((rs = dalloc_t(E, &vr_d, 1)) != LPA_OK) return rs;
    LPA_CUDA(cudaMemsetAsync(vr_d, 0, sizeof(ValidateResult), st));
    cudaEvent_t ev = nullptr;
    LPA_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    cudaError_t ce = cudaEventRecord(ev, st);                    // offsets and working state ready
    if (ce == cudaSuccess) ce = cudaStreamWaitEvent(E.cap_body, ev, 0);
    const int rewrite = G > 1 ? 1 : 0;
    if (staged) {
        constexpr int64_t kChunk = 1LL << 24;                    // entries per staged copy
        for (int64_t e0 = 0; e0 < nnz && ce == cudaSuccess; e0 += kChunk) {
            const int64_t c = std::min<int64_t>(kChunk, nnz - e0);
            ce = cudaMemcpyAsync(idx_d + e0, indices + e0, (size_t)c * 4, cudaMemcpyHostToDevice, E.cap_top);
            if (ce == cudaSuccess && weights)
                ce = cudaMemcpyAsync(w_d + e0, weights + e0, (size_t)c * 4, cudaMemcpyHostToDevice, E.cap_top);
            if (ce == cudaSuccess) ce = cudaEventRecord(ev, E.cap_top);
            if (ce == cudaSuccess) ce = cudaStreamWaitEvent(st, ev, 0);
            if (ce == cudaSuccess)
                ce = launch_validate_entries(idx_d, w_d, n, nnz, e0, e0 + c, vo_d, eo_d, G, rewrite, idx_d, vr_d, st,
                                             E.sms);
        }
    } else if (ce == cudaSuccess && n > 0) {
        ce = launch_validate_entries(idx_d, w_d, n, nnz, 0, nnz, vo_d, eo_d, G, rewrite, idx_d, vr_d, st, E.sms);
    }
    cudaEventDestroy(ev);                                        // released once its waits have passed
    LPA_CUDA(ce);
    // static bin lists on the helper stream, meanwhile (blocks this thread
    // until they are built; the copies and checks above keep running)
    LPA_CUDA(build_static_lists(E.s, E.cap_body, E.static_counts, E.static_ents));
    if (n > 0) LPA_CUDA(launch_validate_rows(off_d, idx_d, w_d, n, nnz, vo_d, eo_d, gid_d, G, vr_d, st, E.sms));
    ValidateResult vr{};
    LPA_CUDA(cudaMemcpyAsync(&vr, vr_d, sizeof(vr), cudaMemcpyDeviceToHost, st));
    LPA_CUDA(cudaStreamSynchronize(st));
    if (n == 0 && nnz != 0) return fail(LPA_ERR_INVALID_GRAPH, "n == 0 but nnz != 0");
    if (vr.c[0]) return fail(LPA_ERR_INVALID_GRAPH, "%u rows have invalid offsets", vr.c[0]);
    if (vr.c[1]) return fail(LPA_ERR_INVALID_GRAPH, "%u indices out of range", vr.c[1]);
    if (vr.c[2]) return fail(LPA_ERR_INVALID_GRAPH, "%u weights negative or not finite", vr.c[2]);
    E.max_degree = (int64_t)vr.max_degree;
    // rows without a repeated neighbour (each strictly increasing): the first
    // synchronous sweep, where every label is still the vertex's own id, is a
    // max-weight reduction over each row
    E.s.rows_distinct = (G == 1 && vr.desc_all == vr.desc_row_starts) ? 1 : 0;

    // weight representation: integer sums when every sum is an exact integer
    if (!weights) {
        E.exact = vr.c[5] == 0;
        E.s.weight_kind = E.exact ? W_UNIT : W_F32;
        if (!E.exact) return fail(LPA_ERR_INVALID_GRAPH, "a vertex has degree >= 2^31");
    } else if (!borrow && vr.c[3] == 0 && vr.c[5] == 0) {
        float wmax = 0.f;
        memcpy(&wmax, &vr.max_weight_bits, sizeof(wmax));
        E.exact = true;
        if (wmax <= 255.f && nnz > 0) {
            // one byte per entry: the float copy is converted, then freed
            unsigned char* w8 = nullptr;
            if ((rs = dalloc_t(E, &w8, (size_t)std::max<int64_t>(nnz, 1))) != LPA_OK) return rs;
            LPA_CUDA(launch_weights_to_u8(w_d, w8, nnz, st, E.sms));
            LPA_CUDA(cudaStreamSynchronize(st));
            auto it = std::find(E.owned.begin(), E.owned.end(), static_cast<void*>(w_d));
            if (it != E.owned.end()) {
                E.owned.erase(it);
                std::vector<void*> old{static_cast<void*>(w_d)};
                pool_free_all(E.device, old);
                E.device_bytes -= nnz * (int64_t)sizeof(float);
            }
            w_d = reinterpret_cast<float*>(w8);
            E.s.weight_kind = W_U8;
        } else {
            LPA_CUDA(launch_weights_to_u32(w_d, nnz, st, E.sms));
            E.s.weight_kind = W_U32;
        }
    } else {
        E.exact = vr.c[3] == 0 && vr.c[4] == 0;
        E.s.weight_kind = W_F32;
    }
    E.s.w = w_d;
    if (order != kOrderCaller && n > 0 && (rs = apply_order(E, order, st)) != LPA_OK) return rs;
    if ((rs = setup_blocks(E, st)) != LPA_OK) return rs;
    LPA_CUDA(cudaStreamSynchronize(st));
    return LPA_OK;
}

// An engine over the first K graphs of `par` (K >= 1), reading the parent's
// CSR (already validated, weights already narrowed) in place and holding its
// own working state: the timed sample of the autotuner.
lpa_status engine_view(Engine& E, const Engine& par, int32_t K, const lpa_config& cfg, cudaStream_t st) {
    E.device = par.device;
    E.sms = par.sms;
    E.s = par.s;
    E.s.G = K;
    E.s.N = par.vtx_off_host[K];
    E.s.E = 0;
    E.s.rows_distinct = par.s.G == 1 ? par.s.rows_distinct : 0;
    if (K == 1) E.s.gid = nullptr;
    E.weighted = par.weighted;
    E.borrowed = true;
    E.exact = par.exact;
    E.max_degree = par.max_degree;
    E.vtx_off_host.assign(par.vtx_off_host.begin(), par.vtx_off_host.begin() + K + 1);
    E.edge_off_host.assign(par.edge_off_host.begin(), par.edge_off_host.begin() + K + 1);
    E.cfg = cfg;
    E.owned.clear();
    E.device_bytes = 0;
    LPA_CUDA(cudaStreamCreateWithFlags(&E.cap_top, cudaStreamNonBlocking));
    LPA_CUDA(cudaStreamCreateWithFlags(&E.cap_body, cudaStreamNonBlocking));
    E.s.E = par.edge_off_host[K];
    lpa_status rs = alloc_state(E, st);
    if (rs != LPA_OK) return rs;
    LPA_CUDA(build_static_lists(E.s, st, E.static_counts, E.static_ents));
    if ((rs = setup_blocks(E, st)) != LPA_OK) return rs;
    LPA_CUDA(cudaStreamSynchronize(st));
    return LPA_OK;
}

cudaError_t launch_bin(Engine& E, int mode, int bin, cudaStream_t st) {
    if (bin == 0) return launch_sweep_small(E.s, mode, st, E.sms);
    if (bin == 1) return launch_sweep_warp(E.s, mode, st, E.sms);
    return launch_sweep_block(E.s, mode, bin, E.sms, st);
}

// A sweep's frontier is a subset of the static bin lists (same thresholds,
// vertices with no entries never join), so a bin that is statically empty is
// not launched at all.
// Launch order of the bins in a pass.  Asynchronous passes run the last bin
// first: in the first sweep every neighbour of its rows is then still
// unprocessed, so those rows read initial labels (their vertex ids) -- a
// valid interleaving of the parallel loop -- and take the max-over-row path
// on graphs whose rows repeat no neighbour.
int bin_at(int mode, int k) {
    if ((mode & ~kModeNonstrict) == MODE_ASYNC) return k == 0 ? kBins - 1 : k - 1;
    return k;
}

cudaError_t enqueue_pass(Engine& E, int mode, cudaStream_t st) {
    for (int k = 0; k < kBins; ++k) {
        const int b = bin_at(mode, k);
        if (E.s.bin_static[b] == 0) continue;
        cudaError_t err = launch_bin(E, mode, b, st);
        if (err != cudaSuccess) return err;
    }
    return cudaSuccess;
}

// One sweep (lpaMove of Algorithm 1).  Sync modes: one pass over the frontier,
// then the finish kernel (apply, compaction, control).  Async mode: a main
// pass over the frontier, a compaction of the vertices it marked that were
// not in the frontier, and a catch-up pass over them within the same sweep --
// the parallel counterpart of the serial loop, which reaches a vertex marked
// by an earlier vertex later in the same sweep, while a vertex it has already
// scanned keeps its mark for the next sweep -- then the finish kernel.
// `mode` may carry kModeNonstrict, which only the sweep kernels take.
cudaError_t enqueue_sweep(Engine& E, int mode, cudaGraphConditionalHandle h, int in_graph, cudaStream_t st) {
    const int base = mode & ~kModeNonstrict;
    cudaError_t err = enqueue_pass(E, mode, st);
    if (err != cudaSuccess) return err;
    if (base == MODE_ASYNC) {
        err = launch_finish(E.s, base, kRoleCatchUp, h, in_graph, st, E.sms);
        if (err != cudaSuccess) return err;
        err = enqueue_pass(E, mode, st);
        if (err != cudaSuccess) return err;
    }
    return launch_finish(E.s, base, kRoleEndSweep, h, in_graph, st, E.sms);
}

int graph_index(int mode) { return (mode & ~kModeNonstrict) + ((mode & kModeNonstrict) ? 3 : 0); }

// Graph for one mode:  init -> init_cond -> WHILE { sweep } -> finalize
lpa_status build_graph(Engine& E, int mode) {
    const int gi = graph_index(mode);
    if (E.exec[gi]) return LPA_OK;
    cudaGraph_t top = nullptr;
    LPA_CUDA(cudaGraphCreate(&top, 0));
    cudaGraphConditionalHandle h;
    cudaError_t err = cudaGraphConditionalHandleCreate(&h, top, 0, cudaGraphCondAssignDefault);
    if (err != cudaSuccess) {
        cudaGraphDestroy(top);
        return cuda_fail(err, "cudaGraphConditionalHandleCreate");
    }
    auto bail = [&](cudaError_t e, const char* where) {
        cudaStreamCaptureStatus cs;
        if (cudaStreamIsCapturing(E.cap_top, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone) {
            cudaGraph_t junk;
            cudaStreamEndCapture(E.cap_top, &junk);
        }
        if (cudaStreamIsCapturing(E.cap_body, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone) {
            cudaGraph_t junk;
            cudaStreamEndCapture(E.cap_body, &junk);
        }
        cudaGraphDestroy(top);
        cudaGetLastError();
        return cuda_fail(e, where);
    };
    err = cudaStreamBeginCaptureToGraph(E.cap_top, top, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
    if (err != cudaSuccess) return bail(err, "begin capture (top)");
    if ((err = launch_init(E.s, E.cap_top, E.sms)) != cudaSuccess) return bail(err, "init");
    if ((err = launch_init_cond(E.s, h, 1, E.cap_top)) != cudaSuccess) return bail(err, "init_cond");
    cudaStreamCaptureStatus cst;
    const cudaGraphNode_t* deps = nullptr;
    size_t ndeps = 0;
    cudaGraph_t capg = nullptr;
    err = cudaStreamGetCaptureInfo(E.cap_top, &cst, nullptr, &capg, &deps, nullptr, &ndeps);
    if (err != cudaSuccess) return bail(err, "capture info");
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t cond;
    err = cudaGraphAddNode(&cond, capg, deps, nullptr, ndeps, &cp);
    if (err != cudaSuccess) return bail(err, "add WHILE node");
    err = cudaStreamUpdateCaptureDependencies(E.cap_top, &cond, nullptr, 1, cudaStreamSetCaptureDependencies);
    if (err != cudaSuccess) return bail(err, "update capture deps");
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    err = cudaStreamBeginCaptureToGraph(E.cap_body, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
    if (err != cudaSuccess) return bail(err, "begin capture (body)");
    if ((err = enqueue_sweep(E, mode, h, 1, E.cap_body)) != cudaSuccess) return bail(err, "sweep");
    cudaGraph_t body_out = nullptr;
    err = cudaStreamEndCapture(E.cap_body, &body_out);
    if (err != cudaSuccess) return bail(err, "end capture (body)");
    if ((err = launch_finalize(E.s, E.cap_top, E.sms)) != cudaSuccess) return bail(err, "finalize");
    cudaGraph_t top_out = nullptr;
    err = cudaStreamEndCapture(E.cap_top, &top_out);
    if (err != cudaSuccess) return bail(err, "end capture (top)");
    cudaGraphExec_t ex = nullptr;
    err = cudaGraphInstantiate(&ex, top, 0);
    if (err != cudaSuccess) return bail(err, "instantiate");
    E.graph[gi] = top;
    E.exec[gi] = ex;
    return LPA_OK;
}

// The mode argument of the run calls: an lpa_mode, optionally | LPA_NONSTRICT.
// Pruning is exact in the synchronous mode only for the strict tie-break (a
// pick depends on the neighbours' labels alone); a non-strict pick also
// depends on the sweep, so the synchronous mode then scans every vertex in
// every sweep.
// LPA_PRUNE_OTHER (FLPA's pruning rule) is taken in the asynchronous mode only.
void split_mode(int& mode, int& nonstrict, int& prune_other) {
    nonstrict = (mode & (int)LPA_NONSTRICT) ? 1 : 0;
    prune_other = (mode & (int)LPA_PRUNE_OTHER) ? 1 : 0;
    mode &= ~((int)LPA_NONSTRICT | (int)LPA_PRUNE_OTHER);
    if (nonstrict && mode == MODE_SYNC) mode = MODE_SYNC_FULL;
}

lpa_status check_run_args(const Engine& E, int mode, int prune_other, double tol, int32_t max_iters,
                          const int32_t* labels_out) {
    if (mode < 0 || mode > 2) return fail(LPA_ERR_INVALID_ARG, "unknown mode %d", mode);
    if (prune_other && mode != MODE_ASYNC)
        return fail(LPA_ERR_INVALID_ARG, "LPA_PRUNE_OTHER needs LPA_MODE_ASYNC");
    if (!(tol >= 0.0 && tol <= 1.0)) return fail(LPA_ERR_INVALID_ARG, "tolerance must be in [0, 1]");
    if (max_iters < 0 || max_iters > (1 << 20)) return fail(LPA_ERR_INVALID_ARG, "max_iters must be in [0, 2^20]");
    if (E.s.N > 0 && !labels_out) return fail(LPA_ERR_INVALID_ARG, "labels_out is NULL");
    return LPA_OK;
}

// Device results of the last run -> lpa_run_info per graph (host).
lpa_status collect_info(Engine& E, cudaStream_t st, lpa_run_info* infos, int32_t count) {
    std::vector<int32_t> iters(E.s.G), exits(E.s.G);
    std::vector<long long> hist((size_t)E.s.G * kMaxHist);
    Ctrl c;
    LPA_CUDA(cudaMemcpyAsync(iters.data(), E.s.iters, (size_t)E.s.G * 4, cudaMemcpyDeviceToHost, st));
    LPA_CUDA(cudaMemcpyAsync(exits.data(), E.s.exit_reason, (size_t)E.s.G * 4, cudaMemcpyDeviceToHost, st));
    LPA_CUDA(cudaMemcpyAsync(hist.data(), E.s.hist_changed, hist.size() * 8, cudaMemcpyDeviceToHost, st));
    LPA_CUDA(cudaMemcpyAsync(&c, E.s.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, st));
    LPA_CUDA(cudaStreamSynchronize(st));
    if (c.error == 5) return fail(LPA_ERR_TIMEOUT, "a bounded wait on a bulk copy gave up (code 5)");
    if (c.error) return fail(LPA_ERR_CUDA, "device-side check failed (code %d)", c.error);
    for (int32_t g = 0; g < count; ++g) {
        lpa_run_info& I = infos[g];
        memset(&I, 0, sizeof(I));
        I.iterations = iters[g];
        I.exit_reason = exits[g];
        const int rec = std::min(iters[g], kMaxHist);
        for (int t = 0; t < rec; ++t) I.changed[t] = hist[(size_t)g * kMaxHist + t];
        if (E.s.G == 1) {
            for (int t = 0; t < rec; ++t) {
                I.active[t] = c.hist_active[t];
                I.scanned[t] = c.hist_scanned[t];
                I.edges_touched += c.hist_scanned[t];
            }
        }
    }
    return LPA_OK;
}

lpa_status engine_run(Engine& E, int mode, double tol, int32_t max_iters, int32_t* labels_out, cudaStream_t st,
                      lpa_run_info* infos, int local_ids) {
    int ns = 0, po = 0;
    split_mode(mode, ns, po);
    lpa_status rs = check_run_args(E, mode, po, tol, max_iters, labels_out);
    if (rs != LPA_OK) return rs;
    if (E.s.N == 0) {
        for (int32_t g = 0; infos && g < E.s.G; ++g) {
            memset(&infos[g], 0, sizeof(lpa_run_info));
            infos[g].exit_reason = 2;
        }
        return LPA_OK;
    }
    const int lm = mode | (ns ? kModeNonstrict : 0);
    if ((rs = build_graph(E, lm)) != LPA_OK) return rs;
    LPA_CUDA(launch_set_params(E.s.ctrl, tol, max_iters, mode, ns, po, labels_out, local_ids, st));
    LPA_CUDA(cudaGraphLaunch(E.exec[graph_index(lm)], st));
    ++E.runs_total;
    if (infos) return collect_info(E, st, infos, E.s.G);
    return LPA_OK;
}

// Host-driven run with an event pair around every launch.
lpa_status engine_run_profiled(Engine& E, int mode, double tol, int32_t max_iters, int32_t* labels_out,
                               cudaStream_t st, lpa_run_info* infos, lpa_profile* prof, int local_ids) {
    const int mode_arg = mode;
    int ns = 0, po = 0;
    split_mode(mode, ns, po);
    lpa_status rs = check_run_args(E, mode, po, tol, max_iters, labels_out);
    if (rs != LPA_OK) return rs;
    if (!prof) return fail(LPA_ERR_INVALID_ARG, "prof is NULL");
    memset(prof, 0, sizeof(*prof));
    if (E.s.N == 0) return engine_run(E, mode_arg, tol, max_iters, labels_out, st, infos, local_ids);
    cudaEvent_t ev[kBins + 2];
    for (auto& e : ev) LPA_CUDA(cudaEventCreate(&e));
    auto cleanup = [&]() {
        for (auto& e : ev) cudaEventDestroy(e);
    };
    cudaGraphConditionalHandle none = 0;
    cudaError_t err;
    float ms = 0.f;
#define LPA_P(call)                          \
    do {                                     \
        err = (call);                        \
        if (err != cudaSuccess) {            \
            cleanup();                       \
            return cuda_fail(err, #call);    \
        }                                    \
    } while (0)
    LPA_P(launch_set_params(E.s.ctrl, tol, max_iters, mode, ns, po, labels_out, local_ids, st));
    LPA_P(cudaEventRecord(ev[0], st));
    LPA_P(launch_init(E.s, st, E.sms));
    LPA_P(launch_init_cond(E.s, none, 0, st));
    LPA_P(cudaEventRecord(ev[1], st));
    LPA_P(cudaEventSynchronize(ev[1]));
    LPA_P(cudaEventElapsedTime(&ms, ev[0], ev[1]));
    prof->init_ms = ms;
    Ctrl c;
    LPA_P(cudaMemcpy(&c, E.s.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost));
    int t = 0;
    while (c.any_active) {
        float sweep_ms[kBins] = {0.f}, fin_ms = 0.f;
        const int passes = mode == MODE_ASYNC ? 2 : 1;
        for (int p = 0; p < passes; ++p) {
            for (int k = 0; k < kBins; ++k) {
                const int b = bin_at(mode, k);
                LPA_P(cudaEventRecord(ev[k], st));
                if (E.s.bin_static[b]) LPA_P(launch_bin(E, mode | (ns ? kModeNonstrict : 0), b, st));
            }
            LPA_P(cudaEventRecord(ev[kBins], st));
            LPA_P(launch_finish(E.s, mode, p + 1 < passes ? kRoleCatchUp : kRoleEndSweep, none, 0, st, E.sms));
            LPA_P(cudaEventRecord(ev[kBins + 1], st));
            LPA_P(cudaEventSynchronize(ev[kBins + 1]));
            for (int k = 0; k < kBins; ++k) {
                LPA_P(cudaEventElapsedTime(&ms, ev[k], ev[k + 1]));
                sweep_ms[bin_at(mode, k)] += ms;
            }
            LPA_P(cudaEventElapsedTime(&ms, ev[kBins], ev[kBins + 1]));
            fin_ms += ms;
        }
        LPA_P(cudaMemcpy(&c, E.s.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost));
        if (t < kMaxHist) {
            for (int b = 0; b < kBins; ++b) {
                prof->sweep_ms[t][b] = sweep_ms[b];
                prof->bin_vertices[t][b] = c.hist_bin_vertices[t][b];
                prof->bin_entries[t][b] = c.hist_bin_entries[t][b];
                prof->bin_changed[t][b] = c.hist_bin_changed[t][b];
                prof->bin_changed_entries[t][b] = c.hist_bin_changed_entries[t][b];
            }
            prof->finish_ms[t] = fin_ms;
        }
        ++t;
        if (c.error) break;
    }
    prof->iterations = t;
    LPA_P(launch_finalize(E.s, st, E.sms));
    LPA_P(cudaStreamSynchronize(st));
#undef LPA_P
    cleanup();
    if (infos) return collect_info(E, st, infos, E.s.G);
    if (c.error == 5) return fail(LPA_ERR_TIMEOUT, "a bounded wait on a bulk copy gave up (code 5)");
    if (c.error) return fail(LPA_ERR_CUDA, "device-side check failed (code %d)", c.error);
    return LPA_OK;
}

lpa_status engine_modularity(Engine& E, int64_t v0, int64_t v1, const int32_t* labels, double* q_out,
                             cudaStream_t st) {
    if (!q_out) return fail(LPA_ERR_INVALID_ARG, "q_out is NULL");
    if (v1 > v0 && !labels) return fail(LPA_ERR_INVALID_ARG, "labels is NULL");
    lpa_status rs;
    if (!E.Sigma) {
        if ((rs = dalloc_t(E, &E.Sigma, (size_t)std::max<int64_t>(E.s.N, 1))) != LPA_OK) return rs;
        if ((rs = dalloc_t(E, &E.acc, 1)) != LPA_OK) return rs;
    }
    const int64_t n = v1 - v0;
    if (n == 0) {
        *q_out = 0.0;
        return LPA_OK;
    }
    LPA_CUDA(cudaMemsetAsync(E.Sigma, 0, (size_t)n * 8, st));
    LPA_CUDA(cudaMemsetAsync(E.acc, 0, sizeof(ModAccum), st));
    LPA_CUDA(launch_modularity(E.s, v0, v1, labels, E.Sigma, E.acc, st, E.sms));
    ModAccum a;
    LPA_CUDA(cudaMemcpyAsync(&a, E.acc, sizeof(a), cudaMemcpyDeviceToHost, st));
    LPA_CUDA(cudaStreamSynchronize(st));
    if (a.bad_label) return fail(LPA_ERR_INVALID_ARG, "%u labels outside [0, n)", a.bad_label);
    *q_out = a.two_m > 0.0 ? a.sigma / a.two_m - a.null_sum / (a.two_m * a.two_m) : 0.0;
    return LPA_OK;
}

lpa_status fill_props(const Engine& E, lpa_graph_props* p) {
    Ctrl c;
    LPA_CUDA(cudaDeviceSynchronize());
    LPA_CUDA(cudaMemcpy(&c, E.s.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost));
    memset(p, 0, sizeof(*p));
    p->sweeps_total = c.total_sweeps;
    p->scanned_total = c.total_scanned;
    p->launches_total = E.runs_total * 4 + c.total_sweep_launches;
    p->n = E.s.N;
    p->nnz = E.s.E;
    p->num_graphs = E.s.G;
    p->weighted = E.weighted ? 1 : 0;
    p->weight_bytes = E.s.weight_kind == W_UNIT ? 0 : E.s.weight_kind == W_U8 ? 1 : 4;
    p->exact = E.exact ? 1 : 0;
    p->max_degree = E.max_degree;
    p->rows_distinct = E.s.rows_distinct;
    p->storage_order = E.order;
    p->device_bytes = E.device_bytes + (int64_t)std::max<size_t>(E.s.bin_static[kBins - 1], 1) * sizeof(Overflow);
    return LPA_OK;
}

// ------------------------------------------------------------- autotuner --
// Launch parameters per degree bin (lpa_config) picked for a workload: the
// GPU counterpart of the paper's scheduling choice (Section 4.1.1, OpenMP
// dynamic chunks of 2048 vertices).  Candidate limits are powers of two, so a
// log2 degree histogram gives every candidate's bin of every vertex exactly;
// candidates that bin the workload's vertices the same way as one already
// timed are skipped.  The search is one pass of coordinate descent from the
// configuration in force (always a candidate), each candidate timed on a
// sample of the workload (a prefix of a batch's graphs sharing its CSR).
// Choices are cached per process, keyed by mode, weight storage and the
// histogram rounded to 1/64 of the vertices and of the entries per bucket.
std::mutex g_tune_mu;
std::map<std::string, lpa_config> g_tune_cache;

lpa_status set_config(Engine& E, const lpa_config* cfg) {
    if (!cfg) return fail(LPA_ERR_INVALID_ARG, "cfg is NULL");
    lpa_status rs = check_config(*cfg);
    if (rs != LPA_OK) return rs;
    LPA_CUDA(cudaDeviceSynchronize());
    destroy_graphs(E);
    E.cfg = *cfg;
    apply_config_fields(E);
    LPA_CUDA(build_static_lists(E.s, 0, E.static_counts, E.static_ents));
    return setup_blocks(E, 0);
}

lpa_status degree_histogram(Engine& E, std::vector<unsigned long long>& h, cudaStream_t st) {
    lpa_status rs;
    if (!E.hist_d && (rs = dalloc_t(E, &E.hist_d, 2 * kDegBuckets)) != LPA_OK) return rs;
    LPA_CUDA(launch_degree_hist(E.s, E.hist_d, st, E.sms));
    h.assign(2 * kDegBuckets, 0ull);
    LPA_CUDA(cudaMemcpyAsync(h.data(), E.hist_d, h.size() * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
    LPA_CUDA(cudaStreamSynchronize(st));
    return LPA_OK;
}

bool pow2(int x) { return x > 0 && (x & (x - 1)) == 0; }

// Bin (0..4) of a bucket of degrees (2^(b-1), 2^b] under power-of-two limits.
int bucket_bin(const lpa_config& c, int b) {
    const int64_t hi = (int64_t)1 << b;      // the bucket's largest degree
    return hi <= c.small_max ? 0 : hi <= c.warp_max ? 1 : hi <= c.mid_max ? 2 : hi <= c.large_max ? 3 : 4;
}

// What a configuration does to the workload: the bin of each non-empty
// bucket, and the dense threshold.  Equal signatures launch the same kernels
// on the same vertices.
std::string tune_signature(const lpa_config& c, const std::vector<unsigned long long>& h) {
    std::string sig;
    for (int b = 0; b < kDegBuckets; ++b)
        if (h[b]) sig += (char)('0' + bucket_bin(c, b));
    sig += ":" + std::to_string(c.dense_permille);
    return sig;
}

std::string tune_key(const Engine& E, int mode, const std::vector<unsigned long long>& h) {
    unsigned long long nv = 0, ne = 0;
    for (int b = 0; b < kDegBuckets; ++b) {
        nv += h[b];
        ne += h[kDegBuckets + b];
    }
    std::string key = "m" + std::to_string(mode) + "w" + std::to_string(E.s.weight_kind) + (E.s.G > 1 ? "b" : "s");
    for (int b = 0; b < kDegBuckets; ++b) {
        const long qv = nv ? std::lround(64.0 * (double)h[b] / (double)nv) : 0;
        const long qe = ne ? std::lround(64.0 * (double)h[kDegBuckets + b] / (double)ne) : 0;
        if (qv || qe) key += "," + std::to_string(b) + ":" + std::to_string(qv) + "/" + std::to_string(qe);
    }
    return key;
}

// Best of `trials` timed runs (after one untimed run) of engine T under cfg.
lpa_status time_config(Engine& T, const lpa_config& cfg, int mode, double tol, int32_t max_iters, int32_t trials,
                       cudaStream_t st, cudaEvent_t e0, cudaEvent_t e1, float* best_ms) {
    lpa_status rs = set_config(T, &cfg);
    if (rs != LPA_OK) return rs;
    float best = 1e30f;
    for (int r = 0; r <= trials; ++r) {
        LPA_CUDA(cudaEventRecord(e0, st));
        if ((rs = engine_run(T, mode, tol, max_iters, T.tune_out, st, nullptr, T.s.G > 1 ? 1 : 0)) != LPA_OK)
            return rs;
        LPA_CUDA(cudaEventRecord(e1, st));
        LPA_CUDA(cudaEventSynchronize(e1));
        float ms = 0.f;
        LPA_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        if (r > 0) best = std::min(best, ms);
    }
    *best_ms = best;
    return LPA_OK;
}

lpa_status autotune_engine(Engine& E, int mode, double tol, int32_t max_iters, int32_t trials,
                           int32_t sample_permille, cudaStream_t st, lpa_config* chosen, lpa_autotune_info* info) {
    if (trials < 1 || trials > 100) return fail(LPA_ERR_INVALID_ARG, "trials must be in [1, 100]");
    if (sample_permille < 1 || sample_permille > 1000)
        return fail(LPA_ERR_INVALID_ARG, "sample_permille must be in [1, 1000]");
    int ns = 0, po = 0, base = mode;
    split_mode(base, ns, po);
    if (base < 0 || base > 2) return fail(LPA_ERR_INVALID_ARG, "unknown mode %d", base);
    if (po && base != MODE_ASYNC) return fail(LPA_ERR_INVALID_ARG, "LPA_PRUNE_OTHER needs LPA_MODE_ASYNC");
    if (!(tol >= 0.0 && tol <= 1.0)) return fail(LPA_ERR_INVALID_ARG, "tolerance must be in [0, 1]");
    if (max_iters < 0 || max_iters > (1 << 20)) return fail(LPA_ERR_INVALID_ARG, "max_iters must be in [0, 2^20]");
    lpa_status rs = LPA_OK;
    lpa_autotune_info inf{};
    const auto t_start = std::chrono::steady_clock::now();
    const lpa_config start = E.cfg;
    if (E.s.N == 0) {
        if (chosen) *chosen = start;
        if (info) *info = inf;
        return LPA_OK;
    }
    std::vector<unsigned long long> h;
    if ((rs = degree_histogram(E, h, st)) != LPA_OK) return rs;
    const std::string key = tune_key(E, mode, h);
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            const lpa_config c = it->second;
            if ((rs = set_config(E, &c)) != LPA_OK) return rs;
            inf.cached = 1;
            inf.search_ms = (float)std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() -
                                                                              t_start).count();
            if (chosen) *chosen = c;
            if (info) *info = inf;
            return LPA_OK;
        }
    }
    // the timed sample: the shortest prefix of graphs holding sample_permille
    // of the entries (the whole workload for a single graph)
    int32_t K = E.s.G;
    if (E.s.G > 1) {
        const double want = (double)E.edge_off_host[E.s.G] * sample_permille / 1000.0;
        K = 1;
        while (K < E.s.G && (double)E.edge_off_host[K] < want) ++K;
    }
    Engine view;
    Engine* T = &E;
    if (K < E.s.G) {
        if ((rs = engine_view(view, E, K, start, st)) != LPA_OK) {
            engine_free(view);
            return rs;
        }
        T = &view;
    }
    if (!T->tune_out && (rs = dalloc_t(*T, &T->tune_out, (size_t)std::max<int64_t>(T->s.N, 1))) != LPA_OK) {
        if (T != &E) engine_free(view);
        return rs;
    }
    inf.sample_graphs = K;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const bool exact_bins = pow2(start.small_max) && pow2(start.warp_max) && pow2(start.mid_max) &&
                            pow2(start.large_max);
    std::vector<std::string> seen;
    lpa_config best = start;
    float best_ms = 0.f;
    rs = time_config(*T, start, mode, tol, max_iters, trials, st, e0, e1, &best_ms);
    inf.default_ms = best_ms;
    inf.candidates = 1;
    if (exact_bins) seen.push_back(tune_signature(start, h));
    static const int kSmall[] = {1, 2, 4, 8};
    static const int kWarp[] = {16, 32, 64, 128, 256};
    static const int kMid[] = {256, 512, 1024, 2048};
    static const int kLarge[] = {1024, 2048, 4096};
    static const int kDense[] = {300, 500, 700, 1001};
    struct Axis {
        int lpa_config::*field;
        const int* vals;
        int n;
    };
    const Axis axes[] = {{&lpa_config::warp_max, kWarp, 5}, {&lpa_config::mid_max, kMid, 4},
                         {&lpa_config::small_max, kSmall, 4}, {&lpa_config::large_max, kLarge, 3},
                         {&lpa_config::dense_permille, kDense, 4}};
    for (const Axis& ax : axes) {
        if (rs != LPA_OK) break;
        const lpa_config centre = best;
        for (int q = 0; q < ax.n && rs == LPA_OK; ++q) {
            lpa_config c = centre;
            c.*(ax.field) = ax.vals[q];
            if (c.*(ax.field) == centre.*(ax.field)) continue;
            if (c.small_max >= c.warp_max || c.warp_max >= c.mid_max || c.mid_max >= c.large_max) continue;
            if (check_config(c) != LPA_OK) continue;
            if (exact_bins) {
                const std::string sig = tune_signature(c, h);
                if (std::find(seen.begin(), seen.end(), sig) != seen.end()) continue;
                seen.push_back(sig);
            }
            float ms = 0.f;
            rs = time_config(*T, c, mode, tol, max_iters, trials, st, e0, e1, &ms);
            ++inf.candidates;
            if (rs == LPA_OK && ms < best_ms) {
                best_ms = ms;
                best = c;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (T != &E) engine_free(view);
    if (rs != LPA_OK) {
        set_config(E, &start);
        return rs;
    }
    if ((rs = set_config(E, &best)) != LPA_OK) return rs;
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        g_tune_cache[key] = best;
    }
    inf.chosen_ms = best_ms;
    inf.search_ms =
        (float)std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
    if (chosen) *chosen = best;
    if (info) *info = inf;
    return LPA_OK;
}

}  // namespace

namespace lpa {
// Error text for entry points defined in other translation units.
void set_last_error(lpa_status st, const char* msg) {
    (void)st;
    g_last_error = msg;
}
}  // namespace lpa

struct lpa_graph {
    Engine e;
};
struct lpa_batch {
    Engine e;
};

extern "C" {

const char* lpa_version(void) { return "lpa-gb300 0.1"; }

const char* lpa_status_string(lpa_status st) {
    switch (st) {
        case LPA_OK: return "ok";
        case LPA_ERR_INVALID_ARG: return "invalid argument";
        case LPA_ERR_INVALID_GRAPH: return "invalid graph";
        case LPA_ERR_OUT_OF_MEMORY: return "out of memory";
        case LPA_ERR_CUDA: return "CUDA error";
        case LPA_ERR_TIMEOUT: return "timeout";
        case LPA_ERR_BUSY: return "busy";
        case LPA_ERR_NOT_FOUND: return "not found";
        case LPA_ERR_NOT_READY: return "not ready";
    }
    return "unknown status";
}

const char* lpa_last_error(void) { return g_last_error.c_str(); }

lpa_status lpa_tolerance_threshold(double tolerance, int64_t n, int64_t* out) {
    if (!out) return fail(LPA_ERR_INVALID_ARG, "out is NULL");
    if (!(tolerance >= 0.0 && tolerance <= 1.0)) return fail(LPA_ERR_INVALID_ARG, "tolerance must be in [0, 1]");
    if (n < 0 || n > 0x7fffffffLL) return fail(LPA_ERR_INVALID_ARG, "n out of range [0, 2^31-1]");
    *out = (int64_t)dn_threshold(tolerance, n);
    return LPA_OK;
}

lpa_status lpa_graph_create(int64_t n, int64_t nnz, const int64_t* offsets, const int32_t* indices,
                            const float* weights, uint32_t flags, void* stream, lpa_graph_t* out) {
    g_last_error.clear();
    if (!out) return fail(LPA_ERR_INVALID_ARG, "out is NULL");
    lpa_graph* g = new (std::nothrow) lpa_graph();
    if (!g) return fail(LPA_ERR_OUT_OF_MEMORY, "host allocation");
    const int64_t vo[2] = {0, n};
    const int64_t eo[2] = {0, nnz};
    lpa_status rs = engine_create(g->e, 1, vo, eo, n, nnz, offsets, indices, weights, flags,
                                  static_cast<cudaStream_t>(stream));
    if (rs != LPA_OK) {
        engine_free(g->e);
        delete g;
        return rs;
    }
    *out = g;
    return LPA_OK;
}

lpa_status lpa_graph_destroy(lpa_graph_t g) {
    if (!g) return fail(LPA_ERR_INVALID_ARG, "graph is NULL");
    engine_free(g->e);
    delete g;
    return LPA_OK;
}

lpa_status lpa_graph_props_get(lpa_graph_t g, lpa_graph_props* out) {
    if (!g || !out) return fail(LPA_ERR_INVALID_ARG, "NULL argument");
    return fill_props(g->e, out);
}

lpa_status lpa_graph_get_config(lpa_graph_t g, lpa_config* out) {
    if (!g || !out) return fail(LPA_ERR_INVALID_ARG, "NULL argument");
    *out = g->e.cfg;
    return LPA_OK;
}

lpa_status lpa_graph_set_config(lpa_graph_t g, const lpa_config* cfg) {
    if (!g) return fail(LPA_ERR_INVALID_ARG, "graph is NULL");
    return set_config(g->e, cfg);
}

lpa_status lpa_graph_debug_stall(lpa_graph_t g, int32_t block_threads) {
    if (!g) return fail(LPA_ERR_INVALID_ARG, "graph is NULL");
    if (block_threads != 0 && block_threads != 128 && block_threads != 256 && block_threads != 512)
        return fail(LPA_ERR_INVALID_ARG, "block_threads must be 0, 128, 256 or 512");
    Engine& E = g->e;
    LPA_CUDA(cudaSetDevice(E.device));
    LPA_CUDA(cudaMemcpy(&E.s.ctrl->stall_copy, &block_threads, sizeof(int32_t), cudaMemcpyHostToDevice));
    return LPA_OK;
}

lpa_status lpa_run(lpa_graph_t g, lpa_mode mode, double tolerance, int32_t max_iters, int32_t* labels_out,
                   void* stream, lpa_run_info* info) {
    if (!g) return fail(LPA_ERR_INVALID_ARG, "graph is NULL");
    return engine_run(g->e, (int)mode, tolerance, max_iters, labels_out, static_cast<cudaStream_t>(stream), info, 0);
}

lpa_status lpa_run_profiled(lpa_graph_t g, lpa_mode mode, double tolerance, int32_t max_iters, int32_t* labels_out,
                            void* stream, lpa_run_info* info, lpa_profile* prof) {
    if (!g) return fail(LPA_ERR_INVALID_ARG, "graph is NULL");
    return engine_run_profiled(g->e, (int)mode, tolerance, max_iters, labels_out, static_cast<cudaStream_t>(stream),
                               info, prof, 0);
}

lpa_status lpa_modularity(lpa_graph_t g, const int32_t* labels, double* q_out, void* stream) {
    if (!g) return fail(LPA_ERR_INVALID_ARG, "graph is NULL");
    return engine_modularity(g->e, 0, g->e.s.N, labels, q_out, static_cast<cudaStream_t>(stream));
}

lpa_status lpa_autotune(lpa_graph_t g, lpa_mode mode, double tolerance, int32_t max_iters, int32_t trials,
                        void* stream, lpa_config* chosen, lpa_autotune_info* info) {
    if (!g) return fail(LPA_ERR_INVALID_ARG, "graph is NULL");
    return autotune_engine(g->e, (int)mode, tolerance, max_iters, trials, 1000, static_cast<cudaStream_t>(stream),
                           chosen, info);
}

lpa_status lpa_batch_autotune(lpa_batch_t b, lpa_mode mode, double tolerance, int32_t max_iters, int32_t trials,
                              int32_t sample_permille, void* stream, lpa_config* chosen, lpa_autotune_info* info) {
    if (!b) return fail(LPA_ERR_INVALID_ARG, "batch is NULL");
    return autotune_engine(b->e, (int)mode, tolerance, max_iters, trials, sample_permille,
                           static_cast<cudaStream_t>(stream), chosen, info);
}

lpa_status lpa_autotune_cache_clear(void) {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune_cache.clear();
    return LPA_OK;
}

lpa_status lpa_batch_get_config(lpa_batch_t b, lpa_config* out) {
    if (!b || !out) return fail(LPA_ERR_INVALID_ARG, "NULL argument");
    *out = b->e.cfg;
    return LPA_OK;
}

lpa_status lpa_batch_set_config(lpa_batch_t b, const lpa_config* cfg) {
    if (!b) return fail(LPA_ERR_INVALID_ARG, "batch is NULL");
    return set_config(b->e, cfg);
}

// ------------------------------------------------------------------ batches
lpa_status lpa_release_cached_memory(void) {
    g_last_error.clear();
    std::lock_guard<std::mutex> lock(g_pool_mu);
    for (int d = 0; d < kMaxPoolDevices; ++d) {
        if (!g_pools[d].pool) continue;
        cudaError_t e = cudaMemPoolTrimTo(g_pools[d].pool, 0);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemPoolTrimTo");
    }
    return LPA_OK;
}

lpa_status lpa_batch_create(int32_t G, const int64_t* graph_vtx_off, const int64_t* graph_edge_off,
                            const int64_t* offsets, const int32_t* indices, const float* weights, uint32_t flags,
                            void* stream, lpa_batch_t* out) {
    g_last_error.clear();
    if (!out) return fail(LPA_ERR_INVALID_ARG, "out is NULL");
    if (G < 1) return fail(LPA_ERR_INVALID_ARG, "G must be >= 1");
    if (!graph_vtx_off || !graph_edge_off) return fail(LPA_ERR_INVALID_ARG, "graph offsets are NULL");
    if (graph_vtx_off[0] != 0 || graph_edge_off[0] != 0)
        return fail(LPA_ERR_INVALID_ARG, "graph offsets must start at 0");
    for (int32_t g = 0; g < G; ++g)
        if (graph_vtx_off[g + 1] < graph_vtx_off[g] || graph_edge_off[g + 1] < graph_edge_off[g])
            return fail(LPA_ERR_INVALID_ARG, "graph offsets must be non-decreasing");
    if (flags & LPA_BORROW) return fail(LPA_ERR_INVALID_ARG, "LPA_BORROW is not accepted for batches");
    lpa_batch* b = new (std::nothrow) lpa_batch();
    if (!b) return fail(LPA_ERR_OUT_OF_MEMORY, "host allocation");
    lpa_status rs = engine_create(b->e, G, graph_vtx_off, graph_edge_off, graph_vtx_off[G], graph_edge_off[G],
                                  offsets, indices, weights, flags, static_cast<cudaStream_t>(stream));
    if (rs != LPA_OK) {
        engine_free(b->e);
        delete b;
        return rs;
    }
    *out = b;
    return LPA_OK;
}

lpa_status lpa_batch_destroy(lpa_batch_t b) {
    if (!b) return fail(LPA_ERR_INVALID_ARG, "batch is NULL");
    engine_free(b->e);
    delete b;
    return LPA_OK;
}

lpa_status lpa_batch_props_get(lpa_batch_t b, lpa_graph_props* out) {
    if (!b || !out) return fail(LPA_ERR_INVALID_ARG, "NULL argument");
    return fill_props(b->e, out);
}

lpa_status lpa_batch_run(lpa_batch_t b, lpa_mode mode, double tolerance, int32_t max_iters, int32_t* labels_out,
                         void* stream, lpa_run_info* infos) {
    if (!b) return fail(LPA_ERR_INVALID_ARG, "batch is NULL");
    return engine_run(b->e, (int)mode, tolerance, max_iters, labels_out, static_cast<cudaStream_t>(stream), infos,
                      1);
}

lpa_status lpa_batch_modularity(lpa_batch_t b, int32_t g, const int32_t* labels, double* q_out, void* stream) {
    if (!b) return fail(LPA_ERR_INVALID_ARG, "batch is NULL");
    if (g < 0 || g >= b->e.s.G) return fail(LPA_ERR_INVALID_ARG, "graph index out of range");
    return engine_modularity(b->e, b->e.vtx_off_host[g], b->e.vtx_off_host[g + 1], labels, q_out,
                             static_cast<cudaStream_t>(stream));
}

}  // extern "C"
