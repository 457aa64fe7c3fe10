// lpa_serve.cu -- continuous-batching server for label propagation requests
// (lpa_serve_* in include/lpa.h).
//
// Requests are independent graphs.  Small ones share a device-resident arena:
// a fixed-capacity CSR (separate row-begin and row-end offsets, so a request
// may occupy any free vertex range and entry range) with per-slot state
// (convergence test dN/N <= tau, sweep count and cap of Algorithm 1, done
// bit).  A worker thread runs the arena cycle by cycle: each cycle compacts
// the marks of every active request into one frontier, runs one sweep over
// it with the ordinary sweep kernels, and applies each slot's tolerance test.
// Requests that arrive while others run are admitted at the next cycle
// (their vertices marked unprocessed, their labels set to their ids), and a
// request leaves as soon as its own test is met, freeing its ranges and its
// slot.  Because labels never cross graphs and each slot keeps its own
// counters, a synchronous-mode result is the same alone and in the mix.
//
// Requests with at least `solo_min_entries` entries run on a separate lane
// (their own graph handle and stream, one at a time) so that they do not slow
// the arena's cycles.  Admission is by device memory: the arena is allocated
// up front from the budget; a solo request needs its estimated footprint to
// fit in what the budget leaves; otherwise submit returns LPA_ERR_BUSY.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/lpa.h"
#include "lpa_internal.h"

namespace lpa {
void set_last_error(lpa_status st, const char* msg);
}

using namespace lpa;

namespace {

lpa_status err(lpa_status st, const std::string& msg) {
    set_last_error(st, msg.c_str());
    return st;
}

lpa_status cuda_err(cudaError_t e, const char* where) {
    return err(e == cudaErrorMemoryAllocation ? LPA_ERR_OUT_OF_MEMORY : LPA_ERR_CUDA,
               std::string(where) + ": " + cudaGetErrorString(e));
}

#define SRV_CUDA(call)                                         \
    do {                                                       \
        cudaError_t e__ = (call);                              \
        if (e__ != cudaSuccess) return cuda_err(e__, #call);   \
    } while (0)

// ------------------------------------------------------------------ kernels
// New request at vertices [v0, v0+n), entries [e0, e0+nnz): the row offsets
// were copied as local positions; make them arena positions, make the
// indices arena vertex ids, set labels to ids and the slot of each vertex.
// The request's CSR is checked here (rows in order within [0, nnz], indices
// in [0, n), weights finite and >= 0); any failure sets bad[slot] and the
// request is never run.  A row found out of order is emptied so that no later
// read can leave the request's entry range.
__global__ void k_admit(int64_t* begin, int64_t* end, int32_t* idx, float* w, int32_t* lab0, int32_t* lab1,
                        int32_t* gid, int64_t v0, int64_t n, int64_t e0, int64_t nnz, int unit, int32_t slot,
                        int32_t* bad) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int fail = 0;
    for (int64_t i = t; i < n; i += stride) {
        int64_t b = begin[v0 + i], e = end[v0 + i];
        if (b < 0 || e < b || e > nnz) {
            fail = 1;
            b = e = 0;
        }
        begin[v0 + i] = b + e0;
        end[v0 + i] = e + e0;
        lab0[v0 + i] = (int32_t)(v0 + i);
        lab1[v0 + i] = (int32_t)(v0 + i);
        gid[v0 + i] = slot;
    }
    for (int64_t e = t; e < nnz; e += stride) {
        const int32_t j = idx[e0 + e];
        if (j < 0 || j >= n) {
            fail = 1;
            idx[e0 + e] = (int32_t)v0;
        } else {
            idx[e0 + e] = j + (int32_t)v0;
        }
        if (unit) {
            w[e0 + e] = 1.0f;
        } else {
            const float x = w[e0 + e];
            if (!isfinite(x) || x < 0.f) fail = 1;
        }
    }
    if (fail) atomicExch(&bad[slot], 1);
}

// Start of a request's run (Algorithm 1, lpa(): every vertex unprocessed).
// A request whose admission check failed starts done, with kExitInvalid as
// its exit reason, and no vertex marked: no sweep touches it.
constexpr int32_t kExitInvalid = -1;

__global__ void k_activate(const int64_t* begin, const int64_t* end, uint8_t* flags, int64_t v0, int64_t n,
                           int32_t slot, int32_t* done, int32_t* iters, int32_t* exit_reason,
                           unsigned long long* dN, long long* hist, int64_t* g_begin, int64_t* g_end,
                           const int32_t* bad) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool ok = bad[slot] == 0;
    for (int64_t i = t; i < n; i += stride) flags[v0 + i] = ok && end[v0 + i] > begin[v0 + i] ? 1 : 0;
    if (t < kMaxHist) hist[(int64_t)slot * kMaxHist + t] = 0;
    if (t == 0) {
        done[slot] = ok ? 0 : 1;
        iters[slot] = 0;
        exit_reason[slot] = ok ? 0 : kExitInvalid;
        dN[slot] = 0;
        g_begin[slot] = v0;
        g_end[slot] = v0 + n;
    }
}

__global__ void k_release(int64_t* begin, int64_t* end, int32_t* gid, uint8_t* flags, int64_t v0, int64_t n,
                          int32_t* bad, int32_t slot) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    if (blockIdx.x == 0 && threadIdx.x == 0) bad[slot] = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        begin[v0 + i] = 0;
        end[v0 + i] = 0;
        gid[v0 + i] = -1;
        flags[v0 + i] = 0;
    }
}

__global__ void k_ctrl_init(Ctrl* c, double tau, int max_iters, int mode) {
    c->tau = tau;
    c->max_iters = max_iters;
    c->mode = mode;
    c->allow_dense = 0;
    c->skip_marks = 0;
    c->cbuf = 0;
    c->rd = 0;
    c->stall_copy = 0;
}

// ---------------------------------------------------------------- allocator
// First-fit over free [start, start+len) intervals.
struct RangeAlloc {
    std::map<int64_t, int64_t> free_;   // start -> len
    int64_t cap_ = 0;
    explicit RangeAlloc(int64_t cap = 0) : cap_(cap) {
        if (cap > 0) free_[0] = cap;
    }
    bool alloc(int64_t len, int64_t* out) {
        if (len == 0) {
            *out = 0;
            return true;
        }
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= len) {
                *out = it->first;
                const int64_t s = it->first + len, l = it->second - len;
                free_.erase(it);
                if (l > 0) free_[s] = l;
                return true;
            }
        }
        return false;
    }
    void release(int64_t start, int64_t len) {
        if (len == 0) return;
        auto it = free_.emplace(start, len).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
    int64_t high_water() const {   // one past the highest allocated position
        if (free_.empty()) return cap_;
        const auto& last = *free_.rbegin();
        return last.first + last.second == cap_ ? last.first : cap_;
    }
};

struct Result {
    int state = 0;              // 0 queued, 1 running, 2 done, 3 failed
    std::vector<int32_t> labels;
    lpa_run_info info{};
    lpa_status status = LPA_OK;
    std::string error;
};

struct Request {
    uint64_t ticket;
    int64_t n, nnz;
    int32_t slot = -1;
    int64_t v0 = 0, e0 = 0;
    cudaEvent_t ready = nullptr;
    // solo lane: the CSR uploaded at submit (stream-ordered allocations)
    int64_t* d_off = nullptr;
    int32_t* d_idx = nullptr;
    float* d_w = nullptr;
    bool weighted = false;
    int64_t est_bytes = 0;
};

}  // namespace

struct lpa_server {
    lpa_serve_config cfg{};
    int device = 0;
    int sms = 1;
    int64_t V = 0, E = 0;
    int32_t S = 0;
    DevState s{};
    std::vector<void*> owned;
    int64_t arena_bytes = 0;
    cudaStream_t run_st = nullptr, copy_st = nullptr, solo_st = nullptr, solo_copy_st = nullptr;
    int32_t* h_done = nullptr;                // pinned mirror of done[S]
    int32_t* bad = nullptr;                   // [S] admission check failed
    // host state (guarded by mu)
    std::mutex mu;
    std::condition_variable cv;
    RangeAlloc vfree, efree;
    std::vector<int32_t> free_slots;
    std::deque<Request*> pending;             // copied, waiting for activation
    std::unordered_map<int32_t, Request*> active;
    std::deque<Request*> solo_q;
    int64_t solo_bytes = 0;
    std::unordered_map<uint64_t, Result> results;
    std::deque<uint64_t> finished;            // not yet reported by poll
    uint64_t next_ticket = 1;
    bool stop = false;
    std::thread worker, solo_worker;
    std::atomic<long long> cycles{0};
    std::string fatal;
};

namespace {

lpa_status dalloc(lpa_server* S, void** p, size_t bytes) {
    cudaError_t e = cudaMalloc(p, bytes ? bytes : 16);
    if (e != cudaSuccess) return cuda_err(e, "cudaMalloc(arena)");
    S->owned.push_back(*p);
    S->arena_bytes += (int64_t)bytes;
    return LPA_OK;
}

template <typename T>
lpa_status dalloc_t(lpa_server* S, T** p, size_t count) {
    return dalloc(S, reinterpret_cast<void**>(p), count * sizeof(T));
}

void free_server(lpa_server* S) {
    for (void* p : S->owned) cudaFree(p);
    S->owned.clear();
    if (S->h_done) cudaFreeHost(S->h_done);
    if (S->run_st) cudaStreamDestroy(S->run_st);
    if (S->copy_st) cudaStreamDestroy(S->copy_st);
    if (S->solo_st) cudaStreamDestroy(S->solo_st);
    if (S->solo_copy_st) cudaStreamDestroy(S->solo_copy_st);
}

int grid_for(int64_t n, int sms) {
    int64_t b = (n + 255) / 256;
    return (int)std::max<int64_t>(1, std::min<int64_t>(b, (int64_t)sms * 8));
}

// One cycle over the arena: compaction, one sweep (two passes in async mode),
// per-slot control.  Leaves the done flags in S->h_done.
cudaError_t run_cycle(lpa_server* S) {
    DevState s = S->s;
    const int mode = S->cfg.mode == LPA_MODE_ASYNC ? MODE_ASYNC : MODE_SYNC;
    cudaGraphConditionalHandle none = 0;
    cudaStream_t st = S->run_st;
    const int passes = mode == MODE_ASYNC ? 2 : 1;
    cudaError_t e = cudaSuccess;
    for (int p = 0; p < passes && e == cudaSuccess; ++p) {
        // compaction: the cycle's frontier, then (async) the catch-up set
        e = launch_finish(s, mode, p == 0 ? kRoleStartSweep : kRoleCatchUp, none, 0, st, S->sms);
        if (e == cudaSuccess) e = launch_sweep_small(s, mode, st, S->sms);
        if (e == cudaSuccess) e = launch_sweep_warp(s, mode, st, S->sms);
        for (int b = 2; b < kBins && e == cudaSuccess; ++b)
            e = launch_sweep_block(s, mode, b, S->sms, st);
    }
    if (e == cudaSuccess) e = launch_finish(s, mode, kRoleControl, none, 0, st, S->sms);   // apply + control
    if (e == cudaSuccess) e = cudaMemcpyAsync(S->h_done, s.done, (size_t)S->S * 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    return e;
}

void retire_arena(lpa_server* S, Request* r) {
    Result res;
    res.state = 2;
    res.labels.resize((size_t)r->n);
    std::vector<long long> hist(kMaxHist);
    int32_t it = 0, ex = 0;
    cudaStream_t st = S->run_st;
    const int32_t* C = S->s.lab[0];          // serving never flips the label buffers
    cudaError_t e = cudaSuccess;
    if (r->n) e = cudaMemcpyAsync(res.labels.data(), C + r->v0, (size_t)r->n * 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&it, S->s.iters + r->slot, 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&ex, S->s.exit_reason + r->slot, 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(hist.data(), S->s.hist_changed + (int64_t)r->slot * kMaxHist, kMaxHist * 8,
                            cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && r->n) {
        k_release<<<grid_for(r->n, S->sms), 256, 0, st>>>(const_cast<int64_t*>(S->s.off),
                                                         const_cast<int64_t*>(S->s.off_end),
                                                         const_cast<int32_t*>(S->s.gid), S->s.flags, r->v0, r->n,
                                                         S->bad, r->slot);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        res.state = 3;
        res.status = LPA_ERR_CUDA;
        res.error = cudaGetErrorString(e);
    } else if (ex == kExitInvalid) {
        res = Result{};
        res.state = 3;
        res.status = LPA_ERR_INVALID_GRAPH;
        res.error = "request CSR failed validation: row offsets out of order or beyond nnz, an index outside "
                    "[0, n), or a weight negative or not finite";
    } else {
        for (auto& x : res.labels) x -= (int32_t)r->v0;
        res.info.iterations = it;
        res.info.exit_reason = ex;
        for (int t = 0; t < std::min(it, kMaxHist); ++t) res.info.changed[t] = hist[t];
    }
    std::lock_guard<std::mutex> lock(S->mu);
    S->vfree.release(r->v0, r->n);
    S->efree.release(r->e0, r->nnz);
    S->free_slots.push_back(r->slot);
    S->active.erase(r->slot);
    S->results[r->ticket] = std::move(res);
    S->finished.push_back(r->ticket);
    if (r->ready) cudaEventDestroy(r->ready);
    delete r;
}

void worker_main(lpa_server* S) {
    cudaSetDevice(S->device);
    for (;;) {
        std::vector<Request*> to_activate;
        {
            std::unique_lock<std::mutex> lock(S->mu);
            S->cv.wait_for(lock, std::chrono::milliseconds(2),
                           [&] { return S->stop || !S->pending.empty() || !S->active.empty(); });
            if (S->stop) return;
            for (auto it = S->pending.begin(); it != S->pending.end();) {
                if (cudaEventQuery((*it)->ready) == cudaSuccess) {
                    to_activate.push_back(*it);
                    it = S->pending.erase(it);
                } else {
                    ++it;
                }
            }
            if (S->active.empty() && to_activate.empty()) {
                if (!S->pending.empty()) {           // copies still in flight
                    lock.unlock();
                    std::this_thread::sleep_for(std::chrono::microseconds(50));
                }
                continue;
            }
            // vertices past the highest allocated range have no marks: bound the compaction
            S->s.N = std::max<int64_t>(S->vfree.high_water(), 1);
        }
        cudaError_t e = cudaSuccess;
        for (Request* r : to_activate) {
            {
                std::lock_guard<std::mutex> lock(S->mu);
                S->results[r->ticket].state = 1;
                S->active[r->slot] = r;
            }
            k_activate<<<grid_for(std::max<int64_t>(r->n, kMaxHist), S->sms), 256, 0, S->run_st>>>(
                S->s.off, S->s.off_end, S->s.flags, r->v0, r->n, r->slot, S->s.done, S->s.iters, S->s.exit_reason,
                S->s.dN, S->s.hist_changed, const_cast<int64_t*>(S->s.g_begin), const_cast<int64_t*>(S->s.g_end),
                S->bad);
            if (e == cudaSuccess) e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = run_cycle(S);
        S->cycles++;
        if (e != cudaSuccess) {
            std::lock_guard<std::mutex> lock(S->mu);
            S->fatal = std::string("serving cycle: ") + cudaGetErrorString(e);
            S->stop = true;
            return;
        }
        std::vector<Request*> done;
        {
            std::lock_guard<std::mutex> lock(S->mu);
            for (auto& kv : S->active)
                if (S->h_done[kv.first]) done.push_back(kv.second);
        }
        for (Request* r : done) retire_arena(S, r);
    }
}

void free_solo_upload(lpa_server* S, Request* r) {
    if (r->d_off) cudaFreeAsync(r->d_off, S->solo_st);
    if (r->d_idx) cudaFreeAsync(r->d_idx, S->solo_st);
    if (r->d_w) cudaFreeAsync(r->d_w, S->solo_st);
    r->d_off = nullptr;
    r->d_idx = nullptr;
    r->d_w = nullptr;
}

void solo_main(lpa_server* S) {
    cudaSetDevice(S->device);
    for (;;) {
        Request* r = nullptr;
        {
            std::unique_lock<std::mutex> lock(S->mu);
            S->cv.wait_for(lock, std::chrono::milliseconds(5), [&] { return S->stop || !S->solo_q.empty(); });
            if (S->stop) return;
            if (S->solo_q.empty()) continue;
            r = S->solo_q.front();
            S->solo_q.pop_front();
            S->results[r->ticket].state = 1;
        }
        Result res;
        lpa_graph_t g = nullptr;
        // borrowed device CSR: validated on the device by lpa_graph_create
        lpa_status st = lpa_graph_create(r->n, r->nnz, r->d_off, r->d_idx, r->weighted ? r->d_w : nullptr,
                                         LPA_DEVICE_PTRS | LPA_BORROW, S->solo_st, &g);
        int32_t* lab = nullptr;
        if (st == LPA_OK &&
            cudaMallocAsync(&lab, (size_t)std::max<int64_t>(r->n, 1) * 4, S->solo_st) != cudaSuccess) {
            cudaGetLastError();
            st = LPA_ERR_OUT_OF_MEMORY;
        }
        const lpa_mode mode = S->cfg.mode == LPA_MODE_ASYNC ? LPA_MODE_ASYNC : LPA_MODE_SYNC;
        if (st == LPA_OK) st = lpa_run(g, mode, S->cfg.tolerance, S->cfg.max_iters, lab, S->solo_st, &res.info);
        if (st == LPA_OK) {
            res.labels.resize((size_t)r->n);
            if (r->n && (cudaMemcpyAsync(res.labels.data(), lab, (size_t)r->n * 4, cudaMemcpyDeviceToHost,
                                         S->solo_st) != cudaSuccess ||
                         cudaStreamSynchronize(S->solo_st) != cudaSuccess))
                st = LPA_ERR_CUDA;
        }
        if (st != LPA_OK) {
            res.state = 3;
            res.status = st;
            res.error = lpa_last_error();
        } else {
            res.state = 2;
        }
        if (g) lpa_graph_destroy(g);
        if (lab) cudaFreeAsync(lab, S->solo_st);
        free_solo_upload(S, r);
        cudaStreamSynchronize(S->solo_st);
        std::lock_guard<std::mutex> lock(S->mu);
        S->solo_bytes -= r->est_bytes;
        S->results[r->ticket] = std::move(res);
        S->finished.push_back(r->ticket);
        delete r;
    }
}

bool host_pinned(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeHost;
}

}  // namespace

extern "C" {

lpa_status lpa_serve_create(const lpa_serve_config* cfg, lpa_server_t* out) {
    if (!cfg || !out) return err(LPA_ERR_INVALID_ARG, "NULL argument");
    if (cfg->arena_vertices < 1 || cfg->arena_entries < 1 || cfg->max_slots < 2)
        return err(LPA_ERR_INVALID_ARG, "arena_vertices and arena_entries must be >= 1, max_slots >= 2");
    if (cfg->arena_vertices > 0x7fffffffLL) return err(LPA_ERR_INVALID_ARG, "arena_vertices above 2^31-1");
    if (cfg->mode < 0 || cfg->mode > 2) return err(LPA_ERR_INVALID_ARG, "unknown mode");
    if (!(cfg->tolerance >= 0.0 && cfg->tolerance <= 1.0)) return err(LPA_ERR_INVALID_ARG, "tolerance must be in [0, 1]");
    if (cfg->max_iters < 0 || cfg->max_iters > (1 << 20)) return err(LPA_ERR_INVALID_ARG, "max_iters out of range");
    lpa_server* S = new (std::nothrow) lpa_server();
    if (!S) return err(LPA_ERR_OUT_OF_MEMORY, "host allocation");
    S->cfg = *cfg;
    S->V = cfg->arena_vertices;
    S->E = cfg->arena_entries;
    S->S = cfg->max_slots;
    lpa_status rs = LPA_OK;
    auto bail = [&](lpa_status st) {
        free_server(S);
        delete S;
        return st;
    };
    if (cudaGetDevice(&S->device) != cudaSuccess) return bail(err(LPA_ERR_CUDA, "cudaGetDevice"));
    cudaDeviceGetAttribute(&S->sms, cudaDevAttrMultiProcessorCount, S->device);
    DevState& s = S->s;
    const size_t V = (size_t)S->V, E = (size_t)S->E, G = (size_t)S->S;
    int64_t *begin, *end, *gb, *ge;
    int32_t *idx, *gid;
    float* w;
    if ((rs = dalloc_t(S, &begin, V)) || (rs = dalloc_t(S, &end, V)) || (rs = dalloc_t(S, &idx, E)) ||
        (rs = dalloc_t(S, &w, E)) || (rs = dalloc_t(S, &gid, V)) || (rs = dalloc_t(S, &gb, G)) ||
        (rs = dalloc_t(S, &ge, G)) || (rs = dalloc_t(S, &s.lab[0], V)) || (rs = dalloc_t(S, &s.lab[1], V)) ||
        (rs = dalloc_t(S, &s.flags, V + 16)) || (rs = dalloc_t(S, &s.fr_bits, V / 16 + 1)) ||
        (rs = dalloc_t(S, &s.slist, 1)) ||
        (rs = dalloc_t(S, &s.flist, V * kBins)) || (rs = dalloc_t(S, &s.chg, V * kBins)) ||
        (rs = dalloc_t(S, &s.ctrl, 1)) || (rs = dalloc_t(S, &s.dN, G)) || (rs = dalloc_t(S, &s.done, G)) ||
        (rs = dalloc_t(S, &s.iters, G)) || (rs = dalloc_t(S, &s.exit_reason, G)) ||
        (rs = dalloc_t(S, &s.hist_changed, G * kMaxHist)) || (rs = dalloc_t(S, &s.ovf, E / 2048 + 1)) ||
        (rs = dalloc_t(S, &S->bad, G)))
        return bail(rs);
    if (S->arena_bytes > cfg->hbm_budget_bytes)
        return bail(err(LPA_ERR_INVALID_ARG, "arena sizes exceed hbm_budget_bytes"));
    auto zero = [&](void* p, size_t b) { return cudaMemset(p, 0, b) == cudaSuccess; };
    bool ok = zero(begin, V * 8) && zero(end, V * 8) && zero(s.flags, V + 16) && zero(s.ctrl, sizeof(Ctrl)) &&
              zero(s.dN, G * 8) && zero(s.iters, G * 4) && zero(s.exit_reason, G * 4) &&
              cudaMemset(gid, 0xff, V * 4) == cudaSuccess && zero(gb, G * 8) && zero(ge, G * 8) && zero(S->bad, G * 4);
    std::vector<int32_t> ones(G, 1);
    ok = ok && cudaMemcpy(s.done, ones.data(), G * 4, cudaMemcpyHostToDevice) == cudaSuccess;
    if (!ok) return bail(err(LPA_ERR_CUDA, "arena initialisation failed"));
    s.N = S->V;
    s.E = S->E;
    s.G = S->S;                    // >= 2: the per-graph (batched) kernel variants
    s.weight_kind = W_F32;
    s.off = begin;
    s.off_end = end;
    s.idx = idx;
    s.w = w;
    s.gid = gid;
    s.vtx_off = gb;
    s.g_begin = gb;
    s.g_end = ge;
    s.small_max = 4;
    s.warp_max = 128;
    s.mid_max = 512;
    s.large_max = 2048;
    s.warp_slots = 256;
    s.block_slots[0] = 1024;
    s.block_slots[1] = 4096;
    s.block_slots[2] = kLargeSlots;
    // overflowing rows take the rescan path (no sliced scratch in the arena)
    s.ovf_pairs = nullptr;
    s.ovf_cnt = nullptr;
    s.ovf_off = nullptr;
    s.ovf_pairs_cap = 0;
    s.ovf_cnt_cap = 0;
    s.ovf_possible = 1;
    s.dense_permille = 1001;
    for (int b = 0; b < kBins; ++b) {
        s.bin_base[b] = (int64_t)b * S->V;
        s.bin_static[b] = 0;
        s.bin_static_entries[b] = 0;
    }
    s.active_entries = S->E;
    k_ctrl_init<<<1, 1>>>(s.ctrl, cfg->tolerance, cfg->max_iters,
                          cfg->mode == LPA_MODE_ASYNC ? MODE_ASYNC : MODE_SYNC);
    if (cudaDeviceSynchronize() != cudaSuccess) return bail(err(LPA_ERR_CUDA, "control initialisation failed"));
    if (cudaMallocHost(&S->h_done, G * 4) != cudaSuccess) return bail(err(LPA_ERR_OUT_OF_MEMORY, "pinned buffer"));
    // arena streams first, the solo lane's at the lowest priority: a large
    // request runs in the gaps left by the arena's cycles
    int prio_low = 0, prio_high = 0;
    cudaDeviceGetStreamPriorityRange(&prio_low, &prio_high);
    if (cudaStreamCreateWithPriority(&S->run_st, cudaStreamNonBlocking, prio_high) != cudaSuccess ||
        cudaStreamCreateWithPriority(&S->copy_st, cudaStreamNonBlocking, prio_high) != cudaSuccess ||
        cudaStreamCreateWithPriority(&S->solo_st, cudaStreamNonBlocking, prio_low) != cudaSuccess ||
        cudaStreamCreateWithPriority(&S->solo_copy_st, cudaStreamNonBlocking, prio_low) != cudaSuccess)
        return bail(err(LPA_ERR_CUDA, "stream creation failed"));
    S->vfree = RangeAlloc(S->V);
    S->efree = RangeAlloc(S->E);
    for (int32_t k = S->S - 1; k >= 0; --k) S->free_slots.push_back(k);
    S->worker = std::thread(worker_main, S);
    S->solo_worker = std::thread(solo_main, S);
    *out = S;
    return LPA_OK;
}

lpa_status lpa_serve_submit(lpa_server_t S, int64_t n, int64_t nnz, const int64_t* offsets, const int32_t* indices,
                            const float* weights, uint64_t* ticket) {
    if (!S || !ticket) return err(LPA_ERR_INVALID_ARG, "NULL argument");
    if (n < 0 || n > 0x7fffffffLL || nnz < 0) return err(LPA_ERR_INVALID_ARG, "n or nnz out of range");
    if (!offsets || (nnz > 0 && !indices)) return err(LPA_ERR_INVALID_ARG, "offsets or indices is NULL");
    const bool solo = S->cfg.solo_min_entries > 0 && nnz >= S->cfg.solo_min_entries;
    if (offsets[0] != 0 || offsets[n] != nnz) return err(LPA_ERR_INVALID_GRAPH, "offsets must start at 0 and end at nnz");

    {
        std::lock_guard<std::mutex> lock(S->mu);
        if (!S->fatal.empty()) return err(LPA_ERR_CUDA, S->fatal);
    }
    Request* r = new Request();
    r->n = n;
    r->nnz = nnz;
    r->weighted = weights != nullptr;
    if (n == 0 || solo) {
        std::lock_guard<std::mutex> lock(S->mu);
        if (solo) {
            r->est_bytes = nnz * 8 + n * 64 + (int64_t)(64 << 20);
            if (S->arena_bytes + S->solo_bytes + r->est_bytes > S->cfg.hbm_budget_bytes) {
                delete r;
                return err(LPA_ERR_BUSY, "request does not fit the device-memory budget now");
            }
            S->solo_bytes += r->est_bytes;
        }
        r->ticket = S->next_ticket++;
        *ticket = r->ticket;
        if (n == 0) {
            Result res;
            res.state = 2;
            res.info.exit_reason = 2;
            S->results[r->ticket] = std::move(res);
            S->finished.push_back(r->ticket);
            delete r;
            return LPA_OK;
        }
        S->results[r->ticket] = Result();
    }
    if (solo) {
        // upload on the solo copy stream and wait, so the caller may reuse its buffers
        cudaStream_t st = S->solo_copy_st;
        cudaError_t e = cudaMallocAsync(&r->d_off, (size_t)(n + 1) * 8, st);
        if (e == cudaSuccess && nnz) e = cudaMallocAsync(&r->d_idx, (size_t)nnz * 4, st);
        if (e == cudaSuccess && nnz && weights) e = cudaMallocAsync(&r->d_w, (size_t)nnz * 4, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(r->d_off, offsets, (size_t)(n + 1) * 8, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess && nnz) e = cudaMemcpyAsync(r->d_idx, indices, (size_t)nnz * 4, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess && nnz && weights)
            e = cudaMemcpyAsync(r->d_w, weights, (size_t)nnz * 4, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        std::lock_guard<std::mutex> lock(S->mu);
        if (e != cudaSuccess) {
            cudaGetLastError();
            if (r->d_off) cudaFreeAsync(r->d_off, st);
            if (r->d_idx) cudaFreeAsync(r->d_idx, st);
            if (r->d_w) cudaFreeAsync(r->d_w, st);
            S->solo_bytes -= r->est_bytes;
            S->results.erase(r->ticket);
            delete r;
            return err(e == cudaErrorMemoryAllocation ? LPA_ERR_OUT_OF_MEMORY : LPA_ERR_CUDA, "solo upload failed");
        }
        S->solo_q.push_back(r);
        S->cv.notify_all();
        return LPA_OK;
    }
    {
        std::lock_guard<std::mutex> lock(S->mu);
        int64_t v0 = 0, e0 = 0;
        if (S->free_slots.empty() || !S->vfree.alloc(n, &v0)) {
            delete r;
            return err(LPA_ERR_BUSY, "no free slot or vertex range in the arena now");
        }
        if (!S->efree.alloc(nnz, &e0)) {
            S->vfree.release(v0, n);
            delete r;
            return err(LPA_ERR_BUSY, "no free entry range in the arena now");
        }
        r->slot = S->free_slots.back();
        S->free_slots.pop_back();
        r->v0 = v0;
        r->e0 = e0;
        r->ticket = S->next_ticket++;
        S->results[r->ticket] = Result();
    }
    cudaStream_t st = S->copy_st;
    DevState& s = S->s;
    cudaError_t e = cudaMemcpyAsync(const_cast<int64_t*>(s.off) + r->v0, offsets, (size_t)n * 8, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(const_cast<int64_t*>(s.off_end) + r->v0, offsets + 1, (size_t)n * 8, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && nnz)
        e = cudaMemcpyAsync(const_cast<int32_t*>(s.idx) + r->e0, indices, (size_t)nnz * 4, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && nnz && weights)
        e = cudaMemcpyAsync(const_cast<float*>(static_cast<const float*>(s.w)) + r->e0, weights, (size_t)nnz * 4,
                            cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) {
        k_admit<<<grid_for(std::max(n, nnz), S->sms), 256, 0, st>>>(
            const_cast<int64_t*>(s.off), const_cast<int64_t*>(s.off_end), const_cast<int32_t*>(s.idx),
            const_cast<float*>(static_cast<const float*>(s.w)), s.lab[0], s.lab[1], const_cast<int32_t*>(s.gid), r->v0,
            n, r->e0, nnz, weights ? 0 : 1, r->slot, S->bad);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&r->ready, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(r->ready, st);
    // Page-locked inputs are read by DMA after this call is enqueued: wait for
    // the copies when any of the three arrays is page-locked, so the caller
    // may reuse its buffers on return.  (Pageable inputs were staged by the
    // copies themselves before they returned.)
    if (e == cudaSuccess && (host_pinned(offsets) || host_pinned(indices) || host_pinned(weights)))
        e = cudaEventSynchronize(r->ready);
    std::lock_guard<std::mutex> lock(S->mu);
    if (e != cudaSuccess) {
        S->vfree.release(r->v0, n);
        S->efree.release(r->e0, nnz);
        S->free_slots.push_back(r->slot);
        S->results.erase(r->ticket);
        delete r;
        return cuda_err(e, "admission copies");
    }
    *ticket = r->ticket;
    S->pending.push_back(r);
    S->cv.notify_all();
    return LPA_OK;
}

lpa_status lpa_serve_poll(lpa_server_t S, uint64_t* done, int32_t cap, int32_t* n_done) {
    if (!S || !n_done || cap < 0 || (cap > 0 && !done)) return err(LPA_ERR_INVALID_ARG, "bad argument");
    std::lock_guard<std::mutex> lock(S->mu);
    int32_t k = 0;
    while (k < cap && !S->finished.empty()) {
        done[k++] = S->finished.front();
        S->finished.pop_front();
    }
    *n_done = k;
    if (!S->fatal.empty()) return err(LPA_ERR_CUDA, S->fatal);
    return LPA_OK;
}

lpa_status lpa_serve_fetch(lpa_server_t S, uint64_t ticket, int32_t* labels_host, lpa_run_info* info) {
    if (!S) return err(LPA_ERR_INVALID_ARG, "server is NULL");
    std::lock_guard<std::mutex> lock(S->mu);
    auto it = S->results.find(ticket);
    if (it == S->results.end()) return err(LPA_ERR_NOT_FOUND, "unknown ticket");
    Result& r = it->second;
    if (r.state < 2) return err(LPA_ERR_NOT_READY, "request not finished");
    if (r.state == 3) return err(r.status, r.error);
    if (labels_host && !r.labels.empty()) memcpy(labels_host, r.labels.data(), r.labels.size() * 4);
    if (info) *info = r.info;
    return LPA_OK;
}

lpa_status lpa_serve_release(lpa_server_t S, uint64_t ticket) {
    if (!S) return err(LPA_ERR_INVALID_ARG, "server is NULL");
    std::lock_guard<std::mutex> lock(S->mu);
    auto it = S->results.find(ticket);
    if (it == S->results.end()) return err(LPA_ERR_NOT_FOUND, "unknown ticket");
    if (it->second.state < 2) return err(LPA_ERR_NOT_READY, "request not finished");
    S->results.erase(it);
    return LPA_OK;
}

lpa_status lpa_serve_stats(lpa_server_t S, lpa_serve_stats_t* out) {
    if (!S || !out) return err(LPA_ERR_INVALID_ARG, "NULL argument");
    std::lock_guard<std::mutex> lock(S->mu);
    memset(out, 0, sizeof(*out));
    out->cycles = S->cycles.load();
    out->active = (int32_t)S->active.size();
    out->pending = (int32_t)(S->pending.size() + S->solo_q.size());
    out->arena_bytes = S->arena_bytes;
    out->solo_bytes = S->solo_bytes;
    return LPA_OK;
}

lpa_status lpa_serve_destroy(lpa_server_t S) {
    if (!S) return err(LPA_ERR_INVALID_ARG, "server is NULL");
    {
        std::lock_guard<std::mutex> lock(S->mu);
        S->stop = true;
        S->cv.notify_all();
    }
    if (S->worker.joinable()) S->worker.join();
    if (S->solo_worker.joinable()) S->solo_worker.join();
    cudaDeviceSynchronize();
    for (Request* r : S->pending) {
        if (r->ready) cudaEventDestroy(r->ready);
        delete r;
    }
    for (auto& kv : S->active) {
        if (kv.second->ready) cudaEventDestroy(kv.second->ready);
        delete kv.second;
    }
    for (Request* r : S->solo_q) {
        free_solo_upload(S, r);
        delete r;
    }
    if (S->solo_st) cudaStreamSynchronize(S->solo_st);
    free_server(S);
    delete S;
    return LPA_OK;
}

}  // extern "C"
