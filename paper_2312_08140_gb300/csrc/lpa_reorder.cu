// lpa_reorder.cu -- storage orders of a graph or batch.
//
// The library may store a graph's vertices in an order of its own while
// labels stay the caller's vertex ids (Algorithm 1 starts from C_i = i and
// breaks ties by the smallest id: both refer to the original ids, so results
// are those of the caller's graph; only the memory layout and the order in
// which the parallel sweep meets the vertices change).  Two orders:
//
//   degree   every vertex by decreasing degree bucket ceil(log2 d), then by
//            id.  The heavy vertices' labels, which most gathers read, sit
//            together in memory (and in L2);
//   shuffle  each graph's vertices in a pseudo-random order of their own (a
//            Feistel permutation of the graph's id range).  The asynchronous
//            sweep walks stored vertices in order, so a graph spanning
//            several waves of warps is then met in a random order rather
//            than by increasing id -- with smallest-id ties, an increasing
//            visit lets the smallest ids flood id-ordered communities.
//
// orig[p] is the original id of stored vertex p and inv[v] the stored
// position of original vertex v.  Rows are rewritten through inv; a graph of
// a batch keeps its id range, so the graph of every vertex is unchanged.
#include <algorithm>
#include <vector>

#include "lpa_device.cuh"

namespace lpa {

constexpr int kReorderThreads = 256;
constexpr int kReorderPerThread = 16;
constexpr int kReorderChunk = kReorderThreads * kReorderPerThread;
constexpr int kOrderKeys = 32;                 // degree buckets 0..31 (d < 2^31)

// ---- shuffle: shuffle_pos (lpa_device.cuh) per graph ---------------------
__global__ void k_shuffle_inv(const int64_t* vtx_off, const int32_t* gid, int32_t G, int64_t N, uint64_t seed,
                              int32_t* inv) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < N; v += stride) {
        const int32_t g = G > 1 ? gid[v] : 0;
        const int64_t v0 = vtx_off[g];
        const uint32_t n = (uint32_t)(vtx_off[g + 1] - v0);
        inv[v] = (int32_t)(v0 + shuffle_pos((uint32_t)(v - v0), n, seed + 0x9E3779B97F4A7C15ull * (uint64_t)g));
    }
}

// ---- degree order: stable counting sort by decreasing degree bucket -------
__device__ __forceinline__ int order_key(const int64_t* off, int64_t v) {
    const int64_t d = off[v + 1] - off[v];
    const int b = d <= 1 ? 0 : 64 - __clzll((unsigned long long)(d - 1));
    return kOrderKeys - 1 - (b < kOrderKeys ? b : kOrderKeys - 1);
}

// counts[key * nblk + block]: vertices of each key in each chunk of vertices.
__global__ void __launch_bounds__(kReorderThreads) k_order_count(const int64_t* off, int64_t N, unsigned* counts) {
    __shared__ unsigned sc[kOrderKeys];
    if (threadIdx.x < kOrderKeys) sc[threadIdx.x] = 0;
    __syncthreads();
    const int64_t v0 = (int64_t)blockIdx.x * kReorderChunk + (int64_t)threadIdx.x * kReorderPerThread;
    for (int q = 0; q < kReorderPerThread; ++q)
        if (v0 + q < N) atomicAdd(&sc[order_key(off, v0 + q)], 1u);
    __syncthreads();
    if (threadIdx.x < kOrderKeys) counts[(size_t)threadIdx.x * gridDim.x + blockIdx.x] = sc[threadIdx.x];
}

// orig[base[key][block] + rank within the block] = v, the rank counting the
// chunk's earlier vertices of the same key (threads own consecutive runs of
// kReorderPerThread vertices; their per-key counts are scanned across the
// block), so the order within a key is by id.
__global__ void __launch_bounds__(kReorderThreads) k_order_scatter(const int64_t* off, int64_t N, const unsigned* base,
                                                                   int32_t* orig) {
    __shared__ unsigned warp_tot[kOrderKeys][kReorderThreads / 32];
    const int64_t v0 = (int64_t)blockIdx.x * kReorderChunk + (int64_t)threadIdx.x * kReorderPerThread;
    const unsigned lane = lane_id();
    const int w = threadIdx.x >> 5;
    unsigned char keys[kReorderPerThread];
    for (int q = 0; q < kReorderPerThread; ++q) keys[q] = (unsigned char)(v0 + q < N ? order_key(off, v0 + q) : 255);
    // per key: exclusive scan of this thread's count across the block
    for (int k = 0; k < kOrderKeys; ++k) {
        unsigned c = 0;
        for (int q = 0; q < kReorderPerThread; ++q) c += keys[q] == k ? 1u : 0u;
        unsigned incl = c;
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned y = __shfl_up_sync(kFull, incl, o);
            if ((int)lane >= o) incl += y;
        }
        if (lane == 31) warp_tot[k][w] = incl;
        __syncthreads();
        unsigned before = 0;
        for (int q = 0; q < w; ++q) before += warp_tot[k][q];
        unsigned pos = base[(size_t)k * gridDim.x + blockIdx.x] + before + incl - c;
        for (int q = 0; q < kReorderPerThread; ++q)
            if (keys[q] == k) orig[pos++] = (int32_t)(v0 + q);
        __syncthreads();
    }
}

// ---- shared steps -----------------------------------------------------------
__global__ void k_invert(const int32_t* from, int64_t N, int32_t* to) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += stride) to[from[i]] = (int32_t)i;
}

// Degrees of the stored rows, summed per chunk of kReorderChunk rows.
__global__ void __launch_bounds__(kReorderThreads) k_row_sums(const int32_t* orig, const int64_t* off, int64_t N,
                                                              unsigned long long* sums) {
    const int64_t p0 = (int64_t)blockIdx.x * kReorderChunk;
    unsigned long long t = 0;
    for (int64_t p = p0 + threadIdx.x; p < p0 + kReorderChunk && p < N; p += kReorderThreads) {
        const int32_t o = orig[p];
        t += (unsigned long long)(off[o + 1] - off[o]);
    }
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(kFull, t, o);
    __shared__ unsigned long long ws[kReorderThreads / 32];
    if (lane_id() == 0) ws[threadIdx.x >> 5] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long a = 0;
        for (int q = 0; q < kReorderThreads / 32; ++q) a += ws[q];
        sums[blockIdx.x] = a;
    }
}

// new_off[p + 1] for the stored rows of one chunk, from the chunk's base.
__global__ void __launch_bounds__(kReorderThreads) k_row_offsets(const int32_t* orig, const int64_t* off, int64_t N,
                                                                 const unsigned long long* bases, int64_t* new_off) {
    __shared__ unsigned long long ws[kReorderThreads / 32];
    const int64_t p0 = (int64_t)blockIdx.x * kReorderChunk;
    unsigned long long carry = bases[blockIdx.x];
    for (int64_t r0 = p0; r0 < p0 + kReorderChunk && r0 < N; r0 += kReorderThreads) {
        const int64_t p = r0 + threadIdx.x;
        unsigned long long d = 0;
        if (p < N) {
            const int32_t o = orig[p];
            d = (unsigned long long)(off[o + 1] - off[o]);
        }
        unsigned long long incl = d;
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(kFull, incl, o);
            if ((int)lane_id() >= o) incl += y;
        }
        if (lane_id() == 31) ws[threadIdx.x >> 5] = incl;
        __syncthreads();
        unsigned long long before = 0, all = 0;
        for (int q = 0; q < kReorderThreads / 32; ++q) {
            if (q < (int)(threadIdx.x >> 5)) before += ws[q];
            all += ws[q];
        }
        if (p < N) new_off[p + 1] = (int64_t)(carry + before + incl);
        carry += all;
        __syncthreads();
    }
}

// Stored row p = original row orig[p], its neighbours renumbered through
// inv; weights (wbytes per entry, 0 for unit weights) moved alongside.  One
// warp per row.
__global__ void k_permute_rows(const int32_t* orig, const int32_t* inv, const int64_t* off, const int32_t* idx,
                               const void* w, int wbytes, const int64_t* new_off, int64_t N, int32_t* new_idx,
                               void* new_w) {
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const unsigned lane = lane_id();
    for (int64_t p = warp; p < N; p += nwarps) {
        const int32_t o = orig[p];
        const int64_t s0 = off[o], d = off[o + 1] - s0, t0 = new_off[p];
        for (int64_t k = lane; k < d; k += 32) {
            new_idx[t0 + k] = inv[idx[s0 + k]];
            if (wbytes == 1)
                static_cast<unsigned char*>(new_w)[t0 + k] = static_cast<const unsigned char*>(w)[s0 + k];
            else if (wbytes == 4)
                static_cast<uint32_t*>(new_w)[t0 + k] = static_cast<const uint32_t*>(w)[s0 + k];
        }
    }
}

cudaError_t reorder_positions(int kind, const int64_t* off, const int64_t* vtx_off, const int32_t* gid, int32_t G,
                              int64_t N, uint64_t seed, int32_t* orig, int32_t* inv, unsigned* scratch,
                              cudaStream_t st, int sms) {
    if (N == 0) return cudaSuccess;
    cudaError_t e;
    if (kind == kOrderShuffle) {
        k_shuffle_inv<<<sms * 8, 256, 0, st>>>(vtx_off, gid, G, N, seed, inv);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        k_invert<<<sms * 8, 256, 0, st>>>(inv, N, orig);
        return cudaGetLastError();
    }
    // degree order
    const int64_t nblk = (N + kReorderChunk - 1) / kReorderChunk;
    k_order_count<<<(unsigned)nblk, kReorderThreads, 0, st>>>(off, N, scratch);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    std::vector<unsigned> h((size_t)nblk * kOrderKeys);
    if ((e = cudaMemcpyAsync(h.data(), scratch, h.size() * 4, cudaMemcpyDeviceToHost, st)) != cudaSuccess) return e;
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
    unsigned run = 0;
    for (auto& x : h) {
        const unsigned c = x;
        x = run;
        run += c;
    }
    if ((e = cudaMemcpyAsync(scratch, h.data(), h.size() * 4, cudaMemcpyHostToDevice, st)) != cudaSuccess) return e;
    k_order_scatter<<<(unsigned)nblk, kReorderThreads, 0, st>>>(off, N, scratch, orig);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_invert<<<sms * 8, 256, 0, st>>>(orig, N, inv);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    return cudaStreamSynchronize(st);        // `h` is read by the copy above
}

int64_t reorder_scratch_words(int64_t N) {
    const int64_t nblk = (N + kReorderChunk - 1) / kReorderChunk;
    return std::max<int64_t>(nblk * kOrderKeys, 2 * nblk + 2);
}

cudaError_t reorder_rows(const int32_t* orig, const int32_t* inv, const int64_t* off, const int32_t* idx,
                         const void* w, int wbytes, int64_t N, int64_t* new_off, int32_t* new_idx, void* new_w,
                         unsigned long long* scratch, cudaStream_t st, int sms) {
    cudaError_t e = cudaMemsetAsync(new_off, 0, sizeof(int64_t), st);
    if (e != cudaSuccess || N == 0) return e;
    const int64_t nblk = (N + kReorderChunk - 1) / kReorderChunk;
    k_row_sums<<<(unsigned)nblk, kReorderThreads, 0, st>>>(orig, off, N, scratch);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    std::vector<unsigned long long> h((size_t)nblk);
    if ((e = cudaMemcpyAsync(h.data(), scratch, h.size() * 8, cudaMemcpyDeviceToHost, st)) != cudaSuccess) return e;
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
    unsigned long long run = 0;
    for (auto& x : h) {
        const unsigned long long c = x;
        x = run;
        run += c;
    }
    if ((e = cudaMemcpyAsync(scratch, h.data(), h.size() * 8, cudaMemcpyHostToDevice, st)) != cudaSuccess) return e;
    k_row_offsets<<<(unsigned)nblk, kReorderThreads, 0, st>>>(orig, off, N, scratch, new_off);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_permute_rows<<<sms * 8, 256, 0, st>>>(orig, inv, off, idx, w, wbytes, new_off, N, new_idx, new_w);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    return cudaStreamSynchronize(st);        // `h` is read by the copy above
}

}  // namespace lpa
