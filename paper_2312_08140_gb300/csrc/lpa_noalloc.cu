// lpa_noalloc.cu -- modularity of a labelling without any device allocation.
//
// Who needs this: code that is not allowed to call cudaMalloc / cudaFree --
// for example a plugin inside a host framework that owns every byte of device
// memory through its own pool and budget, or a latency-critical serving loop
// in which an allocation (and the device synchronisation cudaFree implies) is
// not acceptable.  Such callers cannot create an lpa_graph_t (which allocates
// its CSR copy and working state), yet may still want Q for labels they
// computed.
//
// How: the working memory of the two modularity kernels (one fp64 total per
// community and the fp64 accumulators) is a fixed file-scope __device__ array
// sized for kNoAllocMaxVertices vertices.  Every GPU that loads this library
// holds it (about 8 MiB) until the process exits.  Host code cannot use the
// array's name as a device address, so the first call on each device (with
// that device current) looks the address up with cudaGetSymbolAddress and
// keeps it for later calls in the same CUDA context; a new context on that
// device (after cudaDeviceReset, say) gets a new lookup.  That first call
// should come before any stream capture.  All calls share the array: each
// call clears what must start at zero, and two calls that run on the GPU at
// the same time (other streams, other host threads) race -- serialise them.
#include <cuda.h>
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/lpa.h"
#include "lpa_internal.h"

using namespace lpa;

namespace lpa {
void set_last_error(lpa_status st, const char* msg);
}

namespace {

constexpr int64_t kNoAllocMaxVertices = 1 << 20;
constexpr size_t kSigmaBytes = (size_t)kNoAllocMaxVertices * sizeof(double);
constexpr size_t kScratchBytes = kSigmaBytes + 256;   // + ModAccum

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
struct DeviceScratch {
    unsigned long long ctx_id = 0;   // CUDA context the address belongs to (0: none yet)
    void* addr = nullptr;
    int sms = 1;
};
DeviceScratch g_scratch[kMaxDevices];

// Driver entry points that identify the current context (resolved through
// the runtime, so the library needs no link to the driver library).
using ctx_get_current_fn = CUresult (*)(CUcontext*);
using ctx_get_id_fn = CUresult (*)(CUcontext, unsigned long long*);
ctx_get_current_fn g_ctx_get_current = nullptr;
ctx_get_id_fn g_ctx_get_id = nullptr;

lpa_status err(lpa_status st, const char* msg) {
    set_last_error(st, msg);
    return st;
}

lpa_status cuda_err(cudaError_t e) {
    set_last_error(LPA_ERR_CUDA, cudaGetErrorString(e));
    return LPA_ERR_CUDA;
}

// Id of the calling thread's current context, 0 if none is current.
lpa_status current_context_id(unsigned long long* id) {
    if (!g_ctx_get_current || !g_ctx_get_id) {
        void* f1 = nullptr;
        void* f2 = nullptr;
        cudaDriverEntryPointQueryResult q1, q2;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1);
        if (e == cudaSuccess)
            e = cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2);
        if (e != cudaSuccess) return cuda_err(e);
        if (q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess || !f1 || !f2)
            return err(LPA_ERR_CUDA, "driver entry points cuCtxGetCurrent / cuCtxGetId not found");
        g_ctx_get_current = reinterpret_cast<ctx_get_current_fn>(f1);
        g_ctx_get_id = reinterpret_cast<ctx_get_id_fn>(f2);
    }
    CUcontext ctx = nullptr;
    if (g_ctx_get_current(&ctx) != CUDA_SUCCESS) return err(LPA_ERR_CUDA, "cuCtxGetCurrent failed");
    *id = 0;
    if (ctx && g_ctx_get_id(ctx, id) != CUDA_SUCCESS) return err(LPA_ERR_CUDA, "cuCtxGetId failed");
    return LPA_OK;
}

// Device address of the scratch array on the current device, looked up once
// per device and context.
lpa_status scratch_for_current_device(void** out, int* sms) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_err(e);
    if (dev < 0 || dev >= kMaxDevices) return err(LPA_ERR_INVALID_ARG, "device index beyond 64");
    std::lock_guard<std::mutex> lock(g_mu);
    unsigned long long id = 0;
    lpa_status rs = current_context_id(&id);
    if (rs != LPA_OK) return rs;
    DeviceScratch& D = g_scratch[dev];
    if (id == 0 || D.ctx_id != id) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);    // makes the device's context current
        if (e != cudaSuccess) return cuda_err(e);
        int n = 0;
        e = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return cuda_err(e);
        if ((rs = current_context_id(&id)) != LPA_OK) return rs;
        D.ctx_id = id;
        D.addr = p;
        D.sms = n > 0 ? n : 1;
    }
    *out = D.addr;
    *sms = D.sms;
    return LPA_OK;
}

}  // namespace

extern "C" lpa_status lpa_modularity_noalloc(int64_t n, int64_t nnz, const int64_t* offsets,
                                             const int32_t* indices, const float* weights,
                                             const int32_t* labels, double* q_out, void* stream) {
    if (!q_out) return err(LPA_ERR_INVALID_ARG, "q_out is NULL");
    if (n < 0 || nnz < 0) return err(LPA_ERR_INVALID_ARG, "n and nnz must be >= 0");
    if (n > kNoAllocMaxVertices)
        return err(LPA_ERR_INVALID_ARG,
                   "n exceeds the 1048576-vertex limit of lpa_modularity_noalloc; use lpa_modularity");
    if (n > 0 && (!offsets || !labels)) return err(LPA_ERR_INVALID_ARG, "offsets or labels is NULL");
    if (nnz > 0 && !indices) return err(LPA_ERR_INVALID_ARG, "indices is NULL");
    if (n == 0) {
        *q_out = 0.0;
        return LPA_OK;
    }
    void* scratch = nullptr;
    int sms = 1;
    lpa_status rs = scratch_for_current_device(&scratch, &sms);
    if (rs != LPA_OK) return rs;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    double* Sigma = static_cast<double*>(scratch);
    ModAccum* acc = reinterpret_cast<ModAccum*>(static_cast<unsigned char*>(scratch) + kSigmaBytes);

    DevState s{};
    s.N = n;
    s.E = nnz;
    s.G = 1;
    s.weight_kind = weights ? W_F32 : W_UNIT;
    s.off = offsets;
    s.off_end = offsets + 1;
    s.idx = indices;
    s.w = weights;

    cudaError_t e = cudaMemsetAsync(Sigma, 0, (size_t)n * sizeof(double), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(acc, 0, sizeof(ModAccum), st);
    if (e == cudaSuccess) e = launch_modularity(s, 0, n, labels, Sigma, acc, st, sms);
    ModAccum a{};
    if (e == cudaSuccess) e = cudaMemcpyAsync(&a, acc, sizeof(a), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_err(e);
    if (a.bad_label) return err(LPA_ERR_INVALID_ARG, "labels outside [0, n)");
    *q_out = a.two_m > 0.0 ? a.sigma / a.two_m - a.null_sum / (a.two_m * a.two_m) : 0.0;
    return LPA_OK;
}
