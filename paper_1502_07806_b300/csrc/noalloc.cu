// Folded-spectrum iterations on caller vectors with no device allocation at call time.
//
// Some callers cannot allocate device memory when they call into the library: a code that
// reserves all device memory up front for its own pool, or a latency-critical loop in which the
// device-wide synchronisation of cudaMalloc/cudaFree would stall work on other streams. For them
// this file offers one entry point whose only scratch buffer -- the intermediate
// Y = (A - eps I) X between the two products of each iteration -- lives in a fixed, file-scope
// device array instead of handle workspace (kNoAllocMaxElems doubles, 8 MiB). The array belongs
// to this file's module, which CUDA loads into a context lazily, at the first lookup of the
// array's address: from the first call on a device (in a given context) until the process exits
// (or that context is destroyed), that device holds the array.
#include <mutex>

#include <cuda.h>

#include "pfsm_internal.cuh"

namespace {

constexpr int64_t kNoAllocMaxElems = int64_t(1) << 20;   // count * N doubles (8 MiB)
constexpr int kMaxDevices = 64;

// The scratch array. In host code this name is only a host-side stand-in for the symbol; the
// device address has to be looked up with cudaGetSymbolAddress on each device.
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocMaxElems];

std::mutex g_setup_mutex;

// Per device: the context the address was looked up in (by its process-unique ID, so a context
// created after cudaDeviceReset, or a caller's own driver-API context, is never mistaken for the
// earlier one) and the array's device address in that context.
struct ScratchEntry {
    unsigned long long ctx_id;
    double *addr;
};
ScratchEntry g_scratch[kMaxDevices] = {};

// cuCtxGetCurrent and cuCtxGetId through the runtime's driver entry points, so that the library
// keeps no link-time dependency on the driver library (it loads on machines without a GPU)
typedef CUresult (*CtxGetCurrentFn)(CUcontext *);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long *);

cudaError_t current_context_id(unsigned long long *id)
{
    static CtxGetCurrentFn get_current = nullptr;
    static CtxGetIdFn get_id = nullptr;
    if (!get_current || !get_id) {
        void *p1 = nullptr, *p2 = nullptr;
        cudaDriverEntryPointQueryResult q1, q2;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p1, 12000, cudaEnableDefault, &q1) != cudaSuccess ||
            q1 != cudaDriverEntryPointSuccess ||
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &p2, 12000, cudaEnableDefault, &q2) != cudaSuccess ||
            q2 != cudaDriverEntryPointSuccess)
            return cudaErrorInitializationError;
        get_current = (CtxGetCurrentFn)p1;
        get_id = (CtxGetIdFn)p2;
    }
    CUcontext ctx = nullptr;
    if (get_current(&ctx) != CUDA_SUCCESS) return cudaErrorInitializationError;
    if (!ctx) {
        *id = 0;
        return cudaSuccess;
    }
    return get_id(ctx, id) == CUDA_SUCCESS ? cudaSuccess : cudaErrorInitializationError;
}

// The device address of the scratch array in the current device's current context, looked up
// with that device current the first time a context is seen and cached for later calls. The
// lookup loads this module into the context (allocating the array) if it is not loaded yet.
cudaError_t scratch_for_current_device(double **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    unsigned long long id = 0;
    if ((e = current_context_id(&id)) != cudaSuccess) return e;
    if (id != 0 && g_scratch[dev].addr && g_scratch[dev].ctx_id == id) {
        *out = g_scratch[dev].addr;
        return cudaSuccess;
    }
    double *p = nullptr;
    e = cudaGetSymbolAddress((void **)&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    // the lookup makes the runtime's primary context current if no context was
    if ((e = current_context_id(&id)) != cudaSuccess) return e;
    g_scratch[dev] = {id, p};
    *out = p;
    return cudaSuccess;
}

}  // namespace

extern "C" int pfsm_fs_iterate_noalloc(int64_t N, int64_t count, const double *A, double *X,
                                       const double *eps, const double *alpha, int32_t iters,
                                       void *stream)
{
    if (N < 1 || count < 1 || iters < 0 || !A || !X || !eps || !alpha) return PFSM_ERR_INVALID_ARG;
    if (count > kNoAllocMaxElems / N) return PFSM_ERR_INVALID_ARG;   // count * N over the cap
    double *Y = nullptr;
    if (scratch_for_current_device(&Y) != cudaSuccess) return PFSM_ERR_CUDA;
    cudaStream_t st = (cudaStream_t)stream;
    // Y needs no clearing: the first product of every iteration writes all count x N entries
    // before the second product reads any of them.
    for (int32_t it = 0; it < iters; it++) {
        pfsm::GemmArgs g{};
        g.rows = count; g.cols = N; g.K = N;
        g.P = X; g.ldp = N; g.Q = A; g.ldq = N; g.C = Y; g.ldc = N;
        g.aux_x = X; g.eps = eps;
        if (pfsm::launch_gemm_f64(g, pfsm::EPI_FS1, pfsm::Q_KMAJOR, st) != cudaSuccess) return PFSM_ERR_CUDA;
        pfsm::GemmArgs u{};
        u.rows = count; u.cols = N; u.K = N;
        u.P = Y; u.ldp = N; u.Q = A; u.ldq = N; u.C = X; u.ldc = N;
        u.aux_y = Y; u.eps = eps; u.alpha = alpha;
        if (pfsm::launch_gemm_f64(u, pfsm::EPI_FS2, pfsm::Q_KMAJOR, st) != cudaSuccess) return PFSM_ERR_CUDA;
    }
    return PFSM_OK;
}
