// The conventional path around the method (Section II): the paper diagonalizes conventionally
// for the first SCF steps and needs A diagonally dominant for the method to hold.
//
// k_guard measures the diagonal dominance of A as g = max_i ||A_{i,:} without A_ii||_2 /
// (max_i A_ii - min_i A_ii) (the paper gives no formula; the largest l2 coupling of a basis state
// relative to the spread of the diagonal is the reading used, l2 because couplings of random
// sign add like that in the second-order shifts). run_full_diag diagonalizes A completely with
// cuSOLVER's divide-and-conquer syevd (the counterpart of the paper's LAPACK/MAGMA step), signs
// each vector by the start-vector rule with the whole matrix as its window, and leaves the vectors
// as the rows of X, from where the method's own Rayleigh/output phase takes over.
#include <cusolverDn.h>

#include <algorithm>
#include <cmath>
#include <cstring>

#include "pfsm_internal.cuh"

namespace pfsm {

namespace {

// order-preserving map of a double onto an unsigned 64-bit key (for atomic min/max)
__device__ __forceinline__ unsigned long long okey(double x)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}

// out[0] = max_i sqrt(sum_{j != i} A_ij^2) (bits of a non-negative double), out[1] / out[2] =
// keys of max / min A_ii (out zeroed / max-initialised by the caller). One warp per row.
__global__ void k_guard(const double *__restrict__ A, int64_t N, unsigned long long *__restrict__ out)
{
    const int64_t r = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (r >= N) return;
    const double *row = A + r * N;
    double s = 0.0;
    for (int64_t j = lane; j < N; j += 32)
        if (j != r) s = fma(row[j], row[j], s);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) {
        atomicMax(&out[0], (unsigned long long)__double_as_longlong(sqrt(s)));
        const unsigned long long k = okey(row[r]);
        atomicMax(&out[1], k);
        atomicMin(&out[2], k);
    }
}

// Sign rule on the rows of X (row k = vector k): positive home component k when |X_kk| >= 0.1,
// else positive largest component (first index among equals). One warp per row.
__global__ void k_sign_rows(double *__restrict__ X, int64_t N)
{
    const int64_t k = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (k >= N) return;
    double *row = X + k * N;
    double best = -1.0;
    int64_t arg = N;
    for (int64_t i = lane; i < N; i += 32) {
        const double a = fabs(row[i]);
        if (a > best) { best = a; arg = i; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int64_t oa = __shfl_xor_sync(0xffffffffu, arg, o);
        if (ob > best || (ob == best && oa < arg)) { best = ob; arg = oa; }
    }
    const double yh = row[k];
    const double ref = (fabs(yh) >= 0.1) ? yh : row[arg];
    if (ref < 0.0)
        for (int64_t i = lane; i < N; i += 32) row[i] = -row[i];
}

__global__ void k_info_to_status(const int *__restrict__ info, int32_t *__restrict__ status)
{
    if (*info != 0 && *status == 0) *status = PFSM_ERR_NOT_CONVERGED;
}

}  // namespace

cudaError_t fallback_init(pfsm_handle_s *h)
{
    cusolverDnHandle_t cs = nullptr;
    if (cusolverDnCreate(&cs) != CUSOLVER_STATUS_SUCCESS) return cudaErrorInitializationError;
    h->cusolver = cs;
    int lwork = 0;
    const int n = (int)h->N;
    if (cusolverDnDsyevd_bufferSize(cs, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, n, h->ws.X, n, h->ws.eps,
                                    &lwork) != CUSOLVER_STATUS_SUCCESS)
        return cudaErrorInvalidValue;
    h->syevd_lwork = lwork;
    cudaError_t e;
    if ((e = cudaMalloc((void **)&h->syevd_work, (size_t)std::max(lwork, 1) * sizeof(double))) != cudaSuccess) return e;
    if ((e = cudaMalloc((void **)&h->syevd_info, sizeof(int))) != cudaSuccess) return e;
    return cudaMalloc((void **)&h->guard_buf, 3 * sizeof(unsigned long long));
}

void fallback_free(pfsm_handle_s *h)
{
    if (h->cusolver) cusolverDnDestroy((cusolverDnHandle_t)h->cusolver);
    if (h->syevd_work) cudaFree(h->syevd_work);
    if (h->syevd_info) cudaFree(h->syevd_info);
    if (h->guard_buf) cudaFree(h->guard_buf);
    h->cusolver = nullptr;
    h->syevd_work = nullptr;
    h->syevd_info = nullptr;
    h->guard_buf = nullptr;
}

cudaError_t measure_guard(pfsm_handle_s *h, const double *A, cudaStream_t st, double &g)
{
    const int64_t N = h->N;
    unsigned long long init[3] = {0ull, 0ull, ~0ull};
    unsigned long long res[3];
    cudaError_t e;
    if ((e = cudaMemcpyAsync(h->guard_buf, init, sizeof(init), cudaMemcpyHostToDevice, st)) != cudaSuccess) return e;
    k_guard<<<(unsigned)((N + 7) / 8), 256, 0, st>>>(A, N, h->guard_buf); g_launches++;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = cudaMemcpyAsync(res, h->guard_buf, sizeof(res), cudaMemcpyDeviceToHost, st)) != cudaSuccess) return e;
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
    auto unkey = [](unsigned long long k) {
        const unsigned long long b = (k >> 63) ? (k & 0x7FFFFFFFFFFFFFFFull) : ~k;
        double d;
        std::memcpy(&d, &b, sizeof(d));
        return d;
    };
    double cmax;
    std::memcpy(&cmax, &res[0], sizeof(cmax));
    const double spread = unkey(res[1]) - unkey(res[2]);
    g = (spread > 0.0) ? cmax / spread : ((cmax > 0.0) ? INFINITY : 0.0);
    return cudaSuccess;
}

cudaError_t run_full_diag(pfsm_handle_s *h, const double *A, cudaStream_t st)
{
    Workspace &w = h->ws;
    const int64_t N = h->N;
    const int n = (int)N;
    cusolverDnHandle_t cs = (cusolverDnHandle_t)h->cusolver;
    cudaError_t e;
    if ((e = cudaMemcpyAsync(w.X, A, (size_t)N * N * sizeof(double), cudaMemcpyDeviceToDevice, st)) != cudaSuccess)
        return e;
    if (cusolverDnSetStream(cs, st) != CUSOLVER_STATUS_SUCCESS) return cudaErrorInvalidValue;
    // A symmetric: row-major A is its own column-major copy; the eigenvectors come back as the
    // columns of a column-major matrix, i.e. as the rows of w.X (the method's vector layout)
    if (cusolverDnDsyevd(cs, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, n, w.X, n, w.eps, h->syevd_work,
                         h->syevd_lwork, h->syevd_info) != CUSOLVER_STATUS_SUCCESS)
        return cudaErrorLaunchFailure;
    g_launches++;
    k_info_to_status<<<1, 1, 0, st>>>(h->syevd_info, w.status); g_launches++;
    k_sign_rows<<<(unsigned)((N + 7) / 8), 256, 0, st>>>(w.X, N); g_launches++;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    return cudaMemcpyAsync(w.Xfs, w.X, (size_t)N * N * sizeof(double), cudaMemcpyDeviceToDevice, st);
}

}  // namespace pfsm
