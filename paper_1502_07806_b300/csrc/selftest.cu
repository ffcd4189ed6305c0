// Test entry points for the hand-written FP64 helpers that stand in for CUDA's own division, square
// root and integer -> FP64 conversion on the serial paths (fp64_util.cuh): they evaluate the helpers
// on caller-given inputs so that the tests can hold them to CUDA's correctly rounded results.
#include <cstdint>

#include "fp64_util.cuh"
#include "pfsm.h"

namespace pfsm {
namespace {

__global__ void k_selftest_fp64(const double *__restrict__ x, int64_t n, double *__restrict__ rcp_scaled,
                                double *__restrict__ rsqrt_scaled, double *__restrict__ rcp_fast,
                                double *__restrict__ rsqrt_fast)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double v = x[i];
    rcp_scaled[i] = (v > 0.0) ? scaled_rcp(v) : 0.0;          // defined for positive arguments
    rsqrt_scaled[i] = (v > 0.0) ? scaled_rsqrt(v) : 0.0;
    rcp_fast[i] = fast_rcp(v);
    rsqrt_fast[i] = (v > 0.0) ? fast_rsqrt(v) : 0.0;
}

__global__ void k_selftest_i64(const long long *__restrict__ t, const int32_t *__restrict__ e, int64_t n,
                               double *__restrict__ out)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = oz_i64_to_f64_scaled(t[i], e[i]);
}

}  // namespace
}  // namespace pfsm

extern "C" int pfsm_selftest_fp64_helpers(const double *x, int64_t n, double *rcp_scaled, double *rsqrt_scaled,
                                          double *rcp_fast, double *rsqrt_fast, void *stream)
{
    if (n < 0 || (n > 0 && (!x || !rcp_scaled || !rsqrt_scaled || !rcp_fast || !rsqrt_fast)))
        return PFSM_ERR_INVALID_ARG;
    if (n == 0) return PFSM_OK;
    pfsm::k_selftest_fp64<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(x, n, rcp_scaled,
                                                                                         rsqrt_scaled, rcp_fast,
                                                                                         rsqrt_fast);
    return cudaGetLastError() == cudaSuccess ? PFSM_OK : PFSM_ERR_CUDA;
}

extern "C" int pfsm_selftest_i64_to_f64(const int64_t *t, const int32_t *e, int64_t n, double *out, void *stream)
{
    if (n < 0 || (n > 0 && (!t || !e || !out))) return PFSM_ERR_INVALID_ARG;
    if (n == 0) return PFSM_OK;
    pfsm::k_selftest_i64<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(
        reinterpret_cast<const long long *>(t), e, n, out);
    return cudaGetLastError() == cudaSuccess ? PFSM_OK : PFSM_ERR_CUDA;
}
