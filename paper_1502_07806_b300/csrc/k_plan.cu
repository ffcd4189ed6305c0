// Input validation, Gershgorin interval, and the partition plan (Section II, Fig. 1).
//
// validate_gersh: one warp per row of A (HBM-bound, coalesced row reads). Per row i it records
//   lo_i = A_ii - sum_{j!=i} |A_ij| and hi_i = A_ii + sum_{j!=i} |A_ij|, and flags NaN/Inf in A or
//   prev_eigvals and a descending prev_eigvals.
// plan: one CTA. Reduces the Gershgorin interval, lays out the slices (sizes floor(N/P), first
//   N mod P one larger, or caller sizes), snaps interior boundaries out of near-degenerate
//   clusters of prev_eigvals, and derives each slice's window [s, s+M) with M = min(N, m + 2 halo)
//   and s = clamp(k0 - halo, 0, N - M). It also stores, per 64-row tile of eigen-indices, the
//   column range covered by the windows of the slices in that tile: the first product of Eq. 11
//   only needs those columns because the start vectors are zero outside their windows.
#include "pfsm_internal.cuh"

namespace pfsm {

__global__ void k_validate_gersh(const double *__restrict__ A, const double *__restrict__ prev,
                                 int64_t N, double *__restrict__ gersh, int32_t *status)
{
    const int lane = threadIdx.x & 31;
    const int64_t row = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (row >= N) return;
    const double *a = A + row * N;
    double r = 0.0;
    bool bad = false;
    for (int64_t j = lane; j < N; j += 32) {
        double v = a[j];
        bad |= !isfinite(v);
        r += (j == row) ? 0.0 : fabs(v);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        r += __shfl_xor_sync(0xffffffffu, r, o);
        bad |= (bool)__shfl_xor_sync(0xffffffffu, (int)bad, o);
    }
    if (lane == 0) {
        double d = a[row];
        gersh[2 * row] = d - r;
        gersh[2 * row + 1] = d + r;
        double p = prev[row];
        if (bad || !isfinite(p)) set_status(status, PFSM_ERR_NAN_INPUT);
        else if (row > 0 && p < prev[row - 1]) set_status(status, PFSM_ERR_INVALID_ARG);
    }
}

__global__ void k_plan(const double *__restrict__ prev, int64_t N, int32_t nb, int32_t halo,
                       double cluster_tol, const int32_t *__restrict__ slice_sizes,
                       int32_t *plan, int32_t *tile_krange, double *gersh)
{
    int32_t *k0 = plan, *m = plan + nb, *s = plan + 2 * nb, *M = plan + 3 * nb;
    __shared__ double red_lo[32], red_hi[32];
    const int tid = threadIdx.x, nthr = blockDim.x;

    // Gershgorin interval of A
    double lo = INFINITY, hi = -INFINITY;
    for (int64_t i = tid; i < N; i += nthr) {
        lo = fmin(lo, gersh[2 * i]);
        hi = fmax(hi, gersh[2 * i + 1]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    if ((tid & 31) == 0) { red_lo[tid >> 5] = lo; red_hi[tid >> 5] = hi; }
    __syncthreads();
    if (tid == 0) {
        for (int w = 1; w < (nthr + 31) / 32; w++) { lo = fmin(lo, red_lo[w]); hi = fmax(hi, red_hi[w]); }
        gersh[2 * N] = lo;
        gersh[2 * N + 1] = hi;
        // nominal layout (serial prefix; nb is at most N)
        int32_t start = 0;
        for (int32_t b = 0; b < nb; b++) {
            int32_t sz = slice_sizes ? slice_sizes[b]
                                     : (int32_t)(N / nb) + (b < (int32_t)(N % nb) ? 1 : 0);
            k0[b] = start;
            m[b] = sz;       // nominal size for now
            start += sz;
        }
    }
    __syncthreads();
    // cluster snap of interior boundaries, each decided from the nominal layout alone
    for (int32_t b = tid; b < nb; b += nthr) {
        int32_t k = k0[b];
        if (b > 0 && prev[k] - prev[k - 1] < cluster_tol) {
            int32_t reach = min(m[b - 1], m[b]) / 4;
            for (int32_t d = 1; d <= reach; d++) {
                int32_t dn = k - d, up = k + d;
                if (dn >= 1 && prev[dn] - prev[dn - 1] >= cluster_tol) { k = dn; break; }
                if (up <= N - 1 && prev[up] - prev[up - 1] >= cluster_tol) { k = up; break; }
            }
        }
        s[b] = k;            // snapped start, staged in s
    }
    __syncthreads();
    for (int32_t b = tid; b < nb; b += nthr) k0[b] = s[b];
    __syncthreads();
    for (int32_t b = tid; b < nb; b += nthr) {
        int32_t end = (b + 1 < nb) ? k0[b + 1] : (int32_t)N;
        int32_t mb = end - k0[b];
        int64_t width = (int64_t)mb + 2 * (int64_t)halo;
        int32_t Mb = (int32_t)(width < N ? width : N);
        int64_t lo_s = (int64_t)k0[b] - halo;
        if (lo_s < 0) lo_s = 0;
        if (lo_s > N - Mb) lo_s = N - Mb;
        m[b] = mb;
        M[b] = Mb;
        s[b] = (int32_t)lo_s;
    }
    __syncthreads();
    // per row tile: union of the windows of the slices that own its rows
    const int64_t ntiles = (N + kFsTileRows - 1) / kFsTileRows;
    for (int64_t t = tid; t < ntiles; t += nthr) {
        int32_t r0 = (int32_t)(t * kFsTileRows);
        int64_t tend = (t + 1) * kFsTileRows;
        int32_t r1 = (int32_t)(tend < N ? tend : N) - 1;
        // largest b with k0[b] <= r0, and with k0[b] <= r1
        int32_t lo_b = 0, hi_b = nb - 1;
        while (lo_b < hi_b) { int32_t mid = (lo_b + hi_b + 1) / 2; if (k0[mid] <= r0) lo_b = mid; else hi_b = mid - 1; }
        int32_t bfirst = lo_b;
        lo_b = bfirst; hi_b = nb - 1;
        while (lo_b < hi_b) { int32_t mid = (lo_b + hi_b + 1) / 2; if (k0[mid] <= r1) lo_b = mid; else hi_b = mid - 1; }
        int32_t blast = lo_b;
        int32_t kb = (int32_t)N, ke = 0;
        for (int32_t b = bfirst; b <= blast; b++) {
            kb = min(kb, s[b]);
            ke = max(ke, s[b] + M[b]);
        }
        tile_krange[2 * t] = kb;
        tile_krange[2 * t + 1] = ke;
    }
}

cudaError_t launch_validate_gersh(const double *A, const double *prev, int64_t N, double *gersh,
                                  int32_t *status, cudaStream_t st)
{
    const int warps = 8;
    dim3 grid((unsigned)((N + warps - 1) / warps));
    k_validate_gersh<<<grid, warps * 32, 0, st>>>(A, prev, N, gersh, status); g_launches++;
    return cudaGetLastError();
}

cudaError_t launch_plan(const double *prev, int64_t N, int32_t nb, int32_t halo, double cluster_tol,
                        const int32_t *slice_sizes_dev, int32_t *plan, int32_t *tile_krange,
                        double *gersh, int32_t *status, cudaStream_t st)
{
    (void)status;
    k_plan<<<1, 1024, 0, st>>>(prev, N, nb, halo, cluster_tol, slice_sizes_dev, plan, tile_krange, gersh); g_launches++;
    return cudaGetLastError();
}

}  // namespace pfsm
