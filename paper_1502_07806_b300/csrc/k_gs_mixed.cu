// Gram-Schmidt of the mixed forms (Section II, after the Eq. 11 iterations): the result of
// Gram-Schmidt in ascending index order, V = L^-1 X with S = X X^T = L L^T, computed without an
// FP64 Cholesky factorisation.
//
// B300 runs FP64 at 2 FMA/clk per SM, so the sequential chain of a blocked FP64 Cholesky (one
// diagonal block at a time, each on one SM) and its triangular solve are slow, while FP32 and the
// tensor cores are fast. The steps below move all sequential work to FP32 and all FP64-accurate
// work to dense products on the tensor cores:
//
//   1. S~ = X X^T to about 2^-35 (digit product truncated to five levels).
//   2. A lower-triangular M with positive diagonal and M S M^T close to I. M is a preconditioner
//      only: nothing below needs it to be accurate. Two forms:
//      a. the second-order series of L^-1 for S~ = I + E: with G = Phi(E) the first
//         order of chol(I + E) = I + G_exact, G_exact = Phi(E - G_exact G_exact^T), so
//         L^-1 = I - G + G^2 + Phi(G G^T) + O(E^3), and since G + G^T = E,
//         G^2 + Phi(G G^T) = Phi(G E) + diag(G_ii^2) / 2: M = I - G + Phi(G E) + diag(G_ii^2) / 2,
//         one split product. The vectors entering Gram-Schmidt are nearly orthonormal (window
//         eigenvectors after Eq. 11; |E| ~ 1e-2), so M S M^T - I is O(|E|^3) ~ 1e-7, what the FP32
//         factorisation below reaches. An eager solve measures it after step 4 (one 8-byte
//         read-back); above kSeriesMaxResidual the FP32 factorisation of V1 V1^T follows and V1 is
//         preconditioned again. A solve captured into a CUDA graph cannot read back: it relies on
//         the checks of step 5, which report a residual too large for the fixed point.
//      b. FP32 blocked Cholesky S~ = L~ L~^T and, in the same sweep, M = L~^-1 (the fallback of a).
//   3. V1 = M X with the FP64-accurate digit product. For ANY lower-triangular M with positive
//      diagonal, chol(M S M^T) = M L, so Gram-Schmidt of V1 equals Gram-Schmidt of X.
//   4. E = V1 V1^T - I (digit product). |E| is of the order of cond(S) times the FP32 unit.
//   5. chol(I + E) = I + F: with F lower triangular, F + F^T + F F^T = E, i.e. the fixed point
//      F = Phi(E - F F^T), Phi taking the strict lower triangle and half the diagonal. Each sweep
//      multiplies the error by about 2|E|; F F^T is O(|E|^2) and only needs FP32 accuracy.
//   6. V = (I + F)^-1 V1 = V1 - F W with W = V1 - F V1, exact up to O(|F|^3): W only needs about
//      1e-9 relative accuracy (split product), F W is the FP64-accurate digit product.
// A non-positive FP32 pivot (or one below 1e-8 of the vector's squared norm), |E| >= 1/4 (no
// contraction) or a last sweep that still moves F by more than 1e-13 reports PFSM_ERR_NOT_SPD:
// the overlap matrix is then too ill-conditioned for this scheme (the FP64 form handles it).
#include <cfloat>
#include <cstring>

#include "pfsm_internal.cuh"

namespace pfsm {

namespace {

constexpr int GB = 64;                  // FP32 Cholesky block
constexpr int LDT = GB + 4;             // shared-memory row: 16-byte aligned for float4 reads
constexpr int kFixedPointSweeps = 2;    // sweeps after F0 = Phi(E): error ~ (2|E|)^3 |E|
constexpr size_t kStepSmem = 2 * GB * LDT * sizeof(float) + 6 * GB * sizeof(float);
// largest max|V1 V1^T - I| after the series preconditioner handed to the fixed point of step 5:
// emulated with exact products on perturbed N = 256 vectors, its second sweep still moved F by
// 6e-17 at 1.3e-6 and 4e-14 at 1.2e-5 (the check below is 1e-13), and by 2e-11 at 8e-5
constexpr double kSeriesMaxResidual = 4e-6;

__device__ __forceinline__ float4 ld4(const float *p) { return *reinterpret_cast<const float4 *>(p); }
__device__ __forceinline__ float el(const float4 &v, int i) { return i == 0 ? v.x : i == 1 ? v.y : i == 2 ? v.z : v.w; }

// acc[a][c] += sum_k P[k][4 ty + a] Q[k][4 tx + c] over k < kn (row-major shared tiles, row LDT)
__device__ __forceinline__ void tile_mma(const float (*P)[LDT], const float (*Q)[LDT], int kn, int tx, int ty,
                                         float acc[4][4])
{
#pragma unroll 4
    for (int k = 0; k < kn; k++) {
        const float4 p = ld4(&P[k][4 * ty]), q = ld4(&Q[k][4 * tx]);
#pragma unroll
        for (int a = 0; a < 4; a++)
#pragma unroll
            for (int c = 0; c < 4; c++) acc[a][c] = fmaf(el(p, a), el(q, c), acc[a][c]);
    }
}

// T[k][r] = src[(r0 + r) * N + k0 + k] for r < nr, k < nk (zero elsewhere): 64 x 64 tile stored
// transposed; the 16 loads of a thread are issued before its stores.
__device__ __forceinline__ void load_tile_t(float (*T)[LDT], const float *__restrict__ src, int64_t N,
                                            int64_t r0, int nr, int64_t k0, int nk)
{
    float v[16];
#pragma unroll
    for (int i = 0; i < 16; i++) {
        const int t = threadIdx.x + 256 * i, r = t >> 6, k = t & 63;
        v[i] = (r < nr && k < nk) ? src[(r0 + r) * N + k0 + k] : 0.0f;
    }
#pragma unroll
    for (int i = 0; i < 16; i++) {
        const int t = threadIdx.x + 256 * i;
        T[t & 63][t >> 6] = v[i];
    }
}

// T[k][q] = src[(k0 + k) * N + c0 + q] for k < nk, q < nq (zero elsewhere), not transposed.
__device__ __forceinline__ void load_tile(float (*T)[LDT], const float *__restrict__ src, int64_t N,
                                          int64_t k0, int nk, int64_t c0, int nq)
{
    float v[16];
#pragma unroll
    for (int i = 0; i < 16; i++) {
        const int t = threadIdx.x + 256 * i, k = t >> 6, q = t & 63;
        v[i] = (k < nk && q < nq) ? src[(k0 + k) * N + c0 + q] : 0.0f;
    }
#pragma unroll
    for (int i = 0; i < 16; i++) {
        const int t = threadIdx.x + 256 * i;
        T[t >> 6][t & 63] = v[i];
    }
}

}  // namespace

// S (FP64, lower triangle) -> FP32 working matrix.
__global__ void k_lower_to_f32(const double *__restrict__ S, float *__restrict__ L, int64_t N)
{
    const int64_t r = blockIdx.y;
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c <= r; c += (int64_t)gridDim.x * blockDim.x)
        L[r * N + c] = (float)S[r * N + c];
}

// Cholesky factor inverse of the b x b diagonal block at (jb, jb) of L, in FP32 (every CTA of the
// step does this redundantly: it costs a few microseconds and saves a launch). On exit
// DiT[c][i] = (L_jj^-1)[i][c] (transposed; zero above the diagonal, identity-padded to 64 x 64).
// Right-looking LDL^T elimination, S = U diag(d) U^T with U unit lower: step k subtracts
// u_k a_k^T from the trailing matrix (a_k its column k, u_k = a_k / d_k) and applies the same row
// operation to X = U^-1 (X starts at I: X_i -= u_ik X_k for i > k). At the end
// L^-1 = diag(d)^-1/2 X. Each of the 256 threads keeps the 4 x 4 block (rows 4 ty + a, columns
// 4 tx + c) of both matrices in registers; column k of A and row k of X are published through
// double-buffered shared memory, so a step costs one barrier.
__device__ void factor_diag_block(const float *__restrict__ L, int64_t N, int64_t jb, int b,
                                  const double *__restrict__ sdiag, int32_t *status,
                                  float (*DiT)[LDT], float (*buf)[GB])
{
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    float A[4][4], X[4][4];
#pragma unroll
    for (int a = 0; a < 4; a++)
#pragma unroll
        for (int c = 0; c < 4; c++) {
            const int i = 4 * ty + a, k = 4 * tx + c;
            A[a][c] = (i < b && k <= i) ? L[(jb + i) * N + jb + k] : (i == k ? 1.0f : 0.0f);
            X[a][c] = (i == k) ? 1.0f : 0.0f;
        }
    float *piv = buf[4], *ref = buf[5];
    if (tid < b) ref[tid] = 1e-8f * (float)sdiag[jb + tid];
    __syncthreads();
    bool bad = false;
    for (int kb = 0; kb < 16; kb++) {
#pragma unroll
        for (int kk = 0; kk < 4; kk++) {               // k = 4 kb + kk: register index kk is static
            const int k = 4 * kb + kk;
            if (k < b) {
                float *col = buf[kk & 1], *row = buf[2 + (kk & 1)];
                if (tx == kb)
                    *reinterpret_cast<float4 *>(&col[4 * ty]) = make_float4(A[0][kk], A[1][kk], A[2][kk], A[3][kk]);
                if (ty == kb)
                    *reinterpret_cast<float4 *>(&row[4 * tx]) = make_float4(X[kk][0], X[kk][1], X[kk][2], X[kk][3]);
                __syncthreads();
                float d = col[k];
                const bool good = d > ref[k] && d < FLT_MAX;   // breakdown or NaN: record, keep the
                bad |= !good;                                  // numbers finite
                d = good ? d : 1.0f;
                if (tid == 0) piv[k] = d;
                const float dinv = __frcp_rn(d);
                const float4 cr = ld4(&col[4 * ty]), cc = ld4(&col[4 * tx]), xr = ld4(&row[4 * tx]);
                float u[4], v[4];
#pragma unroll
                for (int a = 0; a < 4; a++) u[a] = (4 * ty + a > k) ? el(cr, a) * dinv : 0.0f;
#pragma unroll
                for (int c = 0; c < 4; c++) v[c] = (4 * tx + c > k) ? el(cc, c) : 0.0f;
#pragma unroll
                for (int a = 0; a < 4; a++)
#pragma unroll
                    for (int c = 0; c < 4; c++) {
                        A[a][c] = fmaf(-u[a], v[c], A[a][c]);
                        X[a][c] = fmaf(-u[a], el(xr, c), X[a][c]);
                    }
            }
        }
    }
    if (bad && tid == 0) set_status(status, PFSM_ERR_NOT_SPD);
    __syncthreads();
#pragma unroll
    for (int a = 0; a < 4; a++) {
        const int i = 4 * ty + a;
        const float s = i < b ? rsqrtf(piv[i]) : 1.0f;
#pragma unroll
        for (int c = 0; c < 4; c++) DiT[4 * tx + c][i] = (4 * tx + c <= i) ? X[a][c] * s : 0.0f;
    }
    __syncthreads();
}

// Step j of the FP32 blocked Cholesky with the augmented inverse. CTAs [0, npanel): panel rows
// L_rj = S_rj L_jj^-T (64 rows each, in place). CTAs [npanel, npanel + j + 1): row block j of
// M = L^-1, M_jc = L_jj^-1 R_jc, where R_jc = delta_jc I - sum_{k<j} L_jk M_kc has been
// accumulated by the update kernel of the earlier steps (R_jj = I).
__global__ void __launch_bounds__(256)
k_chol32_step(float *__restrict__ L, const float *__restrict__ R, float *__restrict__ M, int64_t N,
              int j, int npanel, const double *__restrict__ sdiag, int32_t *status)
{
    extern __shared__ __align__(16) float g32_sm[];
    float(*DiT)[LDT] = reinterpret_cast<float(*)[LDT]>(g32_sm);
    float(*T)[LDT] = reinterpret_cast<float(*)[LDT]>(g32_sm + GB * LDT);
    float(*buf)[GB] = reinterpret_cast<float(*)[GB]>(g32_sm + 2 * GB * LDT);
    const int64_t jb = (int64_t)j * GB;
    const int b = (int)((N - jb) < GB ? (N - jb) : GB);
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const bool panel = (int)blockIdx.x < npanel;
    const int cblk = (int)blockIdx.x - npanel;         // M CTAs: column block 0 .. j
    const int64_t r0 = jb + b + (int64_t)blockIdx.x * GB;
    const int nr = panel ? (int)((N - r0) < GB ? (N - r0) : GB) : 0;
    // the operand tile does not depend on the factorisation: load it first
    if (panel) load_tile_t(T, L, N, r0, nr, jb, b);                        // T[k][r] = S_rj[r][k]
    else if (cblk < j) load_tile(T, R, N, jb, b, (int64_t)cblk * GB, GB);  // T[k][q] = R_jc[k][q]
    factor_diag_block(L, N, jb, b, sdiag, status, DiT, buf);
    if (!panel && cblk == j) {
        for (int t = tid; t < b * b; t += blockDim.x) {
            const int r = t / b, c = t % b;
            if (c <= r) M[(jb + r) * N + jb + c] = DiT[c][r];
        }
        return;
    }
    float acc[4][4] = {};
    if (panel) {
        tile_mma(T, DiT, b, tx, ty, acc);              // sum_k S_rj[r][k] Di[c][k]
#pragma unroll
        for (int a = 0; a < 4; a++) {
            const int r = 4 * ty + a;
#pragma unroll
            for (int c = 0; c < 4; c++) {
                const int cc = 4 * tx + c;
                if (r < nr && cc < b) L[(r0 + r) * N + jb + cc] = acc[a][c];
            }
        }
    } else {
        tile_mma(DiT, T, b, tx, ty, acc);              // sum_k Di[r][k] R_jc[k][q]
        const int64_t cb0 = (int64_t)cblk * GB;
#pragma unroll
        for (int a = 0; a < 4; a++) {
            const int r = 4 * ty + a;
            if (r < b) {
#pragma unroll
                for (int c = 0; c < 4; c++) M[(jb + r) * N + cb0 + 4 * tx + c] = acc[a][c];
            }
        }
    }
}

// Trailing update of step j: S_rc -= L_rj L_cj^T (lower tiles of the trailing matrix) and
// R_rc -= L_rj M_jc for c <= j (the column block c = j is written, not updated: R starts at 0
// below the diagonal blocks). 64 x 64 tiles, K = b <= 64.
__global__ void __launch_bounds__(256)
k_chol32_update(float *__restrict__ L, float *__restrict__ R, const float *__restrict__ M, int64_t N,
                int j, int nr, int ns_tiles)
{
    __shared__ __align__(16) float Ps[GB][LDT], Qs[GB][LDT];
    const int64_t jb = (int64_t)j * GB;
    const int b = (int)((N - jb) < GB ? (N - jb) : GB);
    const int64_t r0 = jb + b;
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    int rt, ct;
    const bool spart = (int)blockIdx.x < ns_tiles;
    if (spart) {                                        // triangular tile index -> (rt, ct), ct <= rt
        const int t = blockIdx.x;
        rt = (int)((sqrtf(8.0f * t + 1.0f) - 1.0f) * 0.5f);
        while ((rt + 1) * (rt + 2) / 2 <= t) rt++;
        while (rt * (rt + 1) / 2 > t) rt--;
        ct = t - rt * (rt + 1) / 2;
    } else {
        const int t = (int)blockIdx.x - ns_tiles;
        rt = t / (j + 1);
        ct = t % (j + 1);
    }
    const int64_t row0 = r0 + (int64_t)rt * GB;
    const int nrow = (int)((N - row0) < GB ? (N - row0) : GB);
    load_tile_t(Ps, L, N, row0, nrow, jb, b);           // Ps[k][r] = L_rj[r][k]
    int64_t col0;
    int ncol;
    if (spart) {
        col0 = r0 + (int64_t)ct * GB;
        ncol = (int)((N - col0) < GB ? (N - col0) : GB);
        load_tile_t(Qs, L, N, col0, ncol, jb, b);       // Qs[k][q] = L_cj[q][k]
    } else {
        col0 = (int64_t)ct * GB;
        ncol = ct == j ? b : GB;
        load_tile(Qs, M, N, jb, b, col0, ncol);         // Qs[k][q] = M_jc[k][q]
    }
    __syncthreads();
    float acc[4][4] = {};
    tile_mma(Ps, Qs, b, tx, ty, acc);
    const bool first = !spart && ct == j;
    float *C = spart ? L : R;
#pragma unroll
    for (int a = 0; a < 4; a++) {
        const int r = 4 * ty + a;
        if (r >= nrow) continue;
#pragma unroll
        for (int c = 0; c < 4; c++) {
            const int q = 4 * tx + c;
            if (q >= ncol) continue;
            const int64_t gr = row0 + r, gc = col0 + q;
            if (spart && gc > gr) continue;
            const int64_t o = gr * N + gc;
            C[o] = first ? -acc[a][c] : C[o] - acc[a][c];
        }
    }
}

// F = Phi(S2 - I - G): strict lower part, half the diagonal, zero above (G may be null). With
// last set, a change of F by more than 1e-13 in this sweep means the fixed point has not settled
// to FP64 accuracy (the overlap matrix is too ill-conditioned for the FP32 preconditioner).
// check: |S2 - I - G| >= 1/4 (no contraction) reports PFSM_ERR_NOT_SPD. emax (may be null): the
// largest |S2 - I - G| of the lower triangle, as FP64 bits (the integer order of non-negative
// doubles is their order), by one atomicMax per CTA.
__global__ void __launch_bounds__(256)
k_phi(const double *__restrict__ S2, const double *__restrict__ G, double *__restrict__ F, int64_t N, int last,
      int check, unsigned long long *__restrict__ emax, int32_t *status)
{
    // magnitudes compared as bit patterns (a NaN's exceeds every bound): no FP64 compare, one or
    // two FP64 subtractions per entry (B300 retires one FP64 warp instruction per 16 cycles per SM)
    constexpr unsigned long long kQuarter = 0x3FD0000000000000ull, kTiny = 0x3D3C25C268497682ull;   // 0.25, 1e-13
    const int64_t r = blockIdx.y;
    unsigned long long m = 0ull;
    bool bad = false;
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < N; c += (int64_t)gridDim.x * blockDim.x) {
        const int64_t o = r * N + c;
        double v = 0.0;
        if (c <= r) {
            v = (c == r) ? S2[o] - 1.0 : S2[o];
            if (G) v -= G[o];
            const unsigned long long a = (unsigned long long)__double_as_longlong(v) & 0x7FFFFFFFFFFFFFFFull;
            m = max(m, a);
            bad |= check && !(a < kQuarter);               // no contraction (or NaN)
            if (c == r) v *= 0.5;
            if (last) {
                const unsigned long long d = (unsigned long long)__double_as_longlong(v - F[o]) & 0x7FFFFFFFFFFFFFFFull;
                bad |= !(d <= kTiny);
            }
        }
        F[o] = v;
    }
    if (bad) set_status(status, PFSM_ERR_NOT_SPD);
    if (emax) {
        __shared__ unsigned long long wm[8];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
        if ((threadIdx.x & 31) == 0) wm[threadIdx.x >> 5] = m;
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int w = 1; w < (int)(blockDim.x >> 5); w++) m = max(m, wm[w]);
            if (m) atomicMax(emax, m);
        }
    }
}

// Series preconditioner, first part: from the overlap S~ (lower triangle stored; the tiles above
// the diagonal are stale) write E = S~ - I in full (symmetric) and G = Phi(E) (zero above the
// diagonal). 32 x 32 tiles; a tile above the diagonal reads the mirrored tile through shared
// memory, so every global access is row-contiguous.
__global__ void __launch_bounds__(256)
k_series_inputs(const double *__restrict__ S, double *__restrict__ E, double *__restrict__ G, int64_t N)
{
    __shared__ double t[32][33];
    const int bi = blockIdx.y, bj = blockIdx.x;                  // output tile (rows bi, cols bj)
    const int bs = max(bi, bj), bt = min(bi, bj);                // source tile in the lower part
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;      // 32 x 8 threads
    for (int q = ty; q < 32; q += 8) {
        const int64_t r = (int64_t)bs * 32 + q, c = (int64_t)bt * 32 + tx;
        t[q][tx] = (r < N && c < N && c <= r) ? S[r * N + c] : 0.0;
    }
    __syncthreads();
    for (int q = ty; q < 32; q += 8) {
        const int64_t r = (int64_t)bi * 32 + q, c = (int64_t)bj * 32 + tx;
        if (r >= N || c >= N) continue;
        // element (r, c) of the symmetric matrix, from the stored lower triangle
        const double v = (c <= r) ? t[q][tx] : t[tx][q];
        const double e = v - (r == c ? 1.0 : 0.0);
        E[r * N + c] = e;
        G[r * N + c] = (c < r) ? e : (c == r ? 0.5 * e : 0.0);
    }
}

// Series preconditioner, second part, in place over G: M = I - G + Phi(C) + diag(G_ii^2) / 2 with
// C = G E (lower triangle read); zero above the diagonal stays zero.
__global__ void k_series_assemble(double *__restrict__ GM, const double *__restrict__ C, int64_t N)
{
    const int64_t r = blockIdx.y;
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c <= r; c += (int64_t)gridDim.x * blockDim.x) {
        const int64_t o = r * N + c;
        const double g = GM[o];
        GM[o] = (c < r) ? C[o] - g : fma(0.5 * g, g, fma(0.5, C[o], 1.0 - g));
    }
}

cudaError_t configure_gs_mixed_kernels()
{
    return cudaFuncSetAttribute(k_chol32_step, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kStepSmem);
}

// M = L~^-1 of the FP32 Cholesky of w.S (lower triangle), into w.M32 (zero above the diagonal).
static cudaError_t fp32_cholesky_inverse(pfsm_handle_s *h, cudaStream_t st)
{
    Workspace &w = h->ws;
    const int64_t N = h->N;
    {
        const int64_t bx = (N + 255) / 256;
        dim3 grid((unsigned)(bx < 8 ? bx : 8), (unsigned)N);
        k_lower_to_f32<<<grid, 256, 0, st>>>(w.S, w.L32, N); g_launches++;
    }
    const int nblk = (int)((N + GB - 1) / GB);
    for (int j = 0; j < nblk; j++) {
        const int64_t jb = (int64_t)j * GB;
        const int64_t rest = N - jb - (N - jb < GB ? N - jb : GB);
        const int nr = (int)((rest + GB - 1) / GB);
        k_chol32_step<<<nr + j + 1, 256, kStepSmem, st>>>(w.L32, w.R32, w.M32, N, j, nr, w.sdiag, w.status);
        g_launches++;
        if (nr > 0) {
            const int ns_tiles = nr * (nr + 1) / 2;
            k_chol32_update<<<ns_tiles + nr * (j + 1), 256, 0, st>>>(w.L32, w.R32, w.M32, N, j, nr, ns_tiles);
            g_launches++;
        }
    }
    return cudaGetLastError();
}

// M = I - G + Phi(G E) + diag(G_ii^2) / 2 from the overlap in w.S (lower triangle), into w.F
// (zero above the diagonal); w.Z and w.Y are scratch.
static cudaError_t series_preconditioner(pfsm_handle_s *h, cudaStream_t st)
{
    Workspace &w = h->ws;
    const int64_t N = h->N;
    const int64_t ld = padded_ld(N);
    const int ns = slices_for(h->prm.precision), kind = slice_kind(h->prm.precision);
    SliceBuf sG{w.slY, N, ld, ns, kind}, sE{w.slZ, N, ld, ns, kind};
    cudaError_t e;
    const unsigned nt = (unsigned)((N + 31) / 32);
    k_series_inputs<<<dim3(nt, nt), 256, 0, st>>>(w.S, w.Z, w.F, N); g_launches++;
    if ((e = launch_split(w.F, N, N, N, sG, false, nullptr, st)) != cudaSuccess) return e;
    if ((e = launch_split(w.Z, N, N, N, sE, false, nullptr, st)) != cudaSuccess) return e;
    TcParams g{};                                        // C = G E^T = G E (lower triangle) -> Y
    g.rows = (int)N; g.cols = (int)N; g.ldo = N; g.status = w.status;
    g.epi = TC_EPI_STORE; g.out = w.Y; g.lower_only = 1;
    if ((e = launch_gemm_tc(sG, sE, g, nullptr, st)) != cudaSuccess) return e;
    const int64_t bx = (N + 255) / 256;
    k_series_assemble<<<dim3((unsigned)(bx < 8 ? bx : 8), (unsigned)N), 256, 0, st>>>(w.F, w.Y, N); g_launches++;
    return cudaGetLastError();
}

// V1 = M X -> w.Y, the digits of M (rows; FP64 in w.F or FP32 in w.M32) against those of X^T
// (rows = basis index, K = vector index); M is lower triangular.
static cudaError_t precondition(pfsm_handle_s *h, const double *M64, const double *X, double *out, cudaStream_t st)
{
    Workspace &w = h->ws;
    const int64_t N = h->N;
    const int64_t ld = padded_ld(N);
    SliceBuf dP{w.ozP, N, ld, OZ_SLICES, 0}, dQ{w.ozQ, N, ld, OZ_SLICES, 0};
    cudaError_t e;
    if ((e = launch_transpose(X, w.W, N, st)) != cudaSuccess) return e;
    if (M64) e = launch_oz_split(M64, N, N, N, dP, w.ozeP, st);
    else e = launch_oz_split_f32(w.M32, N, N, N, dP, w.ozeP, st);
    if (e != cudaSuccess) return e;
    if ((e = launch_oz_split(w.W, N, N, N, dQ, w.ozeQ, st)) != cudaSuccess) return e;
    OzParams o{};
    o.rows = (int)N; o.cols = (int)N; o.C = out; o.ldc = N; o.p_lower = 1; o.status = w.status;
    return launch_gemm_oz(dP, w.ozeP, dQ, w.ozeQ, o, st);
}

// S2 = V1 V1^T (lower, all digit levels) -> w.S
static cudaError_t overlap_full(pfsm_handle_s *h, const double *V1, cudaStream_t st)
{
    Workspace &w = h->ws;
    const int64_t N = h->N;
    const int64_t ld = padded_ld(N);
    SliceBuf dP{w.ozP, N, ld, OZ_SLICES, 0};
    cudaError_t e;
    if ((e = launch_oz_split(V1, N, N, N, dP, w.ozeP, st)) != cudaSuccess) return e;
    OzParams o{};
    o.rows = (int)N; o.cols = (int)N; o.C = w.S; o.ldc = N; o.lower_only = 1; o.status = w.status;
    return launch_gemm_oz(dP, w.ozeP, dP, w.ozeP, o, st);
}

cudaError_t launch_gram_schmidt_mixed(pfsm_handle_s *h, cudaStream_t st)
{
    Workspace &w = h->ws;
    const int64_t N = h->N;
    const int64_t ld = padded_ld(N);
    const int ns = slices_for(h->prm.precision), kind = slice_kind(h->prm.precision);
    SliceBuf sY{w.slY, N, ld, ns, kind}, sZ{w.slZ, N, ld, ns, kind};
    SliceBuf dP{w.ozP, N, ld, OZ_SLICES, 0}, dQ{w.ozQ, N, ld, OZ_SLICES, 0};
    cudaError_t e;
    // 1. S~ = X X^T (lower) to about 2^-35 (five digit levels: a split product accumulated in FP32
    //    would carry sqrt(N) 2^-24, which at large N makes E, and with it F, too large for the
    //    split products of steps 5-6), and its diagonal for the breakdown test
    OzParams o{};
    if ((e = launch_oz_split(w.X, N, N, N, dP, w.ozeP, st)) != cudaSuccess) return e;
    o.rows = (int)N; o.cols = (int)N; o.C = w.S; o.ldc = N; o.lower_only = 1; o.levels = 5; o.status = w.status;
    if ((e = launch_gemm_oz(dP, w.ozeP, dP, w.ozeP, o, st)) != cudaSuccess) return e;
    if ((e = launch_copy_diag(w.S, N, w.sdiag, st)) != cudaSuccess) return e;
    if (h->timing && (e = cudaEventRecord(h->gs_ev[0], st)) != cudaSuccess) return e;
    // 2.-3. the series preconditioner M and V1 = M X -> Y
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if ((e = cudaStreamIsCapturing(st, &cap)) != cudaSuccess) return e;
    const bool readback = cap == cudaStreamCaptureStatusNone && h->fs_rmax;
    h->gs_precond = 2;
    h->gs_precond_resid = 0.0;
    if ((e = series_preconditioner(h, st)) != cudaSuccess) return e;
    if (h->timing && (e = cudaEventRecord(h->gs_ev[1], st)) != cudaSuccess) return e;
    if ((e = precondition(h, w.F, w.X, w.Y, st)) != cudaSuccess) return e;
    // 4. S2 = V1 V1^T (lower) -> S
    if ((e = overlap_full(h, w.Y, st)) != cudaSuccess) return e;
    // 5. F = Phi(E - F F^T), E = S2 - I
    const int64_t bx = (N + 255) / 256;
    const dim3 egrid((unsigned)(bx < 8 ? bx : 8), (unsigned)N);
    if (readback) {
        // measure max|E| (one read-back); too large for the fixed point: FP32 factorisation of S2,
        // V1 <- M' V1 (still Gram-Schmidt of X), S2 again
        if ((e = cudaMemsetAsync(h->fs_rmax, 0, sizeof(unsigned long long), st)) != cudaSuccess) return e;
        k_phi<<<egrid, 256, 0, st>>>(w.S, nullptr, w.F, N, 0, 0, h->fs_rmax, w.status); g_launches++;
        unsigned long long eb = 0ull;
        if ((e = cudaMemcpyAsync(&eb, h->fs_rmax, sizeof(eb), cudaMemcpyDeviceToHost, st)) != cudaSuccess) return e;
        if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
        double emax;
        std::memcpy(&emax, &eb, sizeof(emax));
        h->gs_precond_resid = emax;
        if (!(emax <= kSeriesMaxResidual)) {
            h->gs_precond = 3;
            if ((e = launch_copy_diag(w.S, N, w.sdiag, st)) != cudaSuccess) return e;
            if ((e = fp32_cholesky_inverse(h, st)) != cudaSuccess) return e;
            if ((e = precondition(h, nullptr, w.Y, w.X, st)) != cudaSuccess) return e;
            double *tmp = w.X;                           // V1 in Y, X free again
            w.X = w.Y;
            w.Y = tmp;
            if ((e = overlap_full(h, w.Y, st)) != cudaSuccess) return e;
            k_phi<<<egrid, 256, 0, st>>>(w.S, nullptr, w.F, N, 0, 1, nullptr, w.status); g_launches++;
        }
    } else {
        k_phi<<<egrid, 256, 0, st>>>(w.S, nullptr, w.F, N, 0, 1, nullptr, w.status); g_launches++;
    }
    for (int it = 0; it < kFixedPointSweeps; it++) {
        if ((e = launch_split(w.F, N, N, N, sZ, false, nullptr, st)) != cudaSuccess) return e;
        TcParams g{};
        g.rows = (int)N; g.cols = (int)N; g.ldo = N; g.status = w.status;
        g.epi = TC_EPI_STORE; g.out = w.Z; g.lower_only = 1;
        if ((e = launch_gemm_tc(sZ, sZ, g, nullptr, st)) != cudaSuccess) return e;
        k_phi<<<egrid, 256, 0, st>>>(w.S, w.Z, w.F, N, it + 1 == kFixedPointSweeps, 1, nullptr, w.status); g_launches++;
    }
    // 6. W^T = V1^T - V1^T F^T (split product, in place on V1^T), then V = V1 - F W (digits)
    if ((e = launch_transpose(w.Y, w.W, N, st)) != cudaSuccess) return e;
    if ((e = launch_split(w.W, N, N, N, sY, false, nullptr, st)) != cudaSuccess) return e;
    if ((e = launch_split(w.F, N, N, N, sZ, false, nullptr, st)) != cudaSuccess) return e;
    TcParams t{};
    t.rows = (int)N; t.cols = (int)N; t.ldo = N; t.status = w.status; t.bn = h->tc_bn;
    t.epi = TC_EPI_RSUB; t.out = w.W; t.V = w.W;
    if ((e = launch_gemm_tc(sY, sZ, t, nullptr, st)) != cudaSuccess) return e;
    if ((e = launch_oz_split(w.F, N, N, N, dP, w.ozeP, st)) != cudaSuccess) return e;
    if ((e = launch_oz_split(w.W, N, N, N, dQ, w.ozeQ, st)) != cudaSuccess) return e;
    // F is of order |E| (1e-7 here), so F W needs about 1e-9 of its own size: six digit levels
    // (about sqrt(7 N) 2^-42 / 3 of 2^(e_r + e_c), e_r the exponent of F's row)
    o = OzParams{};
    o.rows = (int)N; o.cols = (int)N; o.C = w.Y; o.ldc = N; o.sub = 1; o.p_lower = 1; o.levels = 6; o.status = w.status;
    if ((e = launch_gemm_oz(dP, w.ozeP, dQ, w.ozeQ, o, st)) != cudaSuccess) return e;
    // the orthonormal vectors now live in Y: swap the buffers so X holds V
    double *tmp = w.X;
    w.X = w.Y;
    w.Y = tmp;
    return cudaGetLastError();
}

}  // namespace pfsm
