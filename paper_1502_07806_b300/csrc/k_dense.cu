// Gram-Schmidt of the FP64 form (Section II, after the Eq. 11 iterations), Rayleigh quotients /
// residuals, and the eigen-adjoint backward, FP64. (The mixed forms orthonormalise in
// k_gs_mixed.cu.)
//
// Gram-Schmidt is done as Cholesky-QR. With the vectors as rows of X:
//   S = X X^T (overlap, lower triangle), S = L L^T (blocked right-looking Cholesky),
//   V = L^-1 X (blocked forward substitution over the rows, as GEMMs with the inverses of the
//   64 x 64 diagonal blocks of L, so nearly all FP64 work runs in the FP64 GEMM kernel).
// In exact arithmetic this is the QR factorisation with positive R diagonal, i.e. Gram-Schmidt
// in ascending index order. L_jj^2 is the squared norm of vector j after projecting out vectors
// 0..j-1 and S_jj its squared norm before, so L_jj < 1e-8 sqrt(S_jj) is the breakdown test.
#include <cfloat>

#include "pfsm_internal.cuh"

namespace pfsm {

constexpr int CB = 64;   // Cholesky / TRSM block

__global__ void k_copy_diag(const double *__restrict__ S, int64_t N, double *__restrict__ d)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) d[i] = S[i * N + i];
}

// 1/sqrt(d) without FP64 sqrt/divide sequences (~10 dependent FP64 instructions, ~64 cycles each
// on B300): FP32 estimate and two Newton steps y <- y (3 - d y^2) / 2. Needs d in FP32 range.
__device__ __forceinline__ double fast_rsqrt(double d)
{
    double y = (double)rsqrtf((float)d);
    y = y * fma(-0.5 * d, y * y, 1.5);
    y = y * fma(-0.5 * d, y * y, 1.5);
    return y;
}

// Cholesky of the b x b diagonal block at (jb, jb), in shared memory, one CTA of 256 threads; also
// writes the block's inverse L_jj^-1 (lower triangular, CB x CB, zero padded) to Linv.
// The inverse is formed in two levels, L = [A 0; B C] -> L^-1 = [A^-1 0; -C^-1 B A^-1 C^-1]: the
// two 32 x 32 diagonal inverses are built concurrently row by row (each row's sums split four
// ways), then the off-diagonal block is two 32 x 32 x 32 products.
__global__ void __launch_bounds__(256)
k_potrf_inv(double *__restrict__ S, int64_t N, int64_t jb, int b, const double *__restrict__ sdiag,
            int32_t *status, double *__restrict__ Linv)
{
    constexpr int H = CB / 2;
    extern __shared__ double potrf_sm[];   // L and X, CB x (CB + 1) each (dynamic: > 48 KB)
    double(*L)[CB + 1] = reinterpret_cast<double(*)[CB + 1]>(potrf_sm);
    double(*X)[CB + 1] = reinterpret_cast<double(*)[CB + 1]>(potrf_sm + CB * (CB + 1));
    __shared__ double R[CB];              // 1 / L_jj
    __shared__ double part[4][2][H];
    const int tid = threadIdx.x;
    for (int t = tid; t < CB * CB; t += blockDim.x) {
        const int i = t / CB, k = t % CB;
        // pad the block to CB x CB with the identity so the fixed-size inverse stays exact
        L[i][k] = (i < b && k < b) ? ((k <= i) ? S[(jb + i) * N + jb + k] : 0.0) : (i == k ? 1.0 : 0.0);
        X[i][k] = 0.0;
    }
    __shared__ double REF[CB];            // sqrt of the overlap's diagonal (norms before projection)
    if (tid < b) REF[tid] = sqrt(fmax(sdiag[jb + tid], 0.0));
    __syncthreads();
    // Right-looking factorisation on the unscaled columns: step j updates the trailing lower
    // triangle with (L[i][j] L[k][j]) / d_j; column j is never read after step j, so all columns
    // are scaled by 1/sqrt(d_j) at the end. Two barriers per column.
    const int warp = tid >> 5, lane = tid & 31, nw = blockDim.x >> 5;
    for (int j = 0; j < b; j++) {
        if (tid == 0) {
            const double d = L[j][j];
            double y = (d > 1e-300 && d < 1e300) ? fast_rsqrt(d) : 0.0;
            const double l = d * y;
            if (!(l >= 1e-8 * REF[j]) || !(y > 0.0) || !isfinite(l)) {
                set_status(status, PFSM_ERR_NOT_SPD);
                y = 1.0;   // keep the arithmetic finite; the result is flagged as invalid
            }
            R[j] = y;
        }
        __syncthreads();
        const double c = R[j] * R[j];
        for (int i = j + 1 + warp; i < b; i += nw) {
            const double aij = L[i][j] * c;
            for (int k = j + 1 + lane; k <= i; k += 32) L[i][k] = fma(-aij, L[k][j], L[i][k]);
        }
        __syncthreads();
    }
    for (int t = tid; t < b * b; t += blockDim.x) {
        const int i = t / b, k = t % b;
        if (k < i) L[i][k] *= R[k];
        else if (k == i) L[i][i] = 1.0 / R[i];      // sqrt(d_i) = d_i / sqrt(d_i)
    }
    for (int j = b + tid; j < CB; j += blockDim.x) R[j] = 1.0;
    __syncthreads();
    for (int t = tid; t < b * b; t += blockDim.x) {
        const int i = t / b, k = t % b;
        if (k <= i) S[(jb + i) * N + jb + k] = L[i][k];
    }
    __syncthreads();
    // level 1: A^-1 (rows 0..H-1) and C^-1 (rows H..CB-1), row by row
    {
        const int half = tid / 128, c = tid % H, pp = (tid % 128) / H;   // pp in 0..3
        const int off = half * H;
        for (int i = 0; i < H; i++) {
            double sum = 0.0;
            for (int k = c + pp; k < i; k += 4) sum = fma(L[off + i][off + k], X[off + k][off + c], sum);
            part[pp][half][c] = sum;
            __syncthreads();
            if (pp == 0 && c <= i) {
                const double t = part[0][half][c] + part[1][half][c] + part[2][half][c] + part[3][half][c];
                X[off + i][off + c] = ((i == c) ? 1.0 - t : -t) * R[off + i];
            }
            __syncthreads();
        }
    }
    // level 2: T = B A^-1 (kept in X's upper-right block, unused otherwise), then -C^-1 T
    for (int t = tid; t < H * H; t += blockDim.x) {
        const int i = t / H, c = t % H;
        double acc = 0.0;
        for (int k = c; k < H; k++) acc = fma(L[H + i][k], X[k][c], acc);
        X[i][H + c] = acc;
    }
    __syncthreads();
    for (int t = tid; t < H * H; t += blockDim.x) {
        const int i = t / H, c = t % H;
        double acc = 0.0;
        for (int k = 0; k <= i; k++) acc = fma(X[H + i][H + k], X[k][H + c], acc);
        X[H + i][c] = -acc;
    }
    __syncthreads();
    for (int t = tid; t < CB * CB; t += blockDim.x) {
        const int i = t / CB, k = t % CB;
        Linv[i * CB + k] = (i < b && k <= i) ? X[i][k] : 0.0;
    }
}

constexpr size_t kPotrfSmem = 2 * CB * (CB + 1) * sizeof(double);

cudaError_t configure_dense_kernels()
{
    return cudaFuncSetAttribute(k_potrf_inv, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kPotrfSmem);
}

cudaError_t launch_gram_schmidt_f64(pfsm_handle_s *h, cudaStream_t st)
{
    Workspace &w = h->ws;
    const int64_t N = h->N;
    cudaError_t e;
    // S = X X^T (lower)
    GemmArgs g{};
    g.rows = N; g.cols = N; g.K = N;
    g.P = w.X; g.ldp = N; g.Q = w.X; g.ldq = N; g.C = w.S; g.ldc = N; g.lower_only = 1;
    if ((e = launch_gemm_f64(g, EPI_STORE, Q_KMAJOR, st)) != cudaSuccess) return e;
    if ((e = launch_copy_diag(w.S, N, w.sdiag, st)) != cudaSuccess) return e;
    if (h->timing && (e = cudaEventRecord(h->gs_ev[0], st)) != cudaSuccess) return e;
    // blocked right-looking Cholesky S = L L^T: diagonal blocks of L stay in S with their inverses in
    // Linv, the off-diagonal panels of L go to W
    for (int64_t jb = 0; jb < N; jb += CB) {
        const int b = (int)((N - jb) < CB ? (N - jb) : CB);
        double *Li = w.Linv + jb * CB;
        k_potrf_inv<<<1, 256, kPotrfSmem, st>>>(w.S, N, jb, b, w.sdiag, w.status, Li); g_launches++;
        const int64_t rest = N - jb - b;
        if (rest <= 0) break;
        // panel: L[rest, jb] = S[rest, jb] L_jj^-T, written to W at the same position (not in
        // place: several CTAs read each row of the operand)
        GemmArgs pn{};
        pn.rows = rest; pn.cols = b; pn.K = b;
        pn.P = w.S + (jb + b) * N + jb; pn.ldp = N;
        pn.Q = Li; pn.ldq = CB;
        pn.C = w.W + (jb + b) * N + jb; pn.ldc = N;
        if ((e = launch_gemm_f64(pn, EPI_STORE, Q_KMAJOR, st)) != cudaSuccess) return e;
        GemmArgs u{};
        u.rows = rest; u.cols = rest; u.K = b;
        u.P = w.W + (jb + b) * N + jb; u.ldp = N;
        u.Q = w.W + (jb + b) * N + jb; u.ldq = N;
        u.C = w.S + (jb + b) * N + jb + b; u.ldc = N; u.lower_only = 1;
        if ((e = launch_gemm_f64(u, EPI_SUB, Q_KMAJOR, st)) != cudaSuccess) return e;
    }
    if (h->timing && (e = cudaEventRecord(h->gs_ev[1], st)) != cudaSuccess) return e;
    // V = L^-1 X by blocks of rows, written to Y: V_b = L_bb^-1 X_b, then X_rest -= L_rest,b V_b
    for (int64_t jb = 0; jb < N; jb += CB) {
        const int b = (int)((N - jb) < CB ? (N - jb) : CB);
        GemmArgs dg{};
        dg.rows = b; dg.cols = N; dg.K = b;
        dg.P = w.Linv + jb * CB; dg.ldp = CB;
        dg.Q = w.X + jb * N; dg.ldq = N;
        dg.C = w.Y + jb * N; dg.ldc = N;
        if ((e = launch_gemm_f64(dg, EPI_STORE, Q_NMAJOR, st)) != cudaSuccess) return e;
        const int64_t rest = N - jb - b;
        if (rest <= 0) break;
        GemmArgs u{};
        u.rows = rest; u.cols = N; u.K = b;
        u.P = w.W + (jb + b) * N + jb; u.ldp = N;        // off-diagonal panels of L live in W
        u.Q = w.Y + jb * N; u.ldq = N;
        u.C = w.X + (jb + b) * N; u.ldc = N;
        if ((e = launch_gemm_f64(u, EPI_SUB, Q_NMAJOR, st)) != cudaSuccess) return e;
    }
    // the orthonormal vectors now live in Y: swap the buffers so X holds V
    double *t = w.X;
    w.X = w.Y;
    w.Y = t;
    return cudaGetLastError();
}

// ---- Rayleigh quotients and residual norms (warp-shuffle row reductions) --------------------

// One warp per vector k: lambda_k = v_k . w_k, r_k = ||w_k - lambda_k v_k|| with W = V A (rows).
// A warp's shuffle tree is five FP64 adds; a CTA-wide sum per vector (shared memory, a barrier and
// a second tree) issued about as many FP64 instructions as the dot products themselves.
__global__ void __launch_bounds__(256)
k_rayleigh_rows(const double *__restrict__ V, const double *__restrict__ W, int64_t N, double *__restrict__ lam,
                double *__restrict__ res)
{
    const int64_t k = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (k >= N) return;
    const double *v = V + k * N, *w = W + k * N;
    double a0 = 0.0, a1 = 0.0;
    int64_t i = lane;
    for (; i + 32 < N; i += 64) { a0 = fma(v[i], w[i], a0); a1 = fma(v[i + 32], w[i + 32], a1); }
    if (i < N) a0 = fma(v[i], w[i], a0);
    double l = a0 + a1;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
    double r0 = 0.0, r1 = 0.0;
    for (i = lane; i + 32 < N; i += 64) {
        const double t0 = fma(-l, v[i], w[i]), t1 = fma(-l, v[i + 32], w[i + 32]);
        r0 = fma(t0, t0, r0);
        r1 = fma(t1, t1, r1);
    }
    if (i < N) { const double t0 = fma(-l, v[i], w[i]); r0 = fma(t0, t0, r0); }
    double r2 = r0 + r1;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) r2 += __shfl_xor_sync(0xffffffffu, r2, o);
    if (lane == 0) { lam[k] = l; res[k] = sqrt(r2); }
}

__global__ void k_transpose(const double *__restrict__ in, double *__restrict__ out, int64_t N)
{
    __shared__ double t[32][33];
    const int64_t bx = (int64_t)blockIdx.x * 32, by = (int64_t)blockIdx.y * 32;
    for (int j = threadIdx.y; j < 32; j += blockDim.y) {
        int64_t r = by + j, c = bx + threadIdx.x;
        if (r < N && c < N) t[j][threadIdx.x] = in[r * N + c];
    }
    __syncthreads();
    for (int j = threadIdx.y; j < 32; j += blockDim.y) {
        int64_t r = bx + j, c = by + threadIdx.x;
        if (r < N && c < N) out[r * N + c] = t[threadIdx.x][j];
    }
}

cudaError_t launch_copy_diag(const double *S, int64_t N, double *d, cudaStream_t st)
{
    k_copy_diag<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(S, N, d); g_launches++;
    return cudaGetLastError();
}

cudaError_t launch_transpose(const double *in, double *out, int64_t N, cudaStream_t st)
{
    dim3 grid((unsigned)((N + 31) / 32), (unsigned)((N + 31) / 32));
    k_transpose<<<grid, dim3(32, 8), 0, st>>>(in, out, N); g_launches++;
    return cudaGetLastError();
}

cudaError_t launch_rayleigh_f64(pfsm_handle_s *h, const double *A, double *eigvals_out,
                                double *V_out, cudaStream_t st)
{
    Workspace &w = h->ws;
    const int64_t N = h->N;
    cudaError_t e;
    if (h->prm.precision != PFSM_FP64) {   // W = V A with FP64-accurate tensor-core digits
        SliceBuf dv{w.ozP, N, padded_ld(N), OZ_SLICES, 0};
        if ((e = launch_oz_split(w.X, N, N, N, dv, w.ozeP, st)) != cudaSuccess) return e;
        // A = diag(d) + E: digits of E only (split during the window eigensolves on the side stream
        // when the handle has one), the diagonal term added exactly in FP64
        const bool presplit = h->a_split;
        SliceBuf da{presplit ? w.ozA : w.ozQ, N, padded_ld(N), OZ_SLICES, 0};
        int32_t *ea = presplit ? w.ozeA : w.ozeQ;
        if (!presplit && (e = launch_oz_split(A, N, N, N, da, ea, st, true, w.dA)) != cudaSuccess) return e;
        OzParams o{};
        o.rows = (int)N; o.cols = (int)N; o.C = w.W; o.ldc = N; o.status = w.status;
        o.Vp = w.X; o.ldv = N; o.dcol = w.dA;
        // six digit levels: E's entries are small against A's diagonal, so the first dropped level
        // (about sqrt(7 N) 2^-42 / 3 of max|V_r| max|E_c|) stays far below FP64 rounding of A V
        o.levels = 6;
        if ((e = launch_gemm_oz(dv, w.ozeP, da, ea, o, st)) != cudaSuccess) return e;
    } else {
        GemmArgs g{};
        g.rows = N; g.cols = N; g.K = N;
        g.P = w.X; g.ldp = N; g.Q = A; g.ldq = N; g.C = w.W; g.ldc = N;
        if ((e = launch_gemm_f64(g, EPI_STORE, Q_KMAJOR, st)) != cudaSuccess) return e;
    }
    k_rayleigh_rows<<<(unsigned)((N + 7) / 8), 256, 0, st>>>(w.X, w.W, N, w.lam, w.res); g_launches++;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = launch_transpose(w.X, w.Vrm, N, st)) != cudaSuccess) return e;
    if (eigvals_out != w.lam &&
        (e = cudaMemcpyAsync(eigvals_out, w.lam, (size_t)N * sizeof(double), cudaMemcpyDeviceToDevice, st)) != cudaSuccess)
        return e;
    if (V_out == w.Vrm) return cudaSuccess;
    return cudaMemcpyAsync(V_out, w.Vrm, (size_t)N * N * sizeof(double), cudaMemcpyDeviceToDevice, st);
}

// ---- adaptive variant of Eq. 11: Rayleigh-quotient shifts and the residual ----------------------

// One warp per vector k (rows of X and Y = (A - eps I) X): delta = x.y / x.x; eps += delta;
// y -= delta x; alpha from the new shift (min(theta / d^2, 1 - 2^-20), d the larger distance to
// the Gershgorin ends); the residual ||y|| / ||x|| into *rmax (atomic max on non-negative bits).
__global__ void k_rq_shift(const double *__restrict__ X, double *__restrict__ Y, double *__restrict__ eps,
                           double *__restrict__ alpha, const double *__restrict__ gersh, double theta, int64_t N,
                           unsigned long long *__restrict__ rmax)
{
    const int64_t k = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (k >= N) return;
    const double *x = X + k * N;
    double *y = Y + k * N;
    double xy = 0.0, xx = 0.0;
    for (int64_t i = lane; i < N; i += 32) { xy = fma(x[i], y[i], xy); xx = fma(x[i], x[i], xx); }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        xy += __shfl_xor_sync(0xffffffffu, xy, o);
        xx += __shfl_xor_sync(0xffffffffu, xx, o);
    }
    const double delta = xy / xx;
    double yy = 0.0;
    for (int64_t i = lane; i < N; i += 32) {
        const double v = fma(-delta, x[i], y[i]);
        y[i] = v;
        yy = fma(v, v, yy);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) yy += __shfl_xor_sync(0xffffffffu, yy, o);
    if (lane == 0) {
        const double e = eps[k] + delta;
        eps[k] = e;
        const double glo = gersh[2 * N], ghi = gersh[2 * N + 1];
        const double dmax = fmax(ghi - e, e - glo);
        const double a = theta / (dmax * dmax), cap = 1.0 - 0x1.0p-20;
        alpha[k] = (a < cap) ? a : cap;
        atomicMax(rmax, (unsigned long long)__double_as_longlong(sqrt(yy / xx)));
    }
}

cudaError_t launch_rq_shift(double *X, double *Y, double *eps, double *alpha, const double *gersh, double theta,
                            int64_t N, unsigned long long *rmax, cudaStream_t st)
{
    k_rq_shift<<<(unsigned)((N + 7) / 8), 256, 0, st>>>(X, Y, eps, alpha, gersh, theta, N, rmax);
    g_launches++;
    return cudaGetLastError();
}

// ---- eigen-adjoint ----------------------------------------------------------------------------

// In place on G = V^T dV: M_kl = sym(diag(dlam) + F o G), F_kl = 1/(lam_l - lam_k) masked.
__global__ void k_adjoint_mix(double *__restrict__ G, int64_t N, const double *__restrict__ lam,
                              const double *__restrict__ dlam, double tau)
{
    const int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t k = blockIdx.y;
    if (l >= N || l < k) return;
    if (l == k) { G[k * N + k] = dlam ? dlam[k] : 0.0; return; }
    const double gap = lam[l] - lam[k];
    const double fkl = (fabs(gap) >= tau) ? 1.0 / gap : 0.0;    // F_kl
    const double flk = (fabs(gap) >= tau) ? -1.0 / gap : 0.0;   // F_lk
    const double m = 0.5 * (fkl * G[k * N + l] + flk * G[l * N + k]);
    G[k * N + l] = m;
    G[l * N + k] = m;
}

__global__ void k_symmetrize(double *__restrict__ D, int64_t N)
{
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t i = blockIdx.y;
    if (j >= N || j <= i) return;
    const double s = 0.5 * (D[i * N + j] + D[j * N + i]);
    D[i * N + j] = s;
    D[j * N + i] = s;
}

cudaError_t launch_backward_f64(pfsm_handle_s *h, const double *dLambda, const double *dV,
                                double *dA_out, cudaStream_t st)
{
    Workspace &w = h->ws;
    const int64_t N = h->N;
    cudaError_t e;
    // G = V^T dV : G[k, l] = sum_i Vt[k, i] dVt[l, i]; Vt = X (rows), dVt = transpose(dV)
    if (dV) {
        if ((e = launch_transpose(dV, w.W, N, st)) != cudaSuccess) return e;
        GemmArgs g{};
        g.rows = N; g.cols = N; g.K = N;
        g.P = w.X; g.ldp = N; g.Q = w.W; g.ldq = N; g.C = w.S; g.ldc = N;
        if ((e = launch_gemm_f64(g, EPI_STORE, Q_KMAJOR, st)) != cudaSuccess) return e;
    } else {
        if ((e = cudaMemsetAsync(w.S, 0, (size_t)N * N * sizeof(double), st)) != cudaSuccess) return e;
    }
    dim3 gm((unsigned)((N + 255) / 256), (unsigned)N);
    k_adjoint_mix<<<gm, 256, 0, st>>>(w.S, N, w.lam, dLambda, h->prm.degen_tol); g_launches++;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    // Ut[j, k] = sum_l V[j, l] M[k, l]
    GemmArgs u{};
    u.rows = N; u.cols = N; u.K = N;
    u.P = w.Vrm; u.ldp = N; u.Q = w.S; u.ldq = N; u.C = w.Y; u.ldc = N;
    if ((e = launch_gemm_f64(u, EPI_STORE, Q_KMAJOR, st)) != cudaSuccess) return e;
    // dA[i, j] = sum_k V[i, k] Ut[j, k]
    GemmArgs d{};
    d.rows = N; d.cols = N; d.K = N;
    d.P = w.Vrm; d.ldp = N; d.Q = w.Y; d.ldq = N; d.C = dA_out; d.ldc = N;
    if ((e = launch_gemm_f64(d, EPI_STORE, Q_KMAJOR, st)) != cudaSuccess) return e;
    k_symmetrize<<<gm, 256, 0, st>>>(dA_out, N); g_launches++;
    return cudaGetLastError();
}


// The same adjoint with its three N^3 products as FP64-accurate digit products on the tensor
// cores (the mixed forms' backward): each operand row is scaled by a power of two and cut into
// seven base-128 digits, digit products of equal level are summed exactly in FP32 and the levels
// combined to FP64 (k_gemm_oz.cu), so every product carries about sqrt(K) 2^-49 of its rows'
// largest entries -- the rounding of the FP64 products it replaces. The elementwise steps
// (F o G with the degenerate-pair mask, the final symmetrisation) are the FP64 kernels above.
cudaError_t launch_backward_mixed(pfsm_handle_s *h, const double *dLambda, const double *dV,
                                  double *dA_out, cudaStream_t st)
{
    Workspace &w = h->ws;
    const int64_t N = h->N;
    const int64_t ld = padded_ld(N);
    SliceBuf dP{w.ozP, N, ld, OZ_SLICES, 0}, dQ{w.ozQ, N, ld, OZ_SLICES, 0};
    cudaError_t e;
    OzParams o{};
    o.rows = (int)N; o.cols = (int)N; o.ldc = N; o.status = w.status;
    // G = V^T dV: rows of X (vector k) against rows of dV^T (column l of dV)
    if (dV) {
        if ((e = launch_transpose(dV, w.W, N, st)) != cudaSuccess) return e;
        if ((e = launch_oz_split(w.X, N, N, N, dP, w.ozeP, st)) != cudaSuccess) return e;
        if ((e = launch_oz_split(w.W, N, N, N, dQ, w.ozeQ, st)) != cudaSuccess) return e;
        o.C = w.S;
        if ((e = launch_gemm_oz(dP, w.ozeP, dQ, w.ozeQ, o, st)) != cudaSuccess) return e;
    } else {
        if ((e = cudaMemsetAsync(w.S, 0, (size_t)N * N * sizeof(double), st)) != cudaSuccess) return e;
    }
    dim3 gm((unsigned)((N + 255) / 256), (unsigned)N);
    k_adjoint_mix<<<gm, 256, 0, st>>>(w.S, N, w.lam, dLambda, h->prm.degen_tol); g_launches++;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    // Ut = V M^T (M symmetric): rows of V (output layout) against rows of M
    if ((e = launch_oz_split(w.Vrm, N, N, N, dP, w.ozeP, st)) != cudaSuccess) return e;
    if ((e = launch_oz_split(w.S, N, N, N, dQ, w.ozeQ, st)) != cudaSuccess) return e;
    o.C = w.Y;
    if ((e = launch_gemm_oz(dP, w.ozeP, dQ, w.ozeQ, o, st)) != cudaSuccess) return e;
    // dA = V Ut^T: V's digits are still in dP
    if ((e = launch_oz_split(w.Y, N, N, N, dQ, w.ozeQ, st)) != cudaSuccess) return e;
    o.C = dA_out;
    if ((e = launch_gemm_oz(dP, w.ozeP, dQ, w.ozeQ, o, st)) != cudaSuccess) return e;
    k_symmetrize<<<gm, 256, 0, st>>>(dA_out, N); g_launches++;
    return cudaGetLastError();
}

}  // namespace pfsm
