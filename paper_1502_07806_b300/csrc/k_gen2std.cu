// Generalized -> standard conversion of A x = lambda B x (Eq. 14-15), the step before the
// eigensolve: B is the overlap matrix, diagonally dominant and close to the identity.
//
// run_gen_to_std: Z = B^{-1} A by the Jacobi iteration of Eq. 14,
//   Z_{n+1} = (I - D^{-1} B) Z_n + D^{-1} A = Z_n + D^{-1} (A - B Z_n),  D = diag(B),  Z_0 = 0,
// stopped when max|A - B Z_n| <= tol max|A| (measured before each update) or after max_iters
// updates. The iteration runs on W = Z^T, so that both operands of its product are read along
// rows (the K-major layout of the tensor-core kernel): W_{n+1} = W_n + (A - W_n B) D^{-1} (A, B
// symmetric). R = A - W B is one FP64-accurate digit product (k_gemm_oz, subtracting into a copy
// of A) with B's digits split once; the update scales column c by 1 / B_cc.
//
// run_gen_to_std_sym: the symmetric form C = B^{-1/2} A B^{-1/2} (a stated deviation: the
// eigensolver needs a symmetric matrix, B^{-1} A is not one; same eigenvalues, eigenvectors
// x = B^{-1/2} y), with S = B^{-1/2} by the coupled Newton-Schulz iteration for the matrix square
// root and its inverse (Higham, Functions of Matrices, 2008): c = the largest Gershgorin row
// bound of B, Y_0 = B / c, Q_0 = I; P_k = Q_k Y_k; T_k = (3 I - P_k) / 2; Y_{k+1} = Y_k T_k;
// Q_{k+1} = T_k Q_k; stop when max|I - P_k| <= tol or after max_iters updates; S = Q / sqrt(c),
// C = S A S. Each product X Y is the digit product of X's rows with the rows of Y^T (a transpose
// first): the iterates are polynomials in B, symmetric in exact arithmetic, but taking Y for Y^T
// lets their rounding asymmetry grow about tenfold every five updates once the iteration has
// converged (seen in an FP64 emulation), while the true product stays at the rounding level.
//
// Both run on the caller's stream with temporaries from cudaMallocAsync and read one 8-byte
// residual back per iteration (the stopping decision).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <utility>

#include "pfsm_internal.cuh"

namespace pfsm {

namespace {

// max |x| over n entries into *out (bit patterns of non-negative doubles order like integers;
// *out zeroed by the caller)
__global__ void k_absmax(const double *__restrict__ x, int64_t n, unsigned long long *__restrict__ out)
{
    double m = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        m = fmax(m, fabs(x[i]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(m));
}

// largest Gershgorin row bound sum_j |B_ij| (one warp per row)
__global__ void k_rowbound(const double *__restrict__ B, int64_t N, unsigned long long *__restrict__ out)
{
    const int64_t r = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (r >= N) return;
    double s = 0.0;
    for (int64_t j = lane; j < N; j += 32) s += fabs(B[r * N + j]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) atomicMax(out, (unsigned long long)__double_as_longlong(s));
}

// dinv = 1 / diag(B); a zero diagonal entry sets *bad
__global__ void k_diag_inv(const double *__restrict__ B, int64_t N, double *__restrict__ dinv, int32_t *__restrict__ bad)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const double d = B[i * N + i];
    if (d == 0.0) *bad = 1;
    dinv[i] = (d != 0.0) ? 1.0 / d : 0.0;
}

// W += R diag(dinv) (column c scaled by dinv[c])
__global__ void k_jacobi_update(double *__restrict__ W, const double *__restrict__ R, const double *__restrict__ dinv,
                                int64_t N)
{
    const int64_t n2 = N * N;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n2; i += (int64_t)gridDim.x * blockDim.x)
        W[i] = fma(R[i], dinv[i % N], W[i]);
}

// dst = s * src (s == 0: the identity)
__global__ void k_scale_or_eye(const double *__restrict__ src, double *__restrict__ dst, int64_t N, double s)
{
    const int64_t n2 = N * N;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n2; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = src ? s * src[i] : ((i / N == i % N) ? 1.0 : 0.0);
}

// T = (3 I - P) / 2 and *rmax = max |I - P| (zeroed by the caller)
__global__ void k_ns_t(const double *__restrict__ P, double *__restrict__ T, int64_t N, unsigned long long *__restrict__ rmax)
{
    const int64_t n2 = N * N;
    double m = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n2; i += (int64_t)gridDim.x * blockDim.x) {
        const double e = (i / N == i % N) ? 1.0 : 0.0;
        const double p = P[i];
        m = fmax(m, fabs(e - p));
        T[i] = 0.5 * (3.0 * e - p);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(rmax, (unsigned long long)__double_as_longlong(m));
}

unsigned grid_for(int64_t n) { return (unsigned)std::min<int64_t>((n + 255) / 256, (int64_t)sm_count() * 8); }

cudaError_t read_max(unsigned long long *dev, double &out, cudaStream_t st)
{
    unsigned long long h = 0;
    cudaError_t e;
    if ((e = cudaMemcpyAsync(&h, dev, sizeof(h), cudaMemcpyDeviceToHost, st)) != cudaSuccess) return e;
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
    std::memcpy(&out, &h, sizeof(out));
    return cudaSuccess;
}

}  // namespace

cudaError_t make_digits(Digits &d, int64_t N, cudaStream_t st)
{
    const int64_t ld = padded_ld(N);
    const size_t bytes = (size_t)OZ_SLICES * N * ld * 2;
    cudaError_t e;
    if ((e = cudaMallocAsync(&d.sl, bytes, st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(d.sl, 0, bytes, st)) != cudaSuccess) return e;   // K padding stays zero
    if ((e = cudaMallocAsync((void **)&d.ex, N * sizeof(int32_t), st)) != cudaSuccess) return e;
    d.buf = SliceBuf{d.sl, N, ld, OZ_SLICES, 0};
    return cudaSuccess;
}

void free_digits(Digits &d, cudaStream_t st)
{
    if (d.sl) cudaFreeAsync(d.sl, st);
    if (d.ex) cudaFreeAsync(d.ex, st);
    d = Digits{};
}

cudaError_t digit_product(const Digits &dx, const Digits &dy, double *C, int64_t N, bool sub, int32_t *status,
                          cudaStream_t st)
{
    OzParams o{};
    o.rows = (int)N; o.cols = (int)N; o.C = C; o.ldc = N; o.sub = sub ? 1 : 0; o.status = status;
    return launch_gemm_oz(dx.buf, dx.ex, dy.buf, dy.ex, o, st);
}

cudaError_t dense_product(const double *X, const double *Yrows, double *C, int64_t N, Digits &dx, Digits &dy,
                          int32_t *status, cudaStream_t st)
{
    cudaError_t e;
    if ((e = launch_oz_split(X, N, N, N, dx.buf, dx.ex, st)) != cudaSuccess) return e;
    if ((e = launch_oz_split(Yrows, N, N, N, dy.buf, dy.ex, st)) != cudaSuccess) return e;
    return digit_product(dx, dy, C, N, false, status, st);
}

namespace {
__global__ void k_symmetrize(const double *__restrict__ T, double *__restrict__ S, int64_t N)
{
    const int64_t n2 = N * N;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n2; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = i / N, c = i % N;
        S[i] = 0.5 * (T[i] + T[c * N + r]);
    }
}
}  // namespace

cudaError_t launch_symmetrize(const double *T, double *S, int64_t N, cudaStream_t st)
{
    const unsigned grid = (unsigned)std::min<int64_t>((N * N + 255) / 256, (int64_t)sm_count() * 8);
    k_symmetrize<<<grid, 256, 0, st>>>(T, S, N);
    g_launches++;
    return cudaGetLastError();
}

cudaError_t run_gen_to_std(int64_t N, const double *A, const double *B, double *Z, int max_iters, double tol,
                           cudaStream_t st, Gen2StdResult &res)
{
    const size_t n2b = (size_t)N * N * sizeof(double);
    double *W = nullptr, *R = nullptr, *dinv = nullptr;
    unsigned long long *mx = nullptr;
    int32_t *flags = nullptr;                      // [0] zero diagonal, [1] device status
    Digits dW, dB;
    cudaError_t e = cudaSuccess;
    res = Gen2StdResult{};
    auto step = [&](cudaError_t x) { if (e == cudaSuccess) e = x; return e == cudaSuccess; };
    step(cudaMallocAsync((void **)&W, n2b, st));
    step(cudaMallocAsync((void **)&R, n2b, st));
    step(cudaMallocAsync((void **)&dinv, N * sizeof(double), st));
    step(cudaMallocAsync((void **)&mx, 2 * sizeof(unsigned long long), st));
    step(cudaMallocAsync((void **)&flags, 2 * sizeof(int32_t), st));
    step(make_digits(dW, N, st));
    step(make_digits(dB, N, st));
    if (e == cudaSuccess) {
        step(cudaMemsetAsync(flags, 0, 2 * sizeof(int32_t), st));
        step(cudaMemsetAsync(mx, 0, 2 * sizeof(unsigned long long), st));
        step(cudaMemsetAsync(W, 0, n2b, st));                                  // W_0 = 0
        k_diag_inv<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(B, N, dinv, flags); g_launches++;
        k_absmax<<<grid_for(N * N), 256, 0, st>>>(A, N * N, mx); g_launches++;
        step(cudaGetLastError());
        step(launch_oz_split(B, N, N, N, dB.buf, dB.ex, st));                 // B's digits, once
    }
    double amax = 0.0;
    int32_t hflags[2] = {0, 0};
    if (e == cudaSuccess) step(read_max(mx, amax, st));
    if (e == cudaSuccess) step(cudaMemcpy(hflags, flags, sizeof(hflags), cudaMemcpyDeviceToHost));
    if (e == cudaSuccess && hflags[0]) res.status = PFSM_ERR_INVALID_ARG;
    if (amax == 0.0) amax = 1.0;
    res.status = res.status ? res.status : PFSM_ERR_NOT_CONVERGED;
    for (int it = 0; e == cudaSuccess && res.status == PFSM_ERR_NOT_CONVERGED; it++) {
        // R = A - W B (B symmetric: W B = W B^T, the product of W's rows with B's rows)
        step(cudaMemcpyAsync(R, A, n2b, cudaMemcpyDeviceToDevice, st));
        if (it > 0) {
            step(launch_oz_split(W, N, N, N, dW.buf, dW.ex, st));
            step(digit_product(dW, dB, R, N, true, flags + 1, st));
        }
        step(cudaMemsetAsync(mx + 1, 0, sizeof(unsigned long long), st));
        k_absmax<<<grid_for(N * N), 256, 0, st>>>(R, N * N, mx + 1); g_launches++;
        step(cudaGetLastError());
        double r = 0.0;
        if (!step(read_max(mx + 1, r, st))) break;
        res.resid = r / amax;
        res.iters = it;
        if (res.resid <= tol) { res.status = PFSM_OK; break; }
        if (it >= max_iters) break;
        k_jacobi_update<<<grid_for(N * N), 256, 0, st>>>(W, R, dinv, N); g_launches++;
        step(cudaGetLastError());
    }
    if (e == cudaSuccess && res.status != PFSM_ERR_INVALID_ARG) step(launch_transpose(W, Z, N, st));   // Z = W^T
    if (e == cudaSuccess) step(cudaMemcpyAsync(hflags, flags, sizeof(hflags), cudaMemcpyDeviceToHost, st));
    if (e == cudaSuccess) step(cudaStreamSynchronize(st));
    if (e == cudaSuccess && hflags[1]) res.status = hflags[1];                 // a device wait gave up
    free_digits(dW, st);
    free_digits(dB, st);
    if (W) cudaFreeAsync(W, st);
    if (R) cudaFreeAsync(R, st);
    if (dinv) cudaFreeAsync(dinv, st);
    if (mx) cudaFreeAsync(mx, st);
    if (flags) cudaFreeAsync(flags, st);
    return e;
}

cudaError_t run_gen_to_std_sym(int64_t N, const double *A, const double *B, double *C, double *S, int max_iters,
                               double tol, cudaStream_t st, Gen2StdResult &res)
{
    const size_t n2b = (size_t)N * N * sizeof(double);
    double *Y = nullptr, *Q = nullptr, *P = nullptr, *T = nullptr, *W = nullptr, *Yt = nullptr;
    unsigned long long *mx = nullptr;
    int32_t *status = nullptr;
    Digits d1, d2;
    cudaError_t e = cudaSuccess;
    res = Gen2StdResult{};
    auto step = [&](cudaError_t x) { if (e == cudaSuccess) e = x; return e == cudaSuccess; };
    step(cudaMallocAsync((void **)&Y, n2b, st));
    step(cudaMallocAsync((void **)&Q, n2b, st));
    step(cudaMallocAsync((void **)&P, n2b, st));
    step(cudaMallocAsync((void **)&T, n2b, st));
    step(cudaMallocAsync((void **)&W, n2b, st));
    step(cudaMallocAsync((void **)&Yt, n2b, st));
    step(cudaMallocAsync((void **)&mx, 2 * sizeof(unsigned long long), st));
    step(cudaMallocAsync((void **)&status, sizeof(int32_t), st));
    step(make_digits(d1, N, st));
    step(make_digits(d2, N, st));
    // C = X Y: digits of X's rows and of Y^T's rows
    auto prod = [&](const double *X, const double *Yv, double *Cout) {
        step(launch_oz_split(X, N, N, N, d1.buf, d1.ex, st));
        step(launch_transpose(Yv, Yt, N, st));
        step(launch_oz_split(Yt, N, N, N, d2.buf, d2.ex, st));
        step(digit_product(d1, d2, Cout, N, false, status, st));
    };
    double c = 0.0;
    if (e == cudaSuccess) {
        step(cudaMemsetAsync(status, 0, sizeof(int32_t), st));
        step(cudaMemsetAsync(mx, 0, 2 * sizeof(unsigned long long), st));
        k_rowbound<<<(unsigned)((N + 7) / 8), 256, 0, st>>>(B, N, mx); g_launches++;
        step(cudaGetLastError());
        step(read_max(mx, c, st));
    }
    if (e == cudaSuccess && !(c > 0.0)) res.status = PFSM_ERR_NOT_SPD;
    if (e == cudaSuccess && res.status == 0) {
        k_scale_or_eye<<<grid_for(N * N), 256, 0, st>>>(B, Y, N, 1.0 / c); g_launches++;   // Y_0 = B / c
        k_scale_or_eye<<<grid_for(N * N), 256, 0, st>>>(nullptr, Q, N, 0.0); g_launches++; // Q_0 = I
        step(cudaGetLastError());
        res.status = PFSM_ERR_NOT_CONVERGED;
        for (int it = 0; e == cudaSuccess; it++) {
            prod(Q, Y, P);                                                     // P = Q Y
            step(cudaMemsetAsync(mx + 1, 0, sizeof(unsigned long long), st));
            k_ns_t<<<grid_for(N * N), 256, 0, st>>>(P, T, N, mx + 1); g_launches++;   // T, max|I - P|
            step(cudaGetLastError());
            double r = 0.0;
            if (!step(read_max(mx + 1, r, st))) break;
            res.resid = r;
            res.iters = it;
            if (r <= tol) { res.status = PFSM_OK; break; }
            if (it >= max_iters) break;
            prod(Y, T, W);                                                     // Y = Y T
            std::swap(Y, W);
            prod(T, Q, W);                                                     // Q = T Q
            std::swap(Q, W);
        }
        // S = Q / sqrt(c); C = S A S
        k_scale_or_eye<<<grid_for(N * N), 256, 0, st>>>(Q, S, N, 1.0 / std::sqrt(c)); g_launches++;
        step(cudaGetLastError());
        prod(S, A, W);
        prod(W, S, C);
    }
    int32_t hs = 0;
    if (e == cudaSuccess) step(cudaMemcpyAsync(&hs, status, sizeof(hs), cudaMemcpyDeviceToHost, st));
    if (e == cudaSuccess) step(cudaStreamSynchronize(st));
    if (e == cudaSuccess && hs) res.status = hs;
    free_digits(d1, st);
    free_digits(d2, st);
    for (double *p : {Y, Q, P, T, W, Yt})
        if (p) cudaFreeAsync(p, st);
    if (mx) cudaFreeAsync(mx, st);
    if (status) cudaFreeAsync(status, st);
    return e;
}

}  // namespace pfsm
