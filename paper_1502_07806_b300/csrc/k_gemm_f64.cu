// FP64 GEMM with fused epilogues for the plain-FP64 path.
//
//   C[r, c] (op)= sum_k P[r, k] * Qop[c, k]
//     Q_KMAJOR: Qop[c, k] = Q[c * ldq + k]   (both operands read along rows)
//     Q_NMAJOR: Qop[c, k] = Q[k * ldq + c]
//
// On B300 FP64 runs on the SM's DFMA units (about 2 DFMA per clock per SM, measured 1.09 TFLOP/s
// for the whole GPU) and tcgen05 has no FP64 kind, so this kernel is FP64-ALU bound: arithmetic
// intensity of a 64x64x16 tile step is 64 DFMA per 16 bytes of shared memory traffic per
// thread, far above what the DFMA rate needs. Tiles: 64x64 outputs per CTA, K step 16, 256
// threads with 4x4 outputs each (rows ty+16i, columns tx+16j), operands staged k-major in
// shared memory with a register prefetch of the next K step.
//
// Epilogues (r = row of C, i.e. the vector index when vectors are stored as rows):
//   EPI_STORE  C = acc
//   EPI_SUB    C = C - acc
//   EPI_FS1    C = acc - eps[r] * X[r, c]                      (Y = (A - eps I) x, Eq. 11)
//   EPI_FS2    X[r, c] = X[r, c] - alpha[r] * (acc - eps[r] * Y[r, c])
//              (x <- x - alpha (A - eps I) y, the second product of Eq. 11, updated in place)
#include "pfsm_internal.cuh"

namespace pfsm {

constexpr int BM = 64, BN = 64, BK = 16, PAD = 1;

template <int EPI, int QL>
__global__ void __launch_bounds__(256)
k_gemm_f64(GemmArgs a)
{
    __shared__ double Ps[BK][BM + PAD];
    __shared__ double Qs[BK][BN + PAD];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int64_t r0 = (int64_t)blockIdx.y * BM, c0 = (int64_t)blockIdx.x * BN;
    if (a.lower_only && c0 > r0 + BM - 1) return;
    int64_t kbeg = 0, kend = a.K;
    if (a.krange) {
        kbeg = a.krange[2 * blockIdx.y];
        kend = a.krange[2 * blockIdx.y + 1];
    }
    double acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) acc[i][j] = 0.0;

    // loader mapping: P tile 64 rows x 16 k: thread -> row t/4, k (t%4)*4 .. +3
    const int pr = threadIdx.x >> 2, pk = (threadIdx.x & 3) * 4;
    // Q tile: K_MAJOR same as P; N_MAJOR: 16 k rows x 64 cols: thread -> k t/16, c (t%16)*4
    const int qk_n = threadIdx.x >> 4, qc_n = (threadIdx.x & 15) * 4;
    double pv[4], qv[4];

    auto load = [&](int64_t k) {
#pragma unroll
        for (int u = 0; u < 4; u++) {
            int64_t row = r0 + pr, kk = k + pk + u;
            pv[u] = (row < a.rows && kk < kend) ? a.P[row * a.ldp + kk] : 0.0;
        }
        if (QL == Q_KMAJOR) {
#pragma unroll
            for (int u = 0; u < 4; u++) {
                int64_t col = c0 + pr, kk = k + pk + u;
                qv[u] = (col < a.cols && kk < kend) ? a.Q[col * a.ldq + kk] : 0.0;
            }
        } else {
#pragma unroll
            for (int u = 0; u < 4; u++) {
                int64_t col = c0 + qc_n + u, kk = k + qk_n;
                qv[u] = (col < a.cols && kk < kend) ? a.Q[kk * a.ldq + col] : 0.0;
            }
        }
    };
    auto stash = [&]() {
#pragma unroll
        for (int u = 0; u < 4; u++) Ps[pk + u][pr] = pv[u];
        if (QL == Q_KMAJOR) {
#pragma unroll
            for (int u = 0; u < 4; u++) Qs[pk + u][pr] = qv[u];
        } else {
#pragma unroll
            for (int u = 0; u < 4; u++) Qs[qk_n][qc_n + u] = qv[u];
        }
    };

    if (kbeg < kend) {
        load(kbeg);
        for (int64_t k = kbeg; k < kend; k += BK) {
            __syncthreads();
            stash();
            __syncthreads();
            if (k + BK < kend) load(k + BK);
#pragma unroll
            for (int kk = 0; kk < BK; kk++) {
                double x[4], y[4];
#pragma unroll
                for (int i = 0; i < 4; i++) x[i] = Ps[kk][ty + 16 * i];
#pragma unroll
                for (int j = 0; j < 4; j++) y[j] = Qs[kk][tx + 16 * j];
#pragma unroll
                for (int i = 0; i < 4; i++)
#pragma unroll
                    for (int j = 0; j < 4; j++) acc[i][j] = fma(x[i], y[j], acc[i][j]);
            }
        }
    }
#pragma unroll
    for (int i = 0; i < 4; i++) {
        const int64_t r = r0 + ty + 16 * i;
        if (r >= a.rows) continue;
#pragma unroll
        for (int j = 0; j < 4; j++) {
            const int64_t c = c0 + tx + 16 * j;
            if (c >= a.cols) continue;
            if (a.lower_only && c > r) continue;
            const int64_t o = r * a.ldc + c;
            if (EPI == EPI_STORE) {
                a.C[o] = acc[i][j];
            } else if (EPI == EPI_SUB) {
                a.C[o] -= acc[i][j];
            } else if (EPI == EPI_FS1) {
                a.C[o] = acc[i][j] - a.eps[r] * a.aux_x[o];
            } else {   // EPI_FS2: C is X
                a.C[o] = a.C[o] - a.alpha[r] * (acc[i][j] - a.eps[r] * a.aux_y[o]);
            }
        }
    }
}

cudaError_t launch_gemm_f64(const GemmArgs &a, int epi, int qlayout, cudaStream_t st)
{
    if (a.rows <= 0 || a.cols <= 0) return cudaSuccess;
    dim3 grid((unsigned)((a.cols + BN - 1) / BN), (unsigned)((a.rows + BM - 1) / BM));
#define PFSM_GEMM_CASE(E, Q) \
    if (epi == E && qlayout == Q) { k_gemm_f64<E, Q><<<grid, 256, 0, st>>>(a); g_launches++; return cudaGetLastError(); }
    PFSM_GEMM_CASE(EPI_STORE, Q_KMAJOR)
    PFSM_GEMM_CASE(EPI_SUB, Q_KMAJOR)
    PFSM_GEMM_CASE(EPI_FS1, Q_KMAJOR)
    PFSM_GEMM_CASE(EPI_FS2, Q_KMAJOR)
    PFSM_GEMM_CASE(EPI_STORE, Q_NMAJOR)
    PFSM_GEMM_CASE(EPI_SUB, Q_NMAJOR)
#undef PFSM_GEMM_CASE
    return cudaErrorInvalidValue;
}

}  // namespace pfsm
