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
// shared memory with a register prefetch of the next K step; skinny products use 32 x 32 tiles.
//
// Epilogues (r = row of C, i.e. the vector index when vectors are stored as rows):
//   EPI_STORE  C = acc
//   EPI_SUB    C = C - acc
//   EPI_FS1    C = acc - eps[r] * X[r, c]                      (Y = (A - eps I) x, Eq. 11)
//   EPI_FS2    X[r, c] = X[r, c] - alpha[r] * (acc - eps[r] * Y[r, c])
//              (x <- x - alpha (A - eps I) y, the second product of Eq. 11, updated in place)
#include "pfsm_internal.cuh"

namespace pfsm {

constexpr int BK = 16, PAD = 1;

// T x T output tile per CTA, (T/4)^2 threads with 4 x 4 outputs each (rows ty + (T/4) i,
// columns tx + (T/4) j); T = 64 (256 threads) for large products, T = 32 (64 threads) for the
// skinny ones of the blocked Cholesky and triangular solve, which otherwise occupy too few SMs.
template <int EPI, int QL, int T>
__global__ void __launch_bounds__((T / 4) * (T / 4))
k_gemm_f64(GemmArgs a)
{
    constexpr int NT = (T / 4) * (T / 4), TS = T / 4;
    constexpr int PER = T * BK / NT;       // operand elements per thread per K step (4 or 8)
    __shared__ double Ps[BK][T + PAD];
    __shared__ double Qs[BK][T + PAD];
    const int tx = threadIdx.x % TS, ty = threadIdx.x / TS;
    const int64_t r0 = (int64_t)blockIdx.y * T, c0 = (int64_t)blockIdx.x * T;
    if (a.lower_only && c0 > r0 + T - 1) return;
    int64_t kbeg = 0, kend = a.K;
    if (a.krange) {                        // only with T = 64 (the K-range granularity)
        kbeg = a.krange[2 * blockIdx.y];
        kend = a.krange[2 * blockIdx.y + 1];
    }
    double acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) acc[i][j] = 0.0;
    double pv[PER], qv[PER];

    // element e = threadIdx.x + u * NT of a tile: K-major tiles (T rows x BK) by (e / BK, e % BK),
    // the N-major Q tile (BK x T) by (e / T, e % T); consecutive threads read consecutive addresses
    auto load = [&](int64_t k) {
#pragma unroll
        for (int u = 0; u < PER; u++) {
            const int e = threadIdx.x + u * NT;
            const int64_t row = r0 + e / BK, kk = k + e % BK;
            pv[u] = (row < a.rows && kk < kend) ? a.P[row * a.ldp + kk] : 0.0;
            if (QL == Q_KMAJOR) {
                const int64_t col = c0 + e / BK;
                qv[u] = (col < a.cols && kk < kend) ? a.Q[col * a.ldq + kk] : 0.0;
            } else {
                const int64_t col = c0 + e % T, k2 = k + e / T;
                qv[u] = (col < a.cols && k2 < kend) ? a.Q[k2 * a.ldq + col] : 0.0;
            }
        }
    };
    auto stash = [&]() {
#pragma unroll
        for (int u = 0; u < PER; u++) {
            const int e = threadIdx.x + u * NT;
            Ps[e % BK][e / BK] = pv[u];
            if (QL == Q_KMAJOR) Qs[e % BK][e / BK] = qv[u];
            else Qs[e / T][e % T] = qv[u];
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
                for (int i = 0; i < 4; i++) x[i] = Ps[kk][ty + TS * i];
#pragma unroll
                for (int j = 0; j < 4; j++) y[j] = Qs[kk][tx + TS * j];
#pragma unroll
                for (int i = 0; i < 4; i++)
#pragma unroll
                    for (int j = 0; j < 4; j++) acc[i][j] = fma(x[i], y[j], acc[i][j]);
            }
        }
    }
#pragma unroll
    for (int i = 0; i < 4; i++) {
        const int64_t r = r0 + ty + TS * i;
        if (r >= a.rows) continue;
#pragma unroll
        for (int j = 0; j < 4; j++) {
            const int64_t c = c0 + tx + TS * j;
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

template <int T>
static cudaError_t launch_tile(const GemmArgs &a, int epi, int qlayout, cudaStream_t st)
{
    dim3 grid((unsigned)((a.cols + T - 1) / T), (unsigned)((a.rows + T - 1) / T));
    constexpr int NT = (T / 4) * (T / 4);
#define PFSM_GEMM_CASE(E, Q) \
    if (epi == E && qlayout == Q) { k_gemm_f64<E, Q, T><<<grid, NT, 0, st>>>(a); g_launches++; return cudaGetLastError(); }
    PFSM_GEMM_CASE(EPI_STORE, Q_KMAJOR)
    PFSM_GEMM_CASE(EPI_SUB, Q_KMAJOR)
    PFSM_GEMM_CASE(EPI_FS1, Q_KMAJOR)
    PFSM_GEMM_CASE(EPI_FS2, Q_KMAJOR)
    PFSM_GEMM_CASE(EPI_STORE, Q_NMAJOR)
    PFSM_GEMM_CASE(EPI_SUB, Q_NMAJOR)
#undef PFSM_GEMM_CASE
    return cudaErrorInvalidValue;
}

cudaError_t launch_gemm_f64(const GemmArgs &a, int epi, int qlayout, cudaStream_t st)
{
    if (a.rows <= 0 || a.cols <= 0) return cudaSuccess;
    // 64-wide tiles unless that leaves most SMs idle (skinny products); the K-range table of
    // the first Eq. 11 product is per 64-row tile
    const int64_t tiles64 = ((a.cols + 63) / 64) * ((a.rows + 63) / 64);
    if (a.krange || tiles64 >= 148) return launch_tile<64>(a, epi, qlayout, st);
    return launch_tile<32>(a, epi, qlayout, st);
}

}  // namespace pfsm
