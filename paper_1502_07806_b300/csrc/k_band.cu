// Two-stage reduction of large windows to tridiagonal form (mixed forms; Section II's submatrix
// eigensolves, whose cost the paper puts at the cube of the window width).
//
// A window of width M (2068 for the silicon-vacancy-like matrix, 1440 for the metal) does not fit
// a thread-block cluster's shared memory, and the one-stage Householder reduction then streams the
// whole trailing matrix through the FP64 pipe at every one of its M steps (2 M^3 FP64 operations,
// about 2 s for 36 such windows). Here the reduction is split as in the two-stage symmetric
// eigensolvers (Bischof, Lang and Sun's successive band reduction; the dense-to-band stage as in
// LAPACK's blocked reduction, Golub & Van Loan Sec. 5.1.7 and 8.3.1):
//
//  1. dense -> band of half-width KB = 32, one panel of KB columns at a time:
//       k_band_panel   Householder QR of the panel B[r0:M, c:c+KB] (r0 = c + KB) in a cluster of
//                      CTAs (rows in shared memory, partial sums exchanged through distributed
//                      shared memory), unit reflectors v_t (beta = 2) with T of the compact-WY
//                      form I - V T V^T (LAPACK's larft recurrence), R written into the band;
//       Y = A22 V      FP64-accurate digit product on the tensor cores (k_gemm_oz.cu) of the
//                      off-diagonal part, the diagonal part added exactly in FP64;
//       k_band_w/u/z   W = Y T, U = T^T (V^T W), Z = W - V U / 2 on the FP64 pipe;
//       A22 -= V Z^T + Z V^T   digit product (K = 64: the strip kernel, a CTA keeping its rows'
//                      digits and walking a strip of column tiles), subtracted into the window.
//     The O(M^3) work of this stage runs on the tensor cores at FP64 accuracy.
//  2. band -> tridiagonal by bulge chasing (k_band_chase, FP64): sweep s annihilates column s below
//     its subdiagonal with one reflector on rows s+1 .. s+KB and then chases the bulge down the
//     band, each task (s, i) annihilating the first column of the bulge the previous one created
//     with a reflector on rows s+1+i KB .. s+(i+1) KB; the rest of each bulge is removed by the
//     following sweeps. Tasks (s, i) run at time 3 s + i, so every time step's tasks touch disjoint
//     band columns; one cluster per window, one warp per task, a cluster barrier per time step.
//  3. the tridiagonal's eigenpairs as before (k_bisect, k_inverse_iter);
//  4. y = Q1 Q2 z: Q2's reflectors applied to the eigenvectors z in float-float arithmetic on the
//     FP32 pipe (k_band_bt2),
//     then Q1 panel by panel, Yr <- Yr - (Yr V T^T) V^T with two digit products per panel
//     (k_band_bt1_u forms X T^T), and the start-vector rules (k_bt_wy.cu).
// The FP64 form keeps the one-stage reduction (no tensor cores).
#include <cooperative_groups.h>
#include <algorithm>

#include "fp64_util.cuh"
#include "pfsm_internal.cuh"

namespace cg = cooperative_groups;

namespace pfsm {

namespace {

constexpr int KB = kBand;
constexpr int kPanelThreads = 256;
constexpr int kChunk = 64;                 // rows per CTA of the W / Z kernels
constexpr int kBtWarps = 8;                // k_band_bt2: warps per CTA
constexpr int kBtVpw = 16;                 // k_band_bt2: vectors per warp (2 lanes each; 4 measured slower)
constexpr int kStrip = 8;                  // column tiles per CTA of the small-K digit products

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

}  // namespace

// Stage-1 panels of a window of width M: panel p (columns p KB .. p KB + KB - 1) exists while its
// trailing rows r0 = (p + 1) KB leave at least two rows, r0 <= M - 2.
__host__ __device__ int band_panels(int M) { return M >= KB + 2 ? (M - 2 - KB) / KB + 1 : 0; }

// ---- set-up: the windows into their work matrices -------------------------------------------
// Grid (ceil(Mmax / 8), nb), 256 threads: warp per row i of window b, G[i][j] = A[s + i][s + j].
// The reflector rows no panel writes (k in [panels * KB, M - 2)) are zeroed with tau = 0.
__global__ void __launch_bounds__(256)
k_band_copy(const double *__restrict__ A, int64_t N, const int32_t *__restrict__ plan, int nb, int Mmax,
            double *__restrict__ G, double *__restrict__ refl, double *__restrict__ tau)
{
    const int b = blockIdx.y;
    const int64_t s0 = plan[2 * nb + b];
    const int M = plan[3 * nb + b];
    const int lane = threadIdx.x & 31;
    const int i = blockIdx.x * 8 + (threadIdx.x >> 5);
    if (i < M) {
        const double *src = A + (s0 + i) * N + s0;
        double *dst = G + ((size_t)b * Mmax + i) * Mmax;
        for (int j = lane; j < M; j += 32) dst[j] = src[j];
    }
    const int k = band_panels(M) * KB + i;      // one uncovered reflector row per warp
    if (i < KB + 2 && k < M - 2) {
        double *rr = refl + ((size_t)b * Mmax + k) * Mmax;
        for (int j = k + 1 + lane; j < M; j += 32) rr[j] = 0.0;
        if (lane == 0) tau[(size_t)b * Mmax + k] = 0.0;
    }
}

// ---- stage 1: panel QR --------------------------------------------------------------------------
// Cluster of CL CTAs per window (grid nb * CL), 256 threads. The panel's n = M - r0 rows are split
// into CL contiguous chunks held in shared memory (rows x (KB + 1) doubles). Per column t: (A)
// partial sums of the column's tail and its head entry, pulled by warp 0 of every CTA after a
// cluster barrier, which forms the reflector's scalars once for its CTA; (B) partial dot products
// of the unit reflector with the later columns, pulled after a second barrier, then the rank-1
// update of the owned rows. Every CTA forms the same scalars from the same partial sums in the same
// order. The dot products and the update touch only the 31 - t later columns: a warp instruction
// covers 32 / g rows of g >= 31 - t columns (g = 32, 16, 8 or 4), so the FP64 pipe, the kernel's
// bound, does not issue for idle columns. Outputs: reflector rows refl[c + t] (zero outside
// rows r0 + t .. M-1), tau = 2 (0 for a column whose tail is already zero), T (KB x KB, upper),
// R into the band of G (rows r0 .. r0 + KB - 1, columns c .. c + KB - 1), and extp[b] = M when the
// window has this panel, else 0 (the later kernels of this panel read their extent from it).
__global__ void __launch_bounds__(kPanelThreads, 1)
k_band_panel(const int32_t *__restrict__ plan, int nb, int Mmax, int c, int rpc_cap, double *__restrict__ G,
             double *__restrict__ refl, double *__restrict__ tau, double *__restrict__ Tb, int32_t *__restrict__ extp)
{
    cg::cluster_group cluster = cg::this_cluster();
    const int CL = (int)cluster.num_blocks();
    const int rank = (int)cluster.block_rank();
    const int b = blockIdx.x / CL;
    const int M = plan[3 * nb + b];
    const int r0 = c + KB;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int NW = kPanelThreads / 32;
    if (r0 > M - 2) {                                  // no panel here (uniform over the cluster)
        if (rank == 0 && tid == 0) extp[b] = 0;
        return;
    }
    const int n = M - r0;
    const int rpc = (n + CL - 1) / CL;
    const int i0 = rank * rpc, i1 = min(n, i0 + rpc), nown = max(0, i1 - i0);
    constexpr int LD = KB + 1;
    extern __shared__ double sm[];
    double *P = sm;                                    // rpc_cap x LD: owned rows of the panel
    double *red = P + (size_t)rpc_cap * LD;            // 32: per-warp partial sums
    double *hx = red + 32;                             // [0] partial tail^2, [1] head entry (owner)
    double *wp = hx + 2;                               // KB partial dots of the current column step
    double *wr = wp + KB;                              // NW x KB per-warp partial dots
    double *alph = wr + NW * KB;                       // KB: R's diagonal (alpha_t)
    double *bet = alph + KB;                           // KB: beta_t (2 or 0)
    double *Gp = bet + KB;                             // KB x KB partial V^T V (own rows, p < q)
    double *Tm = Gp + KB * KB;                         // KB x KB: T (rank 0)
    double *Gs = Tm + KB * KB;                         // KB x KB: V^T V (rank 0)
    double *sc = Gs + KB * KB;                         // 4: the column's 1/||v||, v_0, beta
    double *wsum = sc + 4;                             // KB: -2 w_j of the column step
    double *Gb = G + (size_t)b * Mmax * Mmax;

    for (int il = warp; il < nown; il += NW) P[il * LD + lane] = Gb[(size_t)(r0 + i0 + il) * Mmax + c + lane];
    const int tmax = min(KB, n);
    for (int t = tid; t < KB; t += blockDim.x) { alph[t] = 0.0; bet[t] = 0.0; }
    __syncthreads();
    cluster.sync();                                    // every CTA is running before remote access

    for (int t = 0; t < tmax; t++) {
        // (A) tail of column t (rows t+1 .. n-1) and its head entry (row t)
        double part = 0.0;
        for (int il = tid; il < nown; il += blockDim.x)
            if (i0 + il > t) part = fma(P[il * LD + t], P[il * LD + t], part);
        part = warp_sum(part);
        if (lane == 0) red[warp] = part;
        const int owner = t / rpc;
        __syncthreads();
        if (tid == 0) {
            double s2 = 0.0;
            for (int q = 0; q < NW; q++) s2 += red[q];
            hx[0] = s2;
            hx[1] = (owner == rank) ? P[(t - i0) * LD + t] : 0.0;
        }
        cluster.sync();
        if (warp == 0) {                               // the reflector's scalars, once per CTA
            double tail2 = (lane < CL) ? cluster.map_shared_rank(hx, lane)[0] : 0.0;
            tail2 = warp_sum(tail2);                   // the same order in every CTA
            if (lane == 0) {
                const double x0 = cluster.map_shared_rank(hx, owner)[1];
                double inv = 0.0, v0 = 0.0, alpha = x0, beta = 0.0;
                if (tail2 != 0.0) {
                    const double nn = fma(x0, x0, tail2);
                    const double xn = nn * fast_rsqrt(nn);
                    alpha = (x0 >= 0.0) ? -xn : xn;
                    v0 = x0 - alpha;
                    inv = fast_rsqrt(fma(v0, v0, tail2));
                    beta = 2.0;
                }
                sc[0] = inv;
                sc[1] = v0;
                sc[2] = beta;
                alph[t] = alpha;
                bet[t] = beta;
            }
        }
        __syncthreads();
        const double inv = sc[0], v0 = sc[1], beta = sc[2];
        // the unit reflector into column t of the owned rows >= t (all zero when beta = 0)
        for (int il = tid; il < nown; il += blockDim.x) {
            const int i = i0 + il;
            if (i == t) P[il * LD + t] = v0 * inv;
            else if (i > t) P[il * LD + t] *= inv;
        }
        __syncthreads();
        // (B) partial w_j = v . column j over the owned rows >= t, for the nc = KB - 1 - t later
        // columns: lane -> column t + 1 + (lane mod g), row offset lane / g within the warp's rows
        const int nc = KB - 1 - t;
        const int lg = nc > 16 ? 5 : nc > 8 ? 4 : nc > 4 ? 3 : 2;
        const int g = 1 << lg, rp = 32 >> lg;
        const int j = t + 1 + (lane & (g - 1)), ro = lane >> lg;
        const bool jok = j < KB;
        if (beta != 0.0) {
            double acc = 0.0;
            if (jok)
                for (int il = warp * rp + ro; il < nown; il += NW * rp)
                    if (i0 + il >= t) acc = fma(P[il * LD + t], P[il * LD + j], acc);
            for (int o = g; o < 32; o <<= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
            if (ro == 0 && jok) wr[warp * KB + j] = acc;
            __syncthreads();
            if (warp == 0) {
                double s2 = 0.0;
                if (lane > t)
                    for (int q = 0; q < NW; q++) s2 += wr[q * KB + lane];
                wp[lane] = s2;
            }
        }
        cluster.sync();
        if (beta != 0.0) {
            if (warp == 0) {
                double wj = 0.0;
                if (lane > t)
                    for (int r = 0; r < CL; r++) wj += cluster.map_shared_rank(wp, r)[lane];
                wsum[lane] = -2.0 * wj;
            }
            __syncthreads();
            if (jok) {
                const double m2w = wsum[j];
                for (int il = warp * rp + ro; il < nown; il += NW * rp)
                    if (i0 + il >= t) P[il * LD + j] = fma(m2w, P[il * LD + t], P[il * LD + j]);
            }
        }
        __syncthreads();
    }
    // reflector columns: V[i][t] = P[i][t] for i >= t (the entries above are R's)
    auto vij = [&](int il, int t) -> double { return (t < tmax && i0 + il >= t) ? P[il * LD + t] : 0.0; };
    // partial V^T V over the owned rows, strictly upper entries only (T needs no others): the
    // 496 pairs p < q, two per thread
    {
        constexpr int NPAIR = KB * (KB - 1) / 2;
        int pp[2], qq[2];
#pragma unroll
        for (int k = 0; k < 2; k++) {
            int e = tid + k * kPanelThreads, pr = 0;
            if (e >= NPAIR) e = 0;
            while (e >= KB - 1 - pr) { e -= KB - 1 - pr; pr++; }
            pp[k] = pr;
            qq[k] = pr + 1 + e;
        }
        const bool ok1 = tid + kPanelThreads < NPAIR;
        double g0 = 0.0, g1 = 0.0;
        for (int il = 0; il < nown; il++) {
            g0 = fma(vij(il, pp[0]), vij(il, qq[0]), g0);
            if (ok1) g1 = fma(vij(il, pp[1]), vij(il, qq[1]), g1);
        }
        if (tid < NPAIR) Gp[pp[0] * KB + qq[0]] = g0;
        if (ok1) Gp[pp[1] * KB + qq[1]] = g1;
    }
    // outputs that need only this CTA's rows: reflector rows (zero above row t), R's rows
    double *bref = refl + (size_t)b * Mmax * Mmax;
    for (int t = 0; t < KB; t++)
        for (int il = tid; il < nown; il += blockDim.x)
            bref[(size_t)(c + t) * Mmax + r0 + i0 + il] = vij(il, t);
    for (int il = warp; il < nown; il += NW) {
        const int i = i0 + il;                         // R row i < KB: entries j >= i of row r0 + i
        if (i < KB && lane >= i) Gb[(size_t)(r0 + i) * Mmax + c + lane] = (lane == i) ? alph[i] : P[il * LD + lane];
    }
    cluster.sync();
    if (rank == 0) {
        for (int e = tid; e < KB * KB; e += blockDim.x) {
            const int pr = e / KB, q = e % KB;
            double s2 = 0.0;
            if (pr < q)
                for (int r = 0; r < CL; r++) s2 += cluster.map_shared_rank(Gp, r)[e];
            Gs[e] = s2;
        }
        // reflector rows' entries between the row index and the reflector's first row are zero
        for (int t = warp; t < KB; t += NW) {
            double *rr = bref + (size_t)(c + t) * Mmax;
            for (int jj = c + t + 1 + lane; jj < r0; jj += 32) rr[jj] = 0.0;
            if (lane == 0) tau[(size_t)b * Mmax + c + t] = bet[t];
        }
        if (tid == 0) extp[b] = M;
        __syncthreads();
        // T (larft, forward, columnwise): T[t][t] = beta_t, T[0:t, t] = -beta_t T[0:t, 0:t] G[0:t, t]
        if (warp == 0) {
            for (int q = 0; q < KB; q++) Tm[q * KB + lane] = 0.0;
            __syncwarp();
            for (int t = 0; t < KB; t++) {
                double s2 = 0.0;
                if (lane < t)
                    for (int pq = lane; pq < t; pq++) s2 = fma(Tm[lane * KB + pq], Gs[pq * KB + t], s2);
                __syncwarp();
                if (lane < t) Tm[lane * KB + t] = -bet[t] * s2;
                if (lane == t) Tm[t * KB + t] = bet[t];
                __syncwarp();
            }
            double *Tbb = Tb + (size_t)b * KB * KB;
            for (int q = 0; q < KB; q++) Tbb[q * KB + lane] = Tm[q * KB + lane];
        }
    }
    cluster.sync();                                    // remote reads done before any CTA exits
}

// ---- stage 1: W = Y T (in place) and the chunk partials of V^T W ---------------------------------
// Grid (ceil((Mmax - r0) / kChunk), nb), 256 threads. Rows r0 + bx kChunk .. of window b.
__global__ void __launch_bounds__(256)
k_band_w(const int32_t *__restrict__ extp, int Mmax, int c, const double *__restrict__ refl,
         const double *__restrict__ Tb, double *__restrict__ Y, double *__restrict__ Xp, int nchunk)
{
    const int b = blockIdx.y, bx = blockIdx.x;
    const int r0 = c + KB;
    const int n = max(0, extp[b] - r0);
    const int ib = bx * kChunk;
    if (ib >= n) return;
    const int rows = min(kChunk, n - ib);
    __shared__ double T[KB][KB + 1], Ys[kChunk][KB + 1], Vs[kChunk][KB + 1];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const double *Tbb = Tb + (size_t)b * KB * KB;
    for (int e = tid; e < KB * KB; e += 256) T[e / KB][e % KB] = Tbb[e];
    double *Yb = Y + ((size_t)b * Mmax + r0 + ib) * KB;
    for (int e = tid; e < kChunk * KB; e += 256) {
        const int il = e / KB, q = e % KB;
        Ys[il][q] = (il < rows) ? Yb[(size_t)il * KB + q] : 0.0;
    }
    const double *bref = refl + (size_t)b * Mmax * Mmax;
    for (int p = warp; p < KB; p += 8)
        for (int il = lane; il < kChunk; il += 32)
            Vs[il][p] = (il < rows) ? bref[(size_t)(c + p) * Mmax + r0 + ib + il] : 0.0;
    __syncthreads();
    // W[il][q] = sum_{p <= q} Y[il][p] T[p][q]: thread -> row il = tid / 4, columns q = (tid % 4) + 4 j
    {
        const int il = tid >> 2, q0 = tid & 3;
        double w[8];
#pragma unroll
        for (int j = 0; j < 8; j++) {
            const int q = q0 + 4 * j;
            double s = 0.0;
            for (int p = 0; p <= q; p++) s = fma(Ys[il][p], T[p][q], s);
            w[j] = s;
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < 8; j++) Ys[il][q0 + 4 * j] = w[j];
    }
    __syncthreads();
    for (int e = tid; e < rows * KB; e += 256) Yb[e] = Ys[e / KB][e % KB];
    // partial X[p][q] = sum_il V[il][p] W[il][q]: thread -> p = tid / 8, q = (tid % 8) + 8 j
    {
        const int p = tid >> 3, q0 = tid & 7;
        double x[4] = {0.0, 0.0, 0.0, 0.0};
        for (int il = 0; il < rows; il++) {
            const double v = Vs[il][p];
#pragma unroll
            for (int j = 0; j < 4; j++) x[j] = fma(v, Ys[il][q0 + 8 * j], x[j]);
        }
        double *xo = Xp + ((size_t)b * nchunk + bx) * KB * KB;
#pragma unroll
        for (int j = 0; j < 4; j++) xo[p * KB + q0 + 8 * j] = x[j];
    }
}

// U = T^T X with X = sum over the window's chunks of the partials (fixed order). Grid nb, 256.
__global__ void __launch_bounds__(256)
k_band_u(const int32_t *__restrict__ extp, int c, const double *__restrict__ Tb, const double *__restrict__ Xp,
         int nchunk, double *__restrict__ U)
{
    const int b = blockIdx.x;
    const int n = max(0, extp[b] - (c + KB));
    if (n == 0) return;
    const int nch = (n + kChunk - 1) / kChunk;
    __shared__ double X[KB][KB + 1], T[KB][KB + 1];
    const double *Tbb = Tb + (size_t)b * KB * KB;
    for (int e = threadIdx.x; e < KB * KB; e += 256) {
        double s = 0.0;
        for (int ch = 0; ch < nch; ch++) s += Xp[((size_t)b * nchunk + ch) * KB * KB + e];
        X[e / KB][e % KB] = s;
        T[e / KB][e % KB] = Tbb[e];
    }
    __syncthreads();
    double *Ub = U + (size_t)b * KB * KB;
    for (int e = threadIdx.x; e < KB * KB; e += 256) {
        const int p = e / KB, q = e % KB;
        double s = 0.0;
        for (int r = 0; r <= p; r++) s = fma(T[r][p], X[r][q], s);
        Ub[e] = s;
    }
}

// Z = W - V U / 2 and the operands of the trailing update: row r0 + i of window b in VW = [v z],
// WV = [z v] (rows b * Mmax + r0 + i, 2 KB entries); the reflectors' row r0 + i also into Vrows
// (kept for the back-transformation). Grid (ceil((Mmax - r0) / kChunk), nb), 256.
__global__ void __launch_bounds__(256)
k_band_z(const int32_t *__restrict__ extp, int Mmax, int c, const double *__restrict__ refl,
         const double *__restrict__ Y, const double *__restrict__ U, double *__restrict__ VW, double *__restrict__ WV,
         double *__restrict__ Vrows)
{
    const int b = blockIdx.y, bx = blockIdx.x;
    const int r0 = c + KB;
    const int n = max(0, extp[b] - r0);
    const int ib = bx * kChunk;
    if (ib >= n) return;
    const int rows = min(kChunk, n - ib);
    __shared__ double Us[KB][KB + 1], Vs[kChunk][KB + 1];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const double *Ub = U + (size_t)b * KB * KB;
    for (int e = tid; e < KB * KB; e += 256) Us[e / KB][e % KB] = Ub[e];
    const double *bref = refl + (size_t)b * Mmax * Mmax;
    for (int p = warp; p < KB; p += 8)
        for (int il = lane; il < kChunk; il += 32)
            Vs[il][p] = (il < rows) ? bref[(size_t)(c + p) * Mmax + r0 + ib + il] : 0.0;
    __syncthreads();
    const double *Wb = Y + ((size_t)b * Mmax + r0 + ib) * KB;
    for (int e = tid; e < rows * KB; e += 256) {
        const int il = e / KB, q = e % KB;
        double s = 0.0;
        for (int p = 0; p < KB; p++) s = fma(Vs[il][p], Us[p][q], s);
        const double z = fma(-0.5, s, Wb[e]);
        const size_t row = (size_t)b * Mmax + r0 + ib + il;
        VW[row * 2 * KB + q] = Vs[il][q];
        VW[row * 2 * KB + KB + q] = z;
        WV[row * 2 * KB + q] = z;
        WV[row * 2 * KB + KB + q] = Vs[il][q];
        Vrows[row * KB + q] = Vs[il][q];
    }
}

// ---- stage 2: the band into band storage --------------------------------------------------------
// Bw[b] holds (Mmax + 2 KB) columns of 2 KB entries: Bw[b][j][d] = B[j + d][j] (lower band of
// half-width 2 KB - 1, room for the bulges). Grid (ceil((Mmax + 2 KB) / 8), nb), 256 threads.
__global__ void __launch_bounds__(256)
k_band_extract(const int32_t *__restrict__ plan, int nb, int Mmax, const double *__restrict__ G,
               double *__restrict__ Bw)
{
    const int b = blockIdx.y;
    const int M = plan[3 * nb + b];
    const int j = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (j >= Mmax + 2 * KB) return;
    const double *Gb = G + (size_t)b * Mmax * Mmax;
    double *col = Bw + ((size_t)b * (Mmax + 2 * KB) + j) * 2 * KB;
    for (int d = lane; d < 2 * KB; d += 32)
        col[d] = (j < M && d <= KB && j + d < M) ? Gb[(size_t)(j + d) * Mmax + j] : 0.0;
}

// ---- stage 2: bulge chasing -----------------------------------------------------------------------
// One task (s, i) by one warp (see the file comment). Rows R = [a, a + L), a = s + 1 + i KB,
// L = min(KB, M - a); the column it annihilates, col = s (i = 0) or a - KB; the blocks it touches:
// left (rows R, columns col+1 .. a-1, only for i >= 1), diagonal (R x R, lower triangle stored) and
// below (rows a + L .. a + L + KB - 1, columns R). Every block is loaded with all its loads in
// flight (registers first, then the warp's shared-memory tile S where a transpose is needed),
// updated, and stored back. The reflector goes to refl2 (KB entries, zero past L) and tau2.
// part: 2 = the whole task; 0 = the reflector, the annihilated column and the diagonal block; 1 =
// the left and below blocks. Parts 0 and 1 of one task run on two warps of one CTA (different
// sub-partitions, so their FP64 instruction streams issue side by side), each forming the same
// reflector from the same column; they meet at named barrier bar_id once both have read the column,
// after which part 0 overwrites it.
__device__ __forceinline__ void chase_task(double *__restrict__ B, int M, int s, int i, double *__restrict__ r2,
                                           double *__restrict__ t2, double *vsh, double *wsh, double (*S)[KB + 1],
                                           int lane, int part, int bar_id)
{
    auto at = [&](int r, int cc) -> double & { return B[(size_t)cc * (2 * KB) + (r - cc)]; };
    const int a = s + 1 + i * KB;
    const int L = min(KB, M - a);
    const int col = (i == 0) ? s : a - KB;
    const double x = (lane < L) ? at(a + lane, col) : 0.0;
    const double tail2 = warp_sum(lane >= 1 ? x * x : 0.0);
    const double x0 = __shfl_sync(0xffffffffu, x, 0);
    double beta = 0.0, alpha = x0, v = 0.0;
    if (tail2 != 0.0) {
        const double nn = fma(x0, x0, tail2);
        const double xn = nn * fast_rsqrt(nn);
        alpha = (x0 >= 0.0) ? -xn : xn;
        const double v0 = x0 - alpha;
        beta = 2.0 * fast_rcp(fma(v0, v0, tail2));
        v = (lane == 0) ? v0 : x;
    }
    if (part != 1) {
        r2[lane] = v;
        if (lane == 0) *t2 = beta;
    }
    if (part != 2) asm volatile("bar.sync %0, 64;" ::"r"(bar_id) : "memory");
    if (beta == 0.0) return;
    if (part != 1 && lane < L) at(a + lane, col) = (lane == 0) ? alpha : 0.0;
    vsh[lane] = v;
    __syncwarp();
    double tmp[KB];
    // left block: H from the left on columns col+1 .. a-1 (the rest of the previous bulge); lane =
    // row for the loads and stores, lane = column for the arithmetic
    if (part != 0 && i >= 1) {
#pragma unroll
        for (int q = 0; q < KB - 1; q++) tmp[q] = (lane < L) ? at(a + lane, col + 1 + q) : 0.0;
#pragma unroll
        for (int q = 0; q < KB - 1; q++) S[q][lane] = tmp[q];
        __syncwarp();
        if (lane < KB - 1) {
            double w0 = 0.0, w1 = 0.0, w2 = 0.0, w3 = 0.0;     // four chains of dependent FMAs
#pragma unroll
            for (int r = 0; r < KB; r += 4) {
                w0 = fma(vsh[r], S[lane][r], w0);
                w1 = fma(vsh[r + 1], S[lane][r + 1], w1);
                w2 = fma(vsh[r + 2], S[lane][r + 2], w2);
                w3 = fma(vsh[r + 3], S[lane][r + 3], w3);
            }
            const double w = beta * ((w0 + w1) + (w2 + w3));
#pragma unroll
            for (int r = 0; r < KB; r++) S[lane][r] = fma(-w, vsh[r], S[lane][r]);
        }
        __syncwarp();
#pragma unroll
        for (int q = 0; q < KB - 1; q++) tmp[q] = S[q][lane];
#pragma unroll
        for (int q = 0; q < KB - 1; q++)
            if (lane < L) at(a + lane, col + 1 + q) = tmp[q];
        __syncwarp();
    }
    // diagonal block: D <- H D H = D - v w^T - w v^T, p = beta D v, w = p - (beta / 2)(v.p) v; column
    // c of the lower triangle in S[c][r], r >= c (lane = row)
    if (part != 1) {
#pragma unroll
    for (int c = 0; c < KB; c++) tmp[c] = (c <= lane && lane < L) ? at(a + lane, a + c) : 0.0;
#pragma unroll
    for (int c = 0; c < KB; c++) S[c][lane] = tmp[c];
    __syncwarp();
    double p0 = 0.0, p1 = 0.0, p2 = 0.0, p3 = 0.0;
#pragma unroll
    for (int c = 0; c < KB; c += 4) {
        p0 = fma((c <= lane) ? S[c][lane] : S[lane][c], vsh[c], p0);
        p1 = fma((c + 1 <= lane) ? S[c + 1][lane] : S[lane][c + 1], vsh[c + 1], p1);
        p2 = fma((c + 2 <= lane) ? S[c + 2][lane] : S[lane][c + 2], vsh[c + 2], p2);
        p3 = fma((c + 3 <= lane) ? S[c + 3][lane] : S[lane][c + 3], vsh[c + 3], p3);
    }
    const double p = beta * ((p0 + p1) + (p2 + p3));
    const double vp = warp_sum(v * p);
    const double w = fma(-0.5 * beta * vp, v, p);
    wsh[lane] = w;
    __syncwarp();
    // the 528 lower-triangle entries, 17 per lane: lanes l and l + 16 share rows p = l mod 16 and
    // 31 - p (p + 1 and 32 - p entries), so no FP64 instruction issues for an empty row slot
    {
        const int pr = lane & 15, k0 = 17 * (lane >> 4);
#pragma unroll
        for (int jj = 0; jj < 17; jj++) {
            const int k = k0 + jj;
            if (k <= KB) {
                const int r = (k <= pr) ? pr : KB - 1 - pr;
                const int c = (k <= pr) ? k : k - pr - 1;
                S[c][r] = fma(-vsh[r], wsh[c], fma(-wsh[r], vsh[c], S[c][r]));
            }
        }
    }
    __syncwarp();
#pragma unroll
    for (int c = 0; c < KB; c++)
        if (c <= lane && lane < L) at(a + lane, a + c) = S[c][lane];
    }
    if (part == 0) return;
    // below: rows e .. e + LB - 1 (lane = row, in registers), H from the right (the next bulge)
    const int e = a + L;
    const int LB = min(KB, M - e);
#pragma unroll
    for (int c = 0; c < KB; c++) tmp[c] = (lane < LB && c < L) ? at(e + lane, a + c) : 0.0;
    double u0 = 0.0, u1 = 0.0, u2 = 0.0, u3 = 0.0;
#pragma unroll
    for (int c = 0; c < KB; c += 4) {
        u0 = fma(tmp[c], vsh[c], u0);
        u1 = fma(tmp[c + 1], vsh[c + 1], u1);
        u2 = fma(tmp[c + 2], vsh[c + 2], u2);
        u3 = fma(tmp[c + 3], vsh[c + 3], u3);
    }
    const double u = beta * ((u0 + u1) + (u2 + u3));
#pragma unroll
    for (int c = 0; c < KB; c++)
        if (lane < LB && c < L) at(e + lane, a + c) = fma(-u, vsh[c], tmp[c]);
    __syncwarp();
}

// Cluster of CL CTAs per window (grid nb * CL), NW warps each; task (s, i) at time step 3 s + i; a
// cluster barrier ends every time step. Sweeps before s_pair: warp g of the window runs the
// sweeps s = g (mod CL NW), one warp per task (needs 3 CL NW > the tasks of sweep 0 so that a
// warp's consecutive sweeps never overlap in time). From s_pair on (at most 3 P tasks per sweep,
// P = CL NW / 2) warp pair q (warps 2j, 2j + 1 of CTA r, q = r + CL j) runs the sweeps s_pair + q
// (mod P), one task split over the pair: a task's time is its warp's FP64 instruction count (one
// per 64 cycles per sub-partition), and in these later steps half the warps had no task. Finally
// td/te of the tridiagonal.
// Dynamic shared memory: per warp a KB x (KB + 1) tile and the reflector and w vectors.
__global__ void __launch_bounds__(32 * kChaseWarps, 1)
k_band_chase(const int32_t *__restrict__ plan, int nb, int Mmax, int NT, double *__restrict__ Bw,
             double *__restrict__ refl2, double *__restrict__ tau2, double *__restrict__ td, double *__restrict__ te)
{
    cg::cluster_group cluster = cg::this_cluster();
    const int CL = (int)cluster.num_blocks();
    const int rank = (int)cluster.block_rank();
    const int b = blockIdx.x / CL;
    const int M = plan[3 * nb + b];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // consecutive sweeps (active together) go to different CTAs and sub-partitions
    const int W = CL * kChaseWarps, g = warp * CL + rank;
    extern __shared__ double csm[];
    double(*S)[KB + 1] = reinterpret_cast<double(*)[KB + 1]>(csm + (size_t)warp * (KB * (KB + 1) + 2 * KB));
    double *vsh = csm + (size_t)warp * (KB * (KB + 1) + 2 * KB) + KB * (KB + 1);
    double *wsh = vsh + KB;
    double *B = Bw + (size_t)b * (Mmax + 2 * KB) * 2 * KB;
    const int Sw = M - 2;                              // sweeps 0 .. M-3
    if (Sw > 0) {
        const int nt0 = (M - 2 + KB - 1) / KB;         // tasks of sweep 0
        const int tend = 3 * (Sw - 1) + nt0;
        // sweeps from s_pair on have at most 3 P tasks (P = CL NW / 2 warp pairs), so each can go
        // to a pair of warps with a pair's consecutive sweeps still apart in time; earlier sweeps
        // take one warp per task (the first steps have more tasks than warp pairs)
        const int P = W / 2;
        const int s_pair = max(0, M - 2 - 3 * P * KB);
        const int q = rank + CL * (warp >> 1), part = warp & 1, bar_id = 1 + (warp >> 1);
        for (int t = 0; t < tend; t++) {
            const int smax = t / 3;
            if (smax >= g) {
                const int s = g + ((smax - g) / W) * W;
                const int i = t - 3 * s;
                if (s < min(Sw, s_pair) && i < (M - 2 - s + KB - 1) / KB) {
                    const size_t slot = ((size_t)b * Mmax + s) * NT + i;
                    chase_task(B, M, s, i, refl2 + slot * KB, tau2 + slot, vsh, wsh, S, lane, 2, 0);
                }
            }
            if (smax - s_pair >= q) {
                const int s = s_pair + q + ((smax - s_pair - q) / P) * P;
                const int i = t - 3 * s;
                if (s < Sw && i < (M - 2 - s + KB - 1) / KB) {
                    const size_t slot = ((size_t)b * Mmax + s) * NT + i;
                    chase_task(B, M, s, i, refl2 + slot * KB, tau2 + slot, vsh, wsh, S, lane, part, bar_id);
                }
            }
            // the barrier's release / acquire at cluster scope orders this step's band writes
            // (global memory) before the next step's reads by every CTA of the cluster
            cluster.sync();
        }
    }
    double *btd = td + (size_t)b * Mmax, *bte = te + (size_t)b * Mmax;
    for (int j = rank * blockDim.x + threadIdx.x; j < M; j += CL * blockDim.x) {
        btd[j] = B[(size_t)j * 2 * KB];
        bte[j] = (j + 1 < M) ? B[(size_t)j * 2 * KB + 1] : 0.0;
    }
}

// ---- back-transformation of stage 2: y = Q2 z ----------------------------------------------------
// About 2.4e6 reflectors of 32 entries per solve touch the 252 eigenvectors of each window: 2 M^2 m
// FMAs per window, 65 ms on the FP64 pipe at its peak. They are applied in float-float arithmetic
// on the FP32 pipe (64 times the FP64 rate): a value is the unevaluated sum hi + lo of two floats
// (48 significant bits), products split exactly by FMA (Dekker / Knuth two-product and two-sum,
// as in the double-float arithmetic of Hida, Li and Bailey), which keeps the vectors to ~1e-15
// relative per reflector (about 1e-13 after the ~2000 reflectors an entry meets). The vectors are
// held transposed (row j, column t) as float2 pairs; the reflector v and beta v are converted per
// task (one entry per lane).
struct ff { float h, l; };

__device__ __forceinline__ ff ff_from(double x)
{
    const float h = (float)x;
    return {h, (float)(x - (double)h)};
}

__device__ __forceinline__ double ff_to(ff a) { return (double)a.h + (double)a.l; }

// (s_h + s_l) += (a_h + a_l)(b_h + b_l): exact product of the high parts, cross terms by FMA. The
// rounded operations are written as intrinsics so that the compiler cannot contract them into
// FMAs (which would break the exact two-sum).
__device__ __forceinline__ void ff_fma_acc(float &sh, float &sl, float ah, float al, float bh, float bl)
{
    const float p = __fmul_rn(ah, bh);
    float e = fmaf(ah, bh, -p);
    e = fmaf(ah, bl, fmaf(al, bh, e));
    const float t = __fadd_rn(sh, p), bv = __fsub_rn(t, sh);
    sl = __fadd_rn(sl, __fadd_rn(__fadd_rn(__fsub_rn(sh, __fsub_rn(t, bv)), __fsub_rn(p, bv)), e));
    sh = t;
}

// The chase's reflectors (v, beta) as float-float w = sqrt(beta) v, written in place over the FP64
// reflector rows (a float2 has the size of a double), so that H = I - w w^T and the kernels below
// convert nothing per use. Grid (ceil(Mmax NT / 8), nb), 256 threads: one warp per (sweep, task).
__global__ void __launch_bounds__(256)
k_band_refl_ff(const int32_t *__restrict__ plan, int nb, int Mmax, int NT, double *__restrict__ refl2,
               const double *__restrict__ tau2)
{
    const int b = blockIdx.y;
    const int M = plan[3 * nb + b];
    const int lane = threadIdx.x & 31;
    const int q = blockIdx.x * 8 + (threadIdx.x >> 5);
    const int s = q / NT, i = q % NT;
    if (s >= M - 2 || i >= (M - 2 - s + KB - 1) / KB) return;
    const size_t slot = ((size_t)b * Mmax + s) * NT + i;
    const double w = refl2[slot * KB + lane] * sqrt(tau2[slot]);
    const float h = (float)w;
    __syncwarp();
    reinterpret_cast<float2 *>(refl2)[slot * KB + lane] = make_float2(h, (float)(w - (double)h));
}


// (s_h + s_l) += (b_h + b_l) by two-sum of the high parts (not renormalised)
__device__ __forceinline__ void ff_add(float &sh, float &sl, float bh, float bl)
{
    const float t = __fadd_rn(sh, bh), bv = __fsub_rn(t, sh);
    sl = __fadd_rn(__fadd_rn(sl, bl), __fadd_rn(__fsub_rn(sh, __fsub_rn(t, bv)), __fsub_rn(bh, bv)));
    sh = t;
}

// Yt[b] holds the window's eigenvectors transposed as float-float (row j, column t; ld = mmax).
// Grid (ceil(mmax / VPW), nb), 256 threads, 32 / VPW CTAs per SM: the LPV = 32 / VPW lanes
// l, l + VPW, ... share vector t0 + (l mod VPW), each holding KB / LPV of a reflector's rows (fewer
// registers per lane, so more warps hide the latency of the float-float chains); the reflectors of
// a sweep (disjoint rows) spread over the 8 warps, sweeps in reverse order with a CTA barrier
// between them.
template <int VPW>
__global__ void __launch_bounds__(32 * kBtWarps, 32 / VPW)
k_band_bt2(const int32_t *__restrict__ plan, int nb, int Mmax, int mmax, int NT, const float2 *__restrict__ rf,
           const double *__restrict__ tau2, float2 *__restrict__ Yt)
{
    constexpr int LPV = 32 / VPW, HR = KB / LPV;           // lanes per vector, rows per lane
    const int b = blockIdx.y;
    const int mb = plan[nb + b], M = plan[3 * nb + b];
    const int t0 = blockIdx.x * VPW;
    if (t0 >= mb) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int vi = lane % VPW, hh = lane / VPW;
    float2 *Y = Yt + (size_t)b * Mmax * mmax + t0 + vi;
    const bool act = t0 + vi < mb;
    for (int s = M - 3; s >= 0; s--) {
        const int ntask = (M - 2 - s + KB - 1) / KB;
        for (int i = warp; i < ntask; i += kBtWarps) {
            const size_t slot = ((size_t)b * Mmax + s) * NT + i;
            if (tau2[slot] == 0.0) continue;
            const float2 wl = rf[slot * KB + lane];        // w = sqrt(beta) v, zero past the length
            const int a = s + 1 + i * KB;
            const int L = min(KB, M - a);
            const int r0 = HR * hh;
            float2 yv[HR];
#pragma unroll
            for (int k = 0; k < HR; k++)
                yv[k] = (act && r0 + k < L) ? Y[(size_t)(a + r0 + k) * mmax] : make_float2(0.f, 0.f);
            // d = w . y in float-float: this lane's rows in two accumulators, then the LPV lanes of
            // the vector by a butterfly that adds lower + upper in every lane (identical results)
            float dh0 = 0.f, dl0 = 0.f, dh1 = 0.f, dl1 = 0.f;
#pragma unroll
            for (int k = 0; k < HR; k += 2) {
                ff_fma_acc(dh0, dl0, __shfl_sync(0xffffffffu, wl.x, r0 + k), __shfl_sync(0xffffffffu, wl.y, r0 + k),
                           yv[k].x, yv[k].y);
                ff_fma_acc(dh1, dl1, __shfl_sync(0xffffffffu, wl.x, r0 + k + 1),
                           __shfl_sync(0xffffffffu, wl.y, r0 + k + 1), yv[k + 1].x, yv[k + 1].y);
            }
            ff_add(dh0, dl0, dh1, dl1);
#pragma unroll
            for (int o = VPW; o < 32; o <<= 1) {
                const float ph = __shfl_xor_sync(0xffffffffu, dh0, o), pl = __shfl_xor_sync(0xffffffffu, dl0, o);
                if (lane & o) {
                    float xh = ph, xl = pl;
                    ff_add(xh, xl, dh0, dl0);
                    dh0 = xh;
                    dl0 = xl;
                } else {
                    ff_add(dh0, dl0, ph, pl);
                }
            }
            // y_r -= d w_r, then renormalised
#pragma unroll
            for (int k = 0; k < HR; k++) {
                const float bh = __shfl_sync(0xffffffffu, wl.x, r0 + k), bl = __shfl_sync(0xffffffffu, wl.y, r0 + k);
                float sh = yv[k].x, sl = yv[k].y;
                ff_fma_acc(sh, sl, -dh0, -dl0, bh, bl);
                const float h = __fadd_rn(sh, sl);
                if (act && r0 + k < L) Y[(size_t)(a + r0 + k) * mmax] = make_float2(h, __fsub_rn(sl, __fsub_rn(h, sh)));
            }
        }
        __syncthreads();
    }
}

// sel_vec (rows t, entries j, FP64) <-> Yt (rows j, columns t, float-float), 32 x 32 tiles. Grid
// (ceil(Mmax / 32), ceil(mmax / 32), nb), 256 threads.
__global__ void __launch_bounds__(256)
k_band_transpose(const int32_t *__restrict__ plan, int nb, int Mmax, int mmax, bool to_rows,
                 double *__restrict__ sel_vec, float2 *__restrict__ Yt)
{
    __shared__ double tile[32][33];
    const int b = blockIdx.z;
    const int mb = plan[nb + b], M = plan[3 * nb + b];
    const int j0 = blockIdx.x * 32, t0 = blockIdx.y * 32;
    if (j0 >= M || t0 >= mb) return;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    double *sv = sel_vec + (size_t)b * mmax * Mmax;
    float2 *yt = Yt + (size_t)b * Mmax * mmax;
    if (!to_rows) {
        for (int q = ty; q < 32; q += 8) {
            const int t = t0 + q, j = j0 + tx;
            tile[q][tx] = (t < mb && j < M) ? sv[(size_t)t * Mmax + j] : 0.0;
        }
        __syncthreads();
        for (int q = ty; q < 32; q += 8) {
            const int j = j0 + q, t = t0 + tx;
            if (j < M && t < mb) {
                const ff f = ff_from(tile[tx][q]);
                yt[(size_t)j * mmax + t] = make_float2(f.h, f.l);
            }
        }
    } else {
        for (int q = ty; q < 32; q += 8) {
            const int j = j0 + q, t = t0 + tx;
            if (j < M && t < mb) {
                const float2 f = yt[(size_t)j * mmax + t];
                tile[q][tx] = ff_to({f.x, f.y});
            } else {
                tile[q][tx] = 0.0;
            }
        }
        __syncthreads();
        for (int q = ty; q < 32; q += 8) {
            const int t = t0 + q, j = j0 + tx;
            if (t < mb && j < M) sv[(size_t)t * Mmax + j] = tile[tx][q];
        }
    }
}

// ---- back-transformation of stage 1: y = Q1 y', panel by panel ----------------------------------
// Panel p's reflectors are I - V T V^T; for the eigenvector rows Yr (rows t, entries j) that is
// Yr <- Yr - (Yr V T^T) V^T, applied for p = last .. 0. X = Yr V and Yr -= U V^T are digit
// products; this kernel forms U = X T^T (rows t < m_b of window b, in place). Grid
// (ceil(mmax / 64), nb), 256 threads.
__global__ void __launch_bounds__(256)
k_band_bt1_u(const int32_t *__restrict__ plan, int nb, int mmax, const double *__restrict__ Tp, double *__restrict__ X)
{
    const int b = blockIdx.y;
    const int mb = plan[nb + b];
    const int t0 = blockIdx.x * 64;
    if (t0 >= mb) return;
    const int rows = min(64, mb - t0);
    __shared__ double T[KB][KB + 1], Xs[64][KB + 1];
    const int tid = threadIdx.x;
    const double *Tb = Tp + (size_t)b * KB * KB;
    for (int e = tid; e < KB * KB; e += 256) T[e / KB][e % KB] = Tb[e];
    double *Xb = X + ((size_t)b * mmax + t0) * KB;
    for (int e = tid; e < 64 * KB; e += 256) Xs[e / KB][e % KB] = (e / KB < rows) ? Xb[e] : 0.0;
    __syncthreads();
    const int il = tid >> 2, q0 = tid & 3;
    double u[8];
#pragma unroll
    for (int j = 0; j < 8; j++) {
        const int q = q0 + 4 * j;
        double s = 0.0;
        for (int r = q; r < KB; r++) s = fma(Xs[il][r], T[q][r], s);    // T upper triangular
        u[j] = s;
    }
    if (il < rows)
#pragma unroll
        for (int j = 0; j < 8; j++) Xb[(size_t)il * KB + q0 + 4 * j] = u[j];
}

// ---- host side ------------------------------------------------------------------------------------

size_t chase_smem() { return (size_t)kChaseWarps * (KB * (KB + 1) + 2 * KB) * sizeof(double); }

size_t band_panel_smem(int Mmax)
{
    const int rpc = (Mmax - KB + kPanelCL - 1) / kPanelCL;
    return ((size_t)rpc * (KB + 1) + 32 + 2 + KB + 8 * KB + 2 * KB + 3 * KB * KB + 4 + KB) * sizeof(double);
}

bool band_reduction_fits(int Mmax, size_t smem_cap)
{
    if (Mmax < 2 * KB + 2) return false;
    const int nt0 = (Mmax - 2 + KB - 1) / KB;
    return band_panel_smem(Mmax) <= smem_cap && nt0 < 3 * kChaseCL * kChaseWarps;
}

int band_tasks_per_sweep(int Mmax) { return (Mmax + KB - 1) / KB; }

cudaError_t configure_band_kernels()
{
    int dev = 0, cap = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&cap, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_band_chase, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)chase_smem())) !=
        cudaSuccess)
        return e;
    return cudaFuncSetAttribute(k_band_panel, cudaFuncAttributeMaxDynamicSharedMemorySize, cap);
}

cudaError_t launch_band_reduction(pfsm_handle_s *h, const double *A, cudaStream_t st)
{
    Workspace &w = h->ws;
    const int nb = h->nb, Mmax = h->Mmax;
    const int32_t *plan = w.plan;
    const int64_t MM = (int64_t)Mmax * Mmax;
    cudaError_t e;
    k_band_copy<<<dim3((unsigned)((Mmax + 7) / 8), (unsigned)nb), 256, 0, st>>>(A, h->N, plan, nb, Mmax, w.iiwork,
                                                                                 w.refl, w.tau);
    g_launches++;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const int np = band_panels(Mmax);
    const int nchunk = (Mmax + kChunk - 1) / kChunk;
    const int rpc_cap = (Mmax - KB + kPanelCL - 1) / kPanelCL;
    const size_t psmem = band_panel_smem(Mmax);
    for (int p = 0; p < np; p++) {
        const int c = p * KB, r0 = c + KB;
        // this panel's extents (M, or 0 for a window without it), T factors and reflector rows
        int32_t *extp = w.bExt + (size_t)p * nb;
        double *Tp = w.bT + (size_t)p * nb * KB * KB;
        double *Vrows = w.bV + (size_t)p * nb * Mmax * KB;
        {
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3((unsigned)(nb * kPanelCL));
            cfg.blockDim = dim3(kPanelThreads);
            cfg.dynamicSmemBytes = psmem;
            cfg.stream = st;
            cudaLaunchAttribute attr[1];
            attr[0].id = cudaLaunchAttributeClusterDimension;
            attr[0].val.clusterDim.x = kPanelCL;
            attr[0].val.clusterDim.y = 1;
            attr[0].val.clusterDim.z = 1;
            cfg.attrs = attr;
            cfg.numAttrs = 1;
            if ((e = counted(cudaLaunchKernelEx(&cfg, k_band_panel, plan, nb, Mmax, c, rpc_cap, w.iiwork, w.refl,
                                                w.tau, Tp, extp))) != cudaSuccess)
                return e;
        }
        // Y = A22 V: digits of A22 (rows r0 .. M-1, entries r0 .. M-1) and of V^T (reflector rows)
        const int64_t ldk = padded_ld(Mmax - r0);
        const SliceBuf dA{w.bdA, (int64_t)nb * Mmax, ldk, OZ_SLICES, 0};
        const SliceBuf dV{w.bdV, (int64_t)nb * KB, ldk, OZ_SLICES, 0};
        // A22 = D22 + E22: digits of E22 only (its entries are small against the diagonal, which
        // would otherwise set each row's digit scale), D22 V added exactly in FP64
        if ((e = launch_oz_split_win(w.iiwork, MM, Mmax, r0, r0, extp, r0, 0, nullptr, Mmax - r0, nb, dA, Mmax, r0,
                                     w.bdeA, st, w.bD)) != cudaSuccess)
            return e;
        if ((e = launch_oz_split_win(w.refl, MM, Mmax, c, r0, extp, r0, KB, nullptr, KB, nb, dV, KB, 0, w.bdeV, st)) !=
            cudaSuccess)
            return e;
        OzParams o{};
        o.rows = Mmax; o.cols = KB; o.cols_from_zero = 1; o.C = w.bY; o.ldc = KB; o.status = w.status;
        o.zrow = Mmax; o.zrow_q = KB; o.zc = (int64_t)Mmax * KB; o.row_base = r0; o.ext = extp;
        o.Vp = w.refl + (size_t)c * Mmax; o.ldv = 1; o.vcs = Mmax; o.zv = MM; o.drow = w.bD; o.zd = Mmax;
        if ((e = launch_gemm_oz(dA, w.bdeA, dV, w.bdeV, o, st, nb)) != cudaSuccess) return e;
        // W = Y T, U = T^T V^T W, Z = W - V U / 2 -> [V Z], [Z V]
        const dim3 gch((unsigned)((Mmax - r0 + kChunk - 1) / kChunk), (unsigned)nb);
        k_band_w<<<gch, 256, 0, st>>>(extp, Mmax, c, w.refl, Tp, w.bY, w.bXp, nchunk);
        g_launches++;
        k_band_u<<<nb, 256, 0, st>>>(extp, c, Tp, w.bXp, nchunk, w.bU);
        g_launches++;
        k_band_z<<<gch, 256, 0, st>>>(extp, Mmax, c, w.refl, w.bY, w.bU, w.VW, w.WV, Vrows);
        g_launches++;
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        // A22 -= [V Z] [Z V]^T (rows and columns r0 .. M-1 of every window that had this panel)
        const int64_t srows = (int64_t)nb * Mmax;
        const SliceBuf dP{w.tdP, srows, 2 * KB, OZ_SLICES, 0}, dQ{w.tdQ, srows, 2 * KB, OZ_SLICES, 0};
        if ((e = launch_oz_split(w.VW, srows, 2 * KB, 2 * KB, dP, w.tdeP, st)) != cudaSuccess) return e;
        if ((e = launch_oz_split(w.WV, srows, 2 * KB, 2 * KB, dQ, w.tdeQ, st)) != cudaSuccess) return e;
        OzParams u{};
        u.rows = Mmax; u.cols = Mmax; u.C = w.iiwork; u.ldc = Mmax; u.sub = 1; u.status = w.status;
        u.zrow = Mmax; u.zc = MM; u.row_base = r0; u.ext = extp;
        if ((e = launch_gemm_oz_strip(dP, w.tdeP, dQ, w.tdeQ, u, st, nb, kStrip)) != cudaSuccess) return e;
    }
    if (h->timing && (e = cudaEventRecord(h->band_ev[0], st)) != cudaSuccess) return e;
    k_band_extract<<<dim3((unsigned)((Mmax + 2 * KB + 7) / 8), (unsigned)nb), 256, 0, st>>>(plan, nb, Mmax, w.iiwork,
                                                                                         w.bBw);
    g_launches++;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(nb * kChaseCL));
    cfg.blockDim = dim3(32 * kChaseWarps);
    cfg.dynamicSmemBytes = chase_smem();
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = kChaseCL;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if ((e = counted(cudaLaunchKernelEx(&cfg, k_band_chase, plan, nb, Mmax, band_tasks_per_sweep(Mmax), w.bBw, w.bR2,
                                        w.bT2, w.td, w.te))) != cudaSuccess)
        return e;
    return h->timing ? cudaEventRecord(h->band_ev[1], st) : cudaSuccess;
}

cudaError_t launch_band_backtransform(pfsm_handle_s *h, cudaStream_t st)
{
    Workspace &w = h->ws;
    const int nb = h->nb, Mmax = h->Mmax, mmax = h->mmax;
    const int32_t *plan = w.plan;
    cudaError_t e;
    // stage 2: y' = Q2 z on the transposed eigenvectors
    float2 *Yt = reinterpret_cast<float2 *>(w.iiwork);   // free again after the inverse iteration
    const dim3 gt((unsigned)((Mmax + 31) / 32), (unsigned)((mmax + 31) / 32), (unsigned)nb);
    k_band_transpose<<<gt, 256, 0, st>>>(plan, nb, Mmax, mmax, false, w.sel_vec, Yt);
    g_launches++;
    const int NT = band_tasks_per_sweep(Mmax);
    k_band_refl_ff<<<dim3((unsigned)(((size_t)Mmax * NT + 7) / 8), (unsigned)nb), 256, 0, st>>>(plan, nb, Mmax, NT,
                                                                                              w.bR2, w.bT2);
    g_launches++;
    const float2 *rf = reinterpret_cast<const float2 *>(w.bR2);
    k_band_bt2<kBtVpw><<<dim3((unsigned)((mmax + kBtVpw - 1) / kBtVpw), (unsigned)nb), 32 * kBtWarps, 0, st>>>(
        plan, nb, Mmax, mmax, NT, rf, w.bT2, Yt);
    g_launches++;
    k_band_transpose<<<gt, 256, 0, st>>>(plan, nb, Mmax, mmax, true, w.sel_vec, Yt);
    g_launches++;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (h->timing && (e = cudaEventRecord(h->band_ev[2], st)) != cudaSuccess) return e;
    // stage 1: y = Q1 y', panels last .. first, on the rows of sel_vec (vector t, entries j)
    const int np = band_panels(Mmax);
    const int64_t nbm = (int64_t)nb * mmax, nbM = (int64_t)nb * Mmax;
    for (int p = np - 1; p >= 0; p--) {
        const int c = p * KB, r0 = c + KB;
        const int32_t *extp = w.bExt + (size_t)p * nb;
        const int64_t ldk = padded_ld(Mmax - r0);
        const SliceBuf dY{w.bdA, nbm, ldk, OZ_SLICES, 0}, dV{w.bdV, (int64_t)nb * KB, ldk, OZ_SLICES, 0};
        // X = Yr V: the rows' entries r0 .. M-1 against the reflector rows (zero digits for a window
        // without this panel, so its X, U and update vanish)
        if ((e = launch_oz_split_win(w.sel_vec, (int64_t)mmax * Mmax, Mmax, 0, r0, extp, r0, 0, plan + nb, mmax, nb, dY,
                                     mmax, 0, w.bdeA, st)) != cudaSuccess)
            return e;
        if ((e = launch_oz_split_win(w.refl, (int64_t)Mmax * Mmax, Mmax, c, r0, extp, r0, KB, nullptr, KB, nb, dV, KB, 0,
                                     w.bdeV, st)) != cudaSuccess)
            return e;
        OzParams o{};
        o.rows = mmax; o.cols = KB; o.cols_from_zero = 1; o.C = w.bY; o.ldc = KB; o.status = w.status;
        o.zrow = mmax; o.zrow_q = KB; o.zc = (int64_t)mmax * KB; o.ext = plan + nb; o.ext_c = w.bKB;
        if ((e = launch_gemm_oz(dY, w.bdeA, dV, w.bdeV, o, st, nb)) != cudaSuccess) return e;
        // U = X T^T
        k_band_bt1_u<<<dim3((unsigned)((mmax + 63) / 64), (unsigned)nb), 256, 0, st>>>(
            plan, nb, mmax, w.bT + (size_t)p * nb * KB * KB, w.bY);
        g_launches++;
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        // Yr[:, r0:M] -= U V^T
        const SliceBuf dU{w.tdP, nbm, KB, OZ_SLICES, 0}, dW{w.tdQ, nbM, KB, OZ_SLICES, 0};
        if ((e = launch_oz_split(w.bY, nbm, KB, KB, dU, w.tdeP, st)) != cudaSuccess) return e;
        if ((e = launch_oz_split(w.bV + (size_t)p * nbM * KB, nbM, KB, KB, dW, w.tdeQ, st)) != cudaSuccess) return e;
        OzParams u{};
        u.rows = mmax; u.cols = Mmax; u.col_off = r0; u.C = w.sel_vec; u.ldc = Mmax; u.sub = 1; u.status = w.status;
        u.zrow = mmax; u.zrow_q = Mmax; u.zc = (int64_t)mmax * Mmax; u.ext = plan + nb; u.ext_c = plan + 3 * nb;
        if ((e = launch_gemm_oz_strip(dU, w.tdeP, dW, w.tdeQ, u, st, nb, kStrip)) != cudaSuccess) return e;
    }
    return launch_bt_finish(h, w.sel_vec, st);
}

}  // namespace pfsm
