// Batched FP64 submatrix eigensolves and start vectors (Section II: "solving a sequence of
// eigenvector problems generated from overlapping diagonal submatrices"; the eigenvectors y of
// each submatrix B start Eq. 11 and its eigenvalues are the shifts).
//
// Only the m eigenpairs of each window at the slice's own ascending positions are needed, so
// instead of a full dense eigensolver the pipeline is:
//   1. k_tridiag      Householder reduction of every window B_b to tridiagonal T_b
//                     (Golub & Van Loan Sec. 8.3.1). One thread-block cluster per window; rows
//                     are spread cyclically over the cluster's CTAs (in shared memory when they
//                     fit, else in global memory) and the Householder vector and the product
//                     p = beta B v are exchanged through distributed shared memory.
//   2. k_bisect       the selected eigenvalues of T_b: FP32 Sturm bisection, FP64 Newton steps on
//                     det(T - xI), FP64 Sturm counts certifying the index; one lane each.
//   3. k_inverse_iter their eigenvectors of T_b by inverse iteration (two solves) with a pivoted
//                     tridiagonal LU, re-orthogonalised inside clusters of (nearly) equal
//                     eigenvalues.
//   4. k_backtransform y = H_0 ... H_{M-3} z, sign rule, zero padding to length N, shift eps and
//                     step alpha: one warp per start vector, written straight into X.
#include <cooperative_groups.h>
#include <algorithm>
#include <cfloat>

#include "fp64_util.cuh"
#include "pfsm_internal.cuh"

namespace cg = cooperative_groups;

namespace pfsm {

constexpr int kTriThreads = 256;      // blocked panel kernel
constexpr int kTriLaThreads = 288;    // k_tridiag: warp 0 + eight warps (two per sub-partition)
constexpr size_t kInvSmemCap = 200 * 1024;  // k_inverse_iter: shared memory for the lanes' vectors

// named barrier `id` over n threads: bar.sync waits for all n, bar.arrive counts this warp
// without waiting (the arriving threads' earlier shared-memory writes are visible to the waiters)
__device__ __forceinline__ void named_sync(int id, int n)
{
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}
__device__ __forceinline__ void named_arrive(int id, int n)
{
    asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(n) : "memory");
}

__device__ __forceinline__ double block_sum(double v, double *red)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[w] = v;
    __syncthreads();
    // pairwise over the warps (a serial sum would be a chain of dependent FP64 adds); the same
    // order in every thread and every CTA
    double t = 0.0;
    if (nw == 8) {
        t = ((red[0] + red[1]) + (red[2] + red[3])) + ((red[4] + red[5]) + (red[6] + red[7]));
    } else {
        for (int i = 0; i < nw; i++) t += red[i];
    }
    return t;
}

// Householder scalars of the column c (entries kk+1 .. M-1) that step kk reduces, by one warp:
// x0 = c[kk+1], alpha = -sign(x0) ||c||, v0 = x0 - alpha, beta = 2 / (v0^2 + sum_{i > kk+1} c_i^2)
// (beta = 0 and alpha = x0 when the tail is already zero).
__device__ __forceinline__ void householder_scalars(const double *c, int kk, int M, int lane, double *sc)
{
    const double x0 = c[kk + 1];
    double t2 = 0.0;
    for (int i = kk + 2 + lane; i < M; i += 32) t2 = fma(c[i], c[i], t2);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t2 += __shfl_xor_sync(0xffffffffu, t2, o);
    double beta = 0.0, alpha = x0, v0 = 0.0;
    if (t2 != 0.0) {
        const double nn = fma(x0, x0, t2);
        const double xn = nn * fast_rsqrt(nn);
        alpha = (x0 >= 0.0) ? -xn : xn;
        v0 = x0 - alpha;
        beta = 2.0 * fast_rcp(fma(v0, v0, t2));
    }
    if (lane == 0) { sc[0] = beta; sc[1] = alpha; sc[2] = v0; }
}

// The fused loop of k_tridiag for NG rows (entries j >= rmin, lanes along the row): with UPD the
// rank-2 update B_ij -= v_i w_j + w_i v_j, and acc_g += B_ij c_j on the (updated) entries.
template <int NG, bool UPD>
__device__ __forceinline__ void tri_rows(double *const *rp, const double *vi, const double *wi,
                                         const double *__restrict__ hv, const double *__restrict__ wv,
                                         const double *__restrict__ cv, int rmin, int M, int lane,
                                         double *acc)
{
    for (int j = rmin + lane; j < M; j += 32) {
        const double vj = hv[j], wj = wv[j], cj = cv[j];
#pragma unroll
        for (int g = 0; g < NG; g++) {
            double bb = rp[g][j];
            if (UPD) {
                bb = fma(-vi[g], wj, fma(-wi[g], vj, bb));
                rp[g][j] = bb;
            }
            acc[g] = fma(bb, cj, acc[g]);
        }
    }
}

// Householder reduction of every window to tridiagonal form, one thread-block cluster per window.
// Grid: nb * CL CTAs, clusters of CL along x; CTA `rank` owns the rows i with i % CL == rank (in
// shared memory when they fit, else in the window's global work matrix).
//
// B300 spends ~64 cycles of a sub-partition's FP64 pipe on every FP64 warp instruction and a
// dependent FP64 chain runs at about that pace, so the step is arranged around ONE cluster barrier
// with all of its serial work hidden behind the rank-2 update (a look-ahead form of Golub & Van
// Loan Sec. 8.3.1). Step k starts with, in every CTA: the Householder vector v of column k
// (entries > k) and its scalars (alpha, beta), p_i = beta (B v)_i for every row i > k, the
// partial sums of p.v and row k+1 (entries > k+1), all sent during the previous step.
//   --  cluster barrier
//   S2  w = p - (beta p.v / 2) v, and the next column x' = (row k+1) - v_{k+1} w - w_{k+1} v,
//       i.e. column k+1 after this step's update, in every CTA without a second exchange.
//   S3  warp 0: the scalars of step k+1 from x' and its Householder vector v' (CTA 0 also stores
//       the reflector). Warps 1-8 (two per SM sub-partition): the rank-2 update B -= v w^T + w v^T
//       of the owned rows fused with u = B x' on the freshly updated entries (lanes along the
//       row, up to eight rows per warp in a loop compiled for the exact row count, the per-row
//       sums by one transpose-reduce); then, once warp 0 has published v' (named barrier 1),
//       p'_i = beta' (u_i - alpha' B_{i,k+2}) = beta' (B v')_i and p'_i v'_i for the owned rows;
//       after named barrier 2 the fused warps copy the CTA's p' values as one contiguous block
//       into every CTA (coalesced remote stores), warp 0 sums the CTA's partial p'.v' and sends
//       it, and the owner of row k+2 sends that row.
// B300's SM retires about one FP64 warp instruction per 16 cycles whatever its active lanes, so
// the work outside the fused loop is kept to few FP64 warp instructions (one warp reduces where a
// reduction in every warp would queue eight times the instructions on the same pipe).
// Buffers written by other CTAs (p, the p.v partials, row k+1) and the vector v alternate with
// the step's parity: a CTA can run at most one step ahead of another, since it cannot pass the
// next barrier first.
template <bool SMEM_ROWS>
__global__ void __launch_bounds__(kTriLaThreads, 1)
k_tridiag(const double *__restrict__ A, int64_t N, const int32_t *__restrict__ plan, int32_t nb,
          int32_t Mmax, double *__restrict__ gwork, double *__restrict__ refl,
          double *__restrict__ tau, double *__restrict__ td, double *__restrict__ te)
{
    constexpr int G = 8;                               // rows per warp group in the fused loop
    constexpr int NWQ = kTriLaThreads / 32 - 1;        // warps of the fused loop
    cg::cluster_group cluster = cg::this_cluster();
    const int CL = (int)cluster.num_blocks();
    const int rank = (int)cluster.block_rank();
    const int b = blockIdx.x / CL;
    const int64_t s0 = plan[2 * nb + b];
    const int M = plan[3 * nb + b];
    const int R = (Mmax + CL - 1) / CL;
    extern __shared__ double sm[];
    double *rows = SMEM_ROWS ? sm : (gwork + (size_t)b * Mmax * Mmax);
    double *vec = sm + (SMEM_ROWS ? (size_t)R * Mmax : 0);
    double *xcol = vec;                    // column to reduce next: column 0, then each step's x'
    double *hvb = vec + Mmax;              // [2][Mmax] v of the step of that parity
    double *wv = vec + 3 * Mmax;           // w
    const int PS = Mmax + 16;              // >= CL R
    double *pbuf = vec + 4 * Mmax;         // [2][PS] p: block [CL][R], row li * CL + r at r R + li
    double *rowbuf = pbuf + 2 * PS;        // [2][Mmax] row k+1 (written by its owner)
    double *uu = rowbuf + 2 * Mmax;        // [R] (B x')_i of the owned rows
    double *prod = uu + R;                 // [R] p_i v_i of the owned rows
    double *pst = prod + R;                // [R] p_i of the owned rows (staging for the push)
    double *pvp = pst + R;                 // [2][32] partial p.v of every CTA
    double *scb = pvp + 64;                // [2][4] beta, alpha, v0 of the step of that parity
    double *kcs = scb + 8;                 // beta p.v / 2 of the current step
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    auto rowp = [&](int i) -> double * {
        return SMEM_ROWS ? rows + (size_t)(i / CL) * Mmax : rows + (size_t)i * Mmax;
    };
    double *brefl = refl + (size_t)b * Mmax * Mmax;
    double *btau = tau + (size_t)b * Mmax, *btd = td + (size_t)b * Mmax, *bte = te + (size_t)b * Mmax;
    const int nown = (M - rank + CL - 1) / CL;         // owned rows li * CL + rank < M

    // rows i >= rmin: B_ij -= v_i w_j + w_i v_j for j >= rmin (when upd), and
    // uu = sum_{j >= rmin} B_ij c_j on the updated entries (c_rmin must be 0 or part of the sum).
    // Fused warp wq takes the owned rows li = lfirst + wq + NWQ m, up to G at a time; each group
    // runs a loop compiled for its exact row count (no FP64 work issued for absent rows).
    auto fused = [&](int rmin, const double *cv, const double *hv, bool upd) {
        const int wq = warp - 1;
        const int lfirst = (rmin - rank + CL - 1) / CL;
        for (int t0 = lfirst + wq; t0 < nown; t0 += NWQ * G) {
            double *rp[G];
            double vi[G], wi[G], acc[G];
            int cnt = 0;
#pragma unroll
            for (int g = 0; g < G; g++) {
                const int li = t0 + NWQ * g;
                const bool ok = li < nown;
                const int i = ok ? li * CL + rank : rank;
                rp[g] = rowp(i);
                vi[g] = ok ? hv[i] : 0.0;
                wi[g] = ok ? wv[i] : 0.0;
                acc[g] = 0.0;
                cnt += ok ? 1 : 0;
            }
#define PFSM_TRI_ROWS(NG)                                                                          \
    case NG:                                                                                       \
        if (upd) tri_rows<NG, true>(rp, vi, wi, hv, wv, cv, rmin, M, lane, acc);                 \
        else tri_rows<NG, false>(rp, vi, wi, hv, wv, cv, rmin, M, lane, acc);                    \
        break;
            switch (cnt) {
                PFSM_TRI_ROWS(1)
                PFSM_TRI_ROWS(2)
                PFSM_TRI_ROWS(3)
                PFSM_TRI_ROWS(4)
                PFSM_TRI_ROWS(5)
                PFSM_TRI_ROWS(6)
                PFSM_TRI_ROWS(7)
                default: PFSM_TRI_ROWS(8)
            }
#undef PFSM_TRI_ROWS
            // sums over the 32 lanes: halve the rows held per lane at offsets 16, 8, 4 (lane
            // ends with row (lane >> 2) & 7), then plain butterflies over the last two lane bits
#pragma unroll
            for (int h = 0; h < 4; h++) {
                const bool up = (lane & 16) != 0;
                const double send = up ? acc[h] : acc[h + 4], keep = up ? acc[h + 4] : acc[h];
                acc[h] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
            }
#pragma unroll
            for (int h = 0; h < 2; h++) {
                const bool up = (lane & 8) != 0;
                const double send = up ? acc[h] : acc[h + 2], keep = up ? acc[h + 2] : acc[h];
                acc[h] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
            }
            {
                const bool up = (lane & 4) != 0;
                const double send = up ? acc[0] : acc[1], keep = up ? acc[1] : acc[0];
                acc[0] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
            }
            acc[0] += __shfl_xor_sync(0xffffffffu, acc[0], 2);
            acc[0] += __shfl_xor_sync(0xffffffffu, acc[0], 1);
            const int g = (lane >> 2) & 7;
            if ((lane & 3) == 0 && g < cnt) uu[t0 + NWQ * g] = acc[0];
        }
    };

    // warp 0: scalars of step kn from the column in xcol (entries > kn), its Householder vector
    // into hv[parn] and, in CTA 0, the reflector, alpha and beta into the window's outputs
    auto next_vector = [&](int kn, int parn) {
        const int n1n = kn + 1;
        double *scn = scb + 4 * parn, *hvn = hvb + (size_t)parn * Mmax;
        householder_scalars(xcol, kn, M, lane, scn);
        __syncwarp();
        const double beta = scn[0], alpha = scn[1], v0 = scn[2];
        double *rr = brefl + (size_t)kn * Mmax;
        for (int j = n1n + lane; j < M; j += 32) {
            const double v = (beta != 0.0) ? ((j == n1n) ? v0 : xcol[j]) : 0.0;
            hvn[j] = v;
            if (rank == 0) rr[j] = v;
        }
        if (rank == 0 && lane == 0) { bte[kn] = alpha; btau[kn] = beta; }
    };

    // fused warps, after the fused loop over rows >= rmin and warp 0's next_vector for the step
    // whose first row is n1n: p_i (zero for i < n1n) and p_i v_i of the warp's own rows into pst
    // and prod; after named barrier 2 (with warp 0) the owned rows' p values go to block `rank` of
    // every CTA's p buffer as contiguous runs (coalesced remote stores), and the owner of row n1n
    // sends that row (entries > n1n)
    auto publish = [&](int rmin, int n1n, int parn) {
        const int wq = warp - 1;
        const double *scn = scb + 4 * parn, *hvn = hvb + (size_t)parn * Mmax;
        const double beta = scn[0], alpha = scn[1];
        const int lfirst = (rmin - rank + CL - 1) / CL;
        for (int li = lfirst + wq + NWQ * lane; li < nown; li += NWQ * 32) {
            const int i = li * CL + rank;
            double p = 0.0, pr = 0.0;
            if (i >= n1n) {
                p = beta * fma(-alpha, rowp(i)[n1n], uu[li]);
                pr = p * hvn[i];
            }
            pst[li] = p;
            prod[li] = pr;
        }
        named_sync(2, kTriLaThreads);
        const int cntp = nown - lfirst;
        if (cntp > 0) {
            double *pbn = pbuf + (size_t)parn * PS + (size_t)rank * R;
            for (int idx = tid - 32; idx < CL * cntp; idx += NWQ * 32) {
                const int r = idx / cntp, li = lfirst + idx - r * cntp;
                cluster.map_shared_rank(pbn, r)[li] = pst[li];
            }
        }
        if (n1n % CL == rank) {
            double *rbn = rowbuf + (size_t)parn * Mmax;
            const double *rr = rowp(n1n);
            for (int j = n1n + 1 + (tid - 32); j < M; j += NWQ * 32) {
                const double x = rr[j];
                for (int r = 0; r < CL; r++) cluster.map_shared_rank(rbn, r)[j] = x;
            }
        }
    };

    // warp 0, after named barrier 2: the CTA's partial p.v over its rows >= rmin into every CTA
    // (Every FP64 warp instruction holds the SM's FP64 pipe for ~16 cycles whatever its active
    // lanes, so the sum is one warp's, not a reduction in every warp.)
    auto partial_pv = [&](int rmin, int parn) {
        const int lfirst = (rmin - rank + CL - 1) / CL;
        double t = 0.0;
        for (int q = lfirst + lane; q < nown; q += 32) t += prod[q];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (lane < CL) cluster.map_shared_rank(pvp + 32 * parn, lane)[rank] = t;
    };

    // load owned rows of B = A[s0:s0+M, s0:s0+M]
    for (int i = rank + warp * CL; i < M; i += (kTriLaThreads / 32) * CL) {
        const double *src = A + (s0 + i) * N + s0;
        double *dst = rowp(i);
        for (int j = lane; j < M; j += 32) dst[j] = src[j];
    }
    for (int j = tid; j < 2 * Mmax; j += blockDim.x) hvb[j] = 0.0;
    for (int j = tid; j < Mmax; j += blockDim.x) wv[j] = 0.0;
    // every CTA of the cluster must be running before any distributed-shared-memory access
    cluster.sync();
    // column 0 (entries >= 1) into every CTA
    for (int i = rank + tid * CL; i < M; i += blockDim.x * CL) {
        if (i < 1) continue;
        const double v = rowp(i)[0];
        for (int r = 0; r < CL; r++) cluster.map_shared_rank(xcol, r)[i] = v;
    }
    cluster.sync();
    // step 0's vector, u = B x and p
    if (warp == 0) {
        if (M >= 3) {
            next_vector(0, 0);
            named_arrive(1, kTriLaThreads);
            named_sync(2, kTriLaThreads);
            partial_pv(1, 0);
        }
    } else {
        fused(1, xcol, hvb, false);
        if (M >= 3) {
            named_sync(1, kTriLaThreads);
            publish(1, 1, 0);
        }
    }

    for (int k = 0; k + 2 < M; k++) {
        const int par = k & 1, n1 = k + 1;
        const bool more = k + 3 < M;
        cluster.sync();
        if (k % CL == rank && tid == 0) btd[k] = rowp(k)[k];
        const double *hv = hvb + (size_t)par * Mmax;
        const double *pb = pbuf + (size_t)par * PS, *rb = rowbuf + (size_t)par * Mmax;
        // S2: p.v from the CTAs' partials (in the same order in every CTA) by warp 0
        if (warp == 0) {
            double pv = (lane < CL) ? pvp[32 * par + lane] : 0.0;
#pragma unroll
            for (int o = 8; o > 0; o >>= 1) pv += __shfl_xor_sync(0xffffffffu, pv, o);
            if (lane == 0) kcs[0] = 0.5 * scb[4 * par] * pv;
        }
        __syncthreads();
        const double Kc = kcs[0];
        const double vk1 = hv[n1];
        const double wk1 = fma(-Kc, vk1, pb[(n1 % CL) * R + n1 / CL]);
        for (int j = n1 + tid; j < M; j += blockDim.x) {
            const double vj = hv[j];
            const int jq = j / CL;
            const double wj = fma(-Kc, vj, pb[(j - jq * CL) * R + jq]);
            wv[j] = wj;
            xcol[j] = (j == n1) ? 0.0 : fma(-vk1, wj, fma(-wk1, vj, rb[j]));
        }
        __syncthreads();
        // S3
        if (warp == 0) {
            if (more) {
                next_vector(n1, par ^ 1);
                named_arrive(1, kTriLaThreads);
                named_sync(2, kTriLaThreads);
                partial_pv(n1, par ^ 1);
            }
        } else {
            fused(n1, xcol, hv, true);
            if (more) {
                named_sync(1, kTriLaThreads);
                publish(n1, n1 + 1, par ^ 1);
            }
        }
    }
    __syncthreads();
    // trailing 2x2 (or 1x1)
    if (tid == 0) {
        if (M >= 2) {
            if ((M - 2) % CL == rank) btd[M - 2] = rowp(M - 2)[M - 2];
            if ((M - 1) % CL == rank) { btd[M - 1] = rowp(M - 1)[M - 1]; bte[M - 2] = rowp(M - 1)[M - 2]; }
        } else if (rank == 0) {
            btd[0] = rowp(0)[0];
        }
        if (rank == 0) { bte[M - 1] = 0.0; if (M >= 2) btau[M - 2] = 0.0; btau[M - 1] = 0.0; }
    }
    cluster.sync();   // no CTA leaves while another may still address its shared memory
}

size_t tri_smem_bytes(int Mmax, int CL, bool rows_in_smem)
{
    const size_t R = (size_t)((Mmax + CL - 1) / CL);
    size_t d = (size_t)8 * Mmax + 32 + 3 * R + 64 + 16;
    if (rows_in_smem) d += R * (size_t)Mmax;
    return d * sizeof(double);
}

// ---- blocked reduction (mixed forms) ----------------------------------------------------------
// The same reduction in panels of kPanel = 32 columns (the blocked form of Golub & Van Loan
// Sec. 8.3.1, as in LAPACK's symmetric tridiagonal reduction). Within a panel the trailing matrix
// is NOT updated: with the panel's reflectors v_q and vectors w_q = p_q - (beta_q p_q.v_q / 2) v_q
// collected in V and W, the current matrix is A_ps - V W^T - W V^T (A_ps: the matrix at the start
// of the panel), so step k needs
//   column k:  A_ps[:, k] - V W[k, :]^T - W V[k, :]^T          (O(j M) per step)
//   p = beta (A_ps v - V (W^T v) - W (V^T v))                   (one mat-vec on A_ps)
// and the rank-2 updates of the unblocked loop (2/3 of its FP64 work) become one rank-64 update
// per panel, A_ps -= [V W] [W V]^T, done by the FP64-accurate digit product on the tensor cores
// between panel launches. V and W are stored as the balanced pairs (sqrt(beta) v, w / sqrt(beta))
// (same v w^T, both of order one, as the digit product scales each row of [V W] by one power of
// two). Every step costs two cluster barriers: (A) the updated column k is gathered, (B) the
// mat-vec entries and the partial dot products V^T v, W^T v are gathered.
//
// B300 issues a dependent FP64 FMA every ~64 cycles, so no FP64 reduction here is a long serial
// chain: a warp owns every 8th local row (up to RPW rows), lane q holds V[row][q] and W[row][q] in
// registers, and the per-row sums over q are shuffle trees run for all the warp's rows at once.
// The panel rows' V and W entries (needed by every CTA for the next column) are recomputed
// redundantly in every CTA from the gathered mat-vec. Rows of A_ps sit in shared memory when the
// window fits (M <= Mcap), else they are read from the window matrix in global memory (L2).
template <int RPW>
__global__ void __launch_bounds__(kTriThreads, 1)
k_tridiag_panel(const double *__restrict__ A, int64_t N, const int32_t *__restrict__ plan, int32_t nb,
                int32_t Mmax, int32_t Mcap, int k0, double *__restrict__ gwork, double *__restrict__ refl,
                double *__restrict__ tau, double *__restrict__ td, double *__restrict__ te,
                double *__restrict__ VW, double *__restrict__ WV)
{
    constexpr int NB = kPanel;
    cg::cluster_group cluster = cg::this_cluster();
    const int CL = (int)cluster.num_blocks();
    const int rank = (int)cluster.block_rank();
    const int b = blockIdx.x / CL;
    const int64_t s0 = plan[2 * nb + b];
    const int M = plan[3 * nb + b];
    const int kend = min(k0 + NB, M - 2);              // Householder steps k0 .. kend-1
    if (k0 > 0 && k0 >= M - 2) return;                 // this window finished in an earlier panel
    double *G = gwork + (size_t)b * Mmax * Mmax;       // the window's matrix, updated between panels
    const bool srows = M <= Mcap;
    const int Rcap = (Mcap + CL - 1) / CL;
    extern __shared__ double sm[];
    double *rows = sm;                                 // Rcap x Mcap (when the window fits)
    double *vbuf = sm + (size_t)Rcap * Mcap;
    double *pbuf = vbuf + Mmax;
    double *hv = pbuf + Mmax;
    double *red = hv + Mmax;                           // 64
    double *Vp = red + 64, *Wp = Vp + (NB + 2) * NB;   // panel rows k0 .. k0 + NB + 1
    double *dots = Wp + (NB + 2) * NB;                 // [CL][2 NB] partial V^T v, W^T v
    double *ab = dots + (size_t)CL * 2 * NB;           // a = V^T v (NB), b = W^T v (NB)
    double *wd = ab + 2 * NB;                          // [8 warps][2 NB]
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    auto rowp = [&](int i) -> double * {
        return srows ? rows + (size_t)(i / CL) * Mcap : G + (size_t)i * Mmax;
    };
    auto grow = [&](int t) { return (warp + 8 * t) * CL + rank; };   // global row of slot t
    double *brefl = refl + (size_t)b * Mmax * Mmax;
    double *btau = tau + (size_t)b * Mmax, *btd = td + (size_t)b * Mmax, *bte = te + (size_t)b * Mmax;

    // rows of the panel-start matrix (the first panel copies the window out of A)
    for (int i = rank + warp * CL; i < M; i += 8 * CL) {
        if (i < k0) continue;
        double *dst = rowp(i);
        if (k0 == 0) {
            const double *src = A + (s0 + i) * N + s0;
            double *gdst = G + (size_t)i * Mmax;
            for (int j = lane; j < M; j += 32) {
                const double x = src[j];
                gdst[j] = x;
                if (srows) dst[j] = x;
            }
        } else if (srows) {
            const double *gsrc = G + (size_t)i * Mmax;
            for (int j = k0 + lane; j < M; j += 32) dst[j] = gsrc[j];
        }
    }
    double Vr[RPW], Wr[RPW];                           // V[grow(t)][lane], W[grow(t)][lane]
#pragma unroll
    for (int t = 0; t < RPW; t++) { Vr[t] = 0.0; Wr[t] = 0.0; }
    for (int t = tid; t < 2 * (NB + 2) * NB; t += blockDim.x) Vp[t] = 0.0;
    // every CTA of the cluster must be running before any distributed-shared-memory access
    cluster.sync();

    for (int k = k0; k < kend; k++) {
        const int j = k - k0;
        // (A) column k of the current matrix on owned rows i >= k, gathered into every vbuf
        {
            const double wk = lane < j ? Wp[j * NB + lane] : 0.0, vk = lane < j ? Vp[j * NB + lane] : 0.0;
            double part[RPW];
#pragma unroll
            for (int t = 0; t < RPW; t++) part[t] = fma(Vr[t], wk, Wr[t] * vk);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1)
#pragma unroll
                for (int t = 0; t < RPW; t++) part[t] += __shfl_xor_sync(0xffffffffu, part[t], o);
#pragma unroll
            for (int t = 0; t < RPW; t++) {
                const int i = grow(t);
                if (i < M && i >= k && lane < CL) cluster.map_shared_rank(vbuf, lane)[i] = rowp(i)[k] - part[t];
            }
        }
        cluster.sync();
        // Householder vector of column k (redundantly and identically in every CTA)
        const double x0 = vbuf[k + 1];
        double t2 = 0.0;
        for (int i = k + 2 + tid; i < M; i += blockDim.x) t2 = fma(vbuf[i], vbuf[i], t2);
        const double tail2 = block_sum(t2, red);
        double beta = 0.0, alpha = x0;
        if (tail2 != 0.0) {
            const double nn = fma(x0, x0, tail2);
            const double xn = nn * fast_rsqrt(nn);
            alpha = (x0 >= 0.0) ? -xn : xn;
            const double v0 = x0 - alpha;
            beta = 2.0 * fast_rcp(fma(v0, v0, tail2));
        }
        for (int i = k + 1 + tid; i < M; i += blockDim.x)
            hv[i] = (beta != 0.0) ? ((i == k + 1) ? x0 - alpha : vbuf[i]) : 0.0;
        if (rank == 0) {
            if (tid == 0) { btd[k] = vbuf[k]; bte[k] = alpha; btau[k] = beta; }
            double *rr = brefl + (size_t)k * Mmax;
            for (int i = k + 1 + tid; i < M; i += blockDim.x)
                rr[i] = (beta != 0.0) ? ((i == k + 1) ? x0 - alpha : vbuf[i]) : 0.0;
        }
        __syncthreads();
        // (B) s = A_ps v on owned rows (broadcast), partial V^T v and W^T v over owned rows
        if (beta != 0.0) {
            double acc[RPW];
            const double *rp[RPW];
#pragma unroll
            for (int t = 0; t < RPW; t++) {
                acc[t] = 0.0;
                const int i = grow(t);
                rp[t] = (i < M && i > k) ? rowp(i) : nullptr;
            }
            for (int l = k + 1 + lane; l < M; l += 32) {
                const double h = hv[l];
#pragma unroll
                for (int t = 0; t < RPW; t++)
                    if (rp[t]) acc[t] = fma(rp[t][l], h, acc[t]);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1)
#pragma unroll
                for (int t = 0; t < RPW; t++) acc[t] += __shfl_xor_sync(0xffffffffu, acc[t], o);
            double da = 0.0, db = 0.0, da2 = 0.0, db2 = 0.0;   // two chains each
#pragma unroll
            for (int t = 0; t < RPW; t++) {
                const int i = grow(t);
                if (i < M && i > k) {
                    if (lane < CL) cluster.map_shared_rank(pbuf, lane)[i] = acc[t];
                    const double h = hv[i];
                    if (t & 1) { da2 = fma(Vr[t], h, da2); db2 = fma(Wr[t], h, db2); }
                    else { da = fma(Vr[t], h, da); db = fma(Wr[t], h, db); }
                }
            }
            wd[warp * 2 * NB + lane] = da + da2;
            wd[warp * 2 * NB + NB + lane] = db + db2;
        }
        __syncthreads();
        if (beta != 0.0 && tid < 2 * NB) {
            const double s01 = wd[tid] + wd[2 * NB + tid], s23 = wd[4 * NB + tid] + wd[6 * NB + tid];
            const double s45 = wd[8 * NB + tid] + wd[10 * NB + tid], s67 = wd[12 * NB + tid] + wd[14 * NB + tid];
            const double sum = (s01 + s23) + (s45 + s67);
            for (int r = 0; r < CL; r++) cluster.map_shared_rank(dots, r)[rank * 2 * NB + tid] = sum;
        }
        cluster.sync();
        if (beta != 0.0) {
            // a = V^T v, b = W^T v (same summation order in every CTA)
            if (tid < 2 * NB) {
                double acc = 0.0;
                for (int r = 0; r < CL; r++) acc += dots[r * 2 * NB + tid];
                ab[tid] = acc;
            }
            double sv = 0.0;
            for (int i = k + 1 + tid; i < M; i += blockDim.x) sv = fma(pbuf[i], hv[i], sv);
            sv = block_sum(sv, red);                   // also orders the ab[] writes before use
            const double aq = ab[lane], bq = ab[NB + lane];
            double ab2 = aq * bq;                      // a . b over the lanes (zero beyond j)
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) ab2 += __shfl_xor_sync(0xffffffffu, ab2, o);
            const double Kc = 0.5 * beta * beta * (sv - 2.0 * ab2);
            const double isb = scaled_rsqrt(beta), sb = beta * isb;
            // w = beta (s - V b - W a) - Kc v on owned rows; store column j of (V, W) balanced
            double part[RPW];
#pragma unroll
            for (int t = 0; t < RPW; t++) part[t] = fma(Vr[t], bq, Wr[t] * aq);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1)
#pragma unroll
                for (int t = 0; t < RPW; t++) part[t] += __shfl_xor_sync(0xffffffffu, part[t], o);
#pragma unroll
            for (int t = 0; t < RPW; t++) {
                const int i = grow(t);
                if (i < M && i > k && lane == j) {
                    const double w = fma(-Kc, hv[i], beta * (pbuf[i] - part[t]));
                    Vr[t] = sb * hv[i];
                    Wr[t] = w * isb;
                }
            }
            // the same for the panel rows k0 + pr > k, kept in every CTA (one warp per row)
            for (int pr = j + 1 + warp; pr < NB + 2 && k0 + pr < M; pr += 8) {
                const int i = k0 + pr;
                double q = fma(Vp[pr * NB + lane], bq, Wp[pr * NB + lane] * aq);
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) q += __shfl_xor_sync(0xffffffffu, q, o);
                if (lane == 0) {
                    const double w = fma(-Kc, hv[i], beta * (pbuf[i] - q));
                    Vp[pr * NB + j] = sb * hv[i];
                    Wp[pr * NB + j] = w * isb;
                }
            }
        }
        __syncthreads();
    }
    const bool last = M - 2 <= k0 + NB;
    if (last) {
        // the trailing 2 x 2 (or 1 x 1) with the panel's corrections
        auto corr = [&](int r1, int r2) {   // (V W^T + W V^T)[r1, r2], both panel rows
            double c = 0.0;
            const int p1 = r1 - k0, p2 = r2 - k0;
            if (p1 >= 0 && p2 >= 0 && p1 < NB + 2 && p2 < NB + 2)
                for (int q = 0; q < NB; q++)
                    c = fma(Vp[p1 * NB + q], Wp[p2 * NB + q], fma(Wp[p1 * NB + q], Vp[p2 * NB + q], c));
            return c;
        };
        if (tid == 0) {
            if (M >= 2) {
                if ((M - 2) % CL == rank) btd[M - 2] = rowp(M - 2)[M - 2] - corr(M - 2, M - 2);
                if ((M - 1) % CL == rank) {
                    btd[M - 1] = rowp(M - 1)[M - 1] - corr(M - 1, M - 1);
                    bte[M - 2] = rowp(M - 1)[M - 2] - corr(M - 1, M - 2);
                }
            } else if (rank == 0) {
                btd[0] = rowp(0)[0];
            }
            if (rank == 0) { bte[M - 1] = 0.0; if (M >= 2) btau[M - 2] = 0.0; btau[M - 1] = 0.0; }
        }
    } else {
        // operands of the trailing update A_ps -= [V W] [W V]^T, rows >= k0 + NB
#pragma unroll
        for (int t = 0; t < RPW; t++) {
            const int i = grow(t);
            if (i < M && i >= kend) {
                double *o1 = VW + ((size_t)b * Mmax + i) * 2 * NB, *o2 = WV + ((size_t)b * Mmax + i) * 2 * NB;
                o1[lane] = Vr[t]; o1[NB + lane] = Wr[t];
                o2[lane] = Wr[t]; o2[NB + lane] = Vr[t];
            }
        }
    }
    cluster.sync();   // keep every CTA's shared memory alive until remote writes are done
}

// ---- tridiagonal helpers -------------------------------------------------------------------

// ---- Sturm counts and Newton steps on a tridiagonal scaled to |d_i| <= 1, e2_i <= 1 -------------
//
// Number of eigenvalues of T (diagonal d, squared off-diagonal e2) below x, as the number of sign
// changes in the leading principal minors p_i of T - xI:
//   p_-1 = 1, p_0 = d_0 - x, p_i = (d_i - x) p_{i-1} - e2_{i-1} p_{i-2}   (Sturm sequence).
// A dependent FP64 instruction takes ~64 cycles on B300, so only the DFMA is on the step's
// dependent path: signs, the exact-zero rule (a zero minor takes the sign opposite to its
// predecessor, as the ratio form's -pivmin does) and the exponents are 32-bit integer work on the
// high words. |d_i - x| is clamped below at 2^-60 (a perturbation of T far below its rounding),
// which bounds how fast the minors can shrink (2^-113 per step, cancellation included); with the
// growth bounded by 4x per step, a renormalisation every four steps (both minors times the power
// of two that brings the larger to 2^0 once it leaves [2^-400, 2^400]) keeps every value normal.
__device__ __forceinline__ double clamp_dx(double dx)
{
    const int hi = __double2hiint(dx);
    return (((hi >> 20) & 0x7FF) < 1023 - 60) ? ((hi < 0) ? -0x1.0p-60 : 0x1.0p-60) : dx;
}

__device__ __forceinline__ int exp_of(double v) { return (__double2hiint(v) >> 20) & 0x7FF; }

template <int NP>
__device__ __forceinline__ void sturm_counts(const double *d, const double *e2, int M, const double (&x)[NP],
                                             int (&cnt)[NP])
{
    double pp[NP], pc[NP];
#pragma unroll
    for (int j = 0; j < NP; j++) {
        pp[j] = 1.0;
        pc[j] = clamp_dx(d[0] - x[j]);
        cnt[j] = __double2hiint(pc[j]) < 0;
    }
    // one step: the exact-zero substitute -2^-60 pc is built on the bit pattern (pc is normal)
    auto step = [&](int j, double dx, double fi) {
        double pn = fma(dx, pc[j], -fi * pp[j]);
        const int hc = __double2hiint(pc[j]), hn = __double2hiint(pn);
        const double alt = __hiloint2double((hc ^ (int)0x80000000) - (60 << 20), __double2loint(pc[j]));
        pn = (((hn & 0x7FFFFFFF) | __double2loint(pn)) == 0) ? alt : pn;
        cnt[j] += (int)((unsigned)(__double2hiint(pn) ^ hc) >> 31);
        pp[j] = pc[j];
        pc[j] = pn;
    };
    int i = 1;
    for (; i + 3 < M; i += 4) {                 // blocks of four: d - x and the loads go first
        double dx[4][NP], f[4];
#pragma unroll
        for (int u = 0; u < 4; u++) {
            f[u] = e2[i + u - 1];
#pragma unroll
            for (int j = 0; j < NP; j++) dx[u][j] = clamp_dx(d[i + u] - x[j]);
        }
#pragma unroll
        for (int u = 0; u < 4; u++) {
#pragma unroll
            for (int j = 0; j < NP; j++) step(j, dx[u][j], f[u]);
        }
#pragma unroll
        for (int j = 0; j < NP; j++) {
            const int em = max(exp_of(pc[j]), exp_of(pp[j]));
            if (em > 1023 + 400 || em < 1023 - 400) {
                const double sc = __hiloint2double((2046 - em) << 20, 0);   // 2^(1023 - em)
                pc[j] *= sc;
                pp[j] *= sc;
            }
        }
    }
    for (; i < M; i++) {                        // at most three steps after the last renormalisation
#pragma unroll
        for (int j = 0; j < NP; j++) step(j, clamp_dx(d[i] - x[j]), e2[i - 1]);
    }
}

__device__ __forceinline__ int sturm3f(const float *d, const float *e2, int M, float x)
{
    float pp = 1.0f, pc = d[0] - x;
    int bc = __float_as_int(pc);
    if ((bc << 1) == 0) { pc = -0x1.0p-30f; bc = __float_as_int(pc); }
    int cnt = bc < 0;
    for (int i = 1; i < M; i++) {
        float pn = fmaf(d[i] - x, pc, -e2[i - 1] * pp);
        int bn = __float_as_int(pn);
        if ((bn << 1) == 0) {
            pn = __int_as_float((bc & 0x7FFFFFFF) ^ (~bc & (int)0x80000000)) * 0x1.0p-30f;
            bn = __float_as_int(pn);
        }
        cnt += (int)(((unsigned)(bn ^ bc)) >> 31);
        const int ex = (bn >> 23) & 0xFF;
        if (ex > 127 + 48 || ex < 127 - 48) {
            const float sc = __int_as_float((254 - ex) << 23);                     // 2^(127 - ex)
            pn *= sc;
            pc *= sc;
            bn = __float_as_int(pn);
        }
        pp = pc;
        pc = pn;
        bc = bn;
    }
    return cnt;
}

// One Newton correction -p_M(x) / p_M'(x) for det(T - xI) (scaled T), from the three-term
// recurrence of the leading minors p_i = (d_i - x) p_{i-1} - e2_{i-1} p_{i-2} and of their
// derivatives p_i' = (d_i - x) p_{i-1}' - p_{i-1} - e2_{i-1} p_{i-2}' (d - x clamped as in
// sturm_counts), one DFMA per chain and step on the dependent path. The two chains are split
// over two warps, i.e. over two sub-partitions' FP64 pipes: warp 0 runs the p chain (three FP64
// instructions per step) and hands d_i - x and p_i to warp 1 through shared memory in chunks of
// kNewtonChunk steps; warp 1 runs the p' chain (two per step). Chunks are double-buffered; named
// barriers 1/2 mark a buffer full, 3/4 empty, and 5 ends the pass, after which both warps hold p_M
// and p_M' and return the same correction. Renormalisation (every fourth step, when the exponent of
// the larger of p_i, p_{i-1} leaves 2^(+-400)) is decided from the p values alone, which both warps
// see, and applied to both chains: exact powers of two, so the result is that of the unscaled
// recurrences. Every lane of both warps must call it the same number of times with the same M.
constexpr int kNewtonChunk = 16;

struct NewtonShared {
    double dx[2][kNewtonChunk][32];
    double p[2][kNewtonChunk][32];
    double pm[2][32], qm[2][32];                 // p_M and p_M' by pass parity
};

template <int ID> __device__ __forceinline__ void named_sync64() { asm volatile("bar.sync %0, 64;" ::"n"(ID) : "memory"); }
template <int ID> __device__ __forceinline__ void named_arrive64() { asm volatile("bar.arrive %0, 64;" ::"n"(ID) : "memory"); }

__device__ __forceinline__ double newton_step_split(const double *d, const double *e2, int M, double x, int warp,
                                                    int lane, int parity, NewtonShared &sh)
{
    const int nch = (M - 1 + kNewtonChunk - 1) / kNewtonChunk;   // steps i = 1 .. M-1
    double pc = clamp_dx(d[0] - x);
    // exponent field of the larger of two values, and whether it left 1023 +- 400 (integer tests)
    auto renorm_em = [](double a, double b, int &em) {
        em = max(exp_of(a), exp_of(b));
        return em > 1023 + 400 || em < 1023 - 400;
    };
    if (warp == 0) {
        double pp = 1.0;
        // step i from dx = d_i - x and f = e2_{i-1}; i = 0 mod 4 closes a block of four
        auto step = [&](int buf, int j, int i, double dx, double f) {
            const double pn = fma(dx, pc, -f * pp);
            sh.dx[buf][j][lane] = dx;
            sh.p[buf][j][lane] = pn;
            pp = pc;
            pc = pn;
            int em;
            if ((i & 3) == 0 && renorm_em(pc, pp, em)) {
                const double sc = __hiloint2double((2046 - em) << 20, 0);   // 2^(1023 - em)
                pc *= sc;
                pp *= sc;
            }
        };
        for (int c = 0; c < nch; c++) {
            const int buf = c & 1, i0 = 1 + c * kNewtonChunk, cnt = min(kNewtonChunk, M - i0);
            if (c >= 2) buf ? named_sync64<4>() : named_sync64<3>();   // warp 1 is done with chunk c - 2
            if (cnt == kNewtonChunk) {
#pragma unroll
                for (int g = 0; g < kNewtonChunk; g += 4) {          // loads and d - x of four steps first
                    double dx[4], f[4];
#pragma unroll
                    for (int u = 0; u < 4; u++) {
                        dx[u] = clamp_dx(d[i0 + g + u] - x);
                        f[u] = e2[i0 + g + u - 1];
                    }
#pragma unroll
                    for (int u = 0; u < 4; u++) step(buf, g + u, i0 + g + u, dx[u], f[u]);
                }
            } else {
                for (int j = 0; j < cnt; j++) step(buf, j, i0 + j, clamp_dx(d[i0 + j] - x), e2[i0 + j - 1]);
            }
            buf ? named_arrive64<2>() : named_arrive64<1>();
        }
        sh.pm[parity][lane] = pc;
    } else {
        double qp = 0.0, qc = -1.0;
        auto step = [&](int i, double dx, double pn, double f) {
            const double qn = fma(dx, qc, -fma(f, qp, pc));
            qp = qc;
            qc = qn;
            const double pprev = pc;
            pc = pn;
            int em;
            if ((i & 3) == 0 && renorm_em(pc, pprev, em)) {
                const double sc = __hiloint2double((2046 - em) << 20, 0);
                pc *= sc;
                qc *= sc;
                qp *= sc;
            }
        };
        for (int c = 0; c < nch; c++) {
            const int buf = c & 1, i0 = 1 + c * kNewtonChunk, cnt = min(kNewtonChunk, M - i0);
            buf ? named_sync64<2>() : named_sync64<1>();        // chunk c is in shared memory
            if (cnt == kNewtonChunk) {
#pragma unroll
                for (int g = 0; g < kNewtonChunk; g += 4) {
                    double dx[4], pn[4], f[4];
#pragma unroll
                    for (int u = 0; u < 4; u++) {
                        dx[u] = sh.dx[buf][g + u][lane];
                        pn[u] = sh.p[buf][g + u][lane];
                        f[u] = e2[i0 + g + u - 1];
                    }
#pragma unroll
                    for (int u = 0; u < 4; u++) step(i0 + g + u, dx[u], pn[u], f[u]);
                }
            } else {
                for (int j = 0; j < cnt; j++) step(i0 + j, sh.dx[buf][j][lane], sh.p[buf][j][lane], e2[i0 + j - 1]);
            }
            if (c < nch - 2) buf ? named_arrive64<4>() : named_arrive64<3>();   // warp 0 waits for chunks 2 .. nch-1
        }
        sh.qm[parity][lane] = qc;
    }
    named_sync64<5>();
    const double p = sh.pm[parity][lane], q = sh.qm[parity][lane];
    return (q != 0.0) ? -p / q : 0.0;
}

// The selected eigenvalues of T_b, the one at ascending position (k0 - s + t) for slice vector t.
// Grid (ceil(mmax / EPC), nb), 32 EPC threads (EPC warps, 8 <= EPC <= 32), EPC eigenvalues per CTA;
// the launch takes the smallest EPC that gives every CTA its own SM (step 3 runs on warps 0 and 1,
// one per sub-partition, and a second CTA's warps would share those sub-partitions' FP64 pipes):
//   1. T is scaled by the power of two that brings its Gershgorin span into [1/2, 1) (exact).
//   2. Warp w brackets eigenvalue w of the CTA by FP32 multisection: the 32 lanes count the
//      eigenvalues below 32 interior points of the bracket (33 subintervals), and the bracket
//      becomes the subinterval where the count passes the position; five rounds reach 8 FP32 ulps
//      of the span (a bisection needs twenty counts one after another).
//   3. Warps 0 and 1, one eigenvalue per lane (EPC lanes; the others repeat lane 0's): up to
//      three FP64 Newton steps on det(T - xI) from the bracket's midpoint (quadratic convergence
//      while |x - lambda| is far below the gap; the warps stop once every lane's correction is
//      below tol), each step's p and p' chains on the two warps (newton_step_split); then one
//      certifying FP64 Sturm count each, warp 0 at x - tol and warp 1 at x + tol, which place the
//      eigenvalue within tol = 4 ulp |x| + 2 ulp of the span. While a lane fails, both warps run
//      one more Newton step for it and count again (twice at most); a lane that still fails is
//      resolved by warp 0 with an FP64 multisection over its 32 lanes (on the widened FP32
//      bracket if its end counts enclose the position, else on the Gershgorin interval).
__global__ void __launch_bounds__(1024, 1)
k_bisect(const int32_t *__restrict__ plan, int32_t nb, int32_t Mmax, int32_t mmax,
         const double *__restrict__ td, const double *__restrict__ te, double *__restrict__ sel_val)
{
    const int b = blockIdx.y;
    const int k0 = plan[b], mb = plan[nb + b], s = plan[2 * nb + b], M = plan[3 * nb + b];
    const int EPC = blockDim.x >> 5;                      // eigenvalues per CTA
    if (blockIdx.x * EPC >= mb) return;                   // whole CTA
    extern __shared__ double smd[];
    double *d = smd, *e2 = smd + Mmax;
    float *df = reinterpret_cast<float *>(smd + 2 * Mmax), *e2f = df + Mmax;
    __shared__ double s_lo, s_hi, s_sc, s_isc;
    __shared__ float brlo[32], brhi[32];
    __shared__ int s_cnt[2][32];
    __shared__ NewtonShared s_newton;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const double *bd = td + (size_t)b * Mmax, *be = te + (size_t)b * Mmax;
    if (warp == 0) {
        double lo = INFINITY, hi = -INFINITY;
        for (int i = lane; i < M; i += 32) {
            const double r = (i > 0 ? fabs(be[i - 1]) : 0.0) + (i + 1 < M ? fabs(be[i]) : 0.0);
            lo = fmin(lo, bd[i] - r);
            hi = fmax(hi, bd[i] + r);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
            hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
        }
        if (lane == 0) {
            const double span = fmax(fabs(lo), fabs(hi));
            int e = 0;
            if (span > 0.0) frexp(span, &e);                // span = f 2^e, f in [1/2, 1)
            const double sc = ldexp(1.0, -e);
            s_sc = sc;
            s_isc = ldexp(1.0, e);
            const double sspan = span * sc;
            s_lo = lo * sc - 2.0 * DBL_EPSILON * sspan - DBL_MIN;
            s_hi = hi * sc + 2.0 * DBL_EPSILON * sspan + DBL_MIN;
        }
    }
    __syncthreads();
    const double sc = s_sc;
    for (int i = tid; i < M; i += blockDim.x) {
        const double di = bd[i] * sc, ei = (i + 1 < M) ? be[i] * sc : 0.0;
        d[i] = di;
        e2[i] = ei * ei;
        df[i] = (float)di;
        e2f[i] = (float)(ei * ei);
    }
    __syncthreads();
    const double sspan = fmax(fabs(s_lo), fabs(s_hi));
    // 2. FP32 multisection, warp w -> eigenvalue blockIdx.x * EPC + w
    {
        const int tw = blockIdx.x * EPC + warp;
        if (tw < mb) {
            const int pos = k0 - s + tw;
            float flo = (float)s_lo, fhi = (float)s_hi;
            const float ftol = 8.0f * FLT_EPSILON * (float)sspan;
            for (int r = 0; r < 8 && fhi - flo > ftol; r++) {
                const float w = (fhi - flo) * (1.0f / 33.0f);
                const float xl = fminf(fmaf(w, (float)(lane + 1), flo), fhi);
                const int cnt = sturm3f(df, e2f, M, xl);
                const unsigned above = __ballot_sync(0xffffffffu, cnt > pos);
                const int f = above ? __ffs(above) - 1 : 32;         // first point above the position
                const float xlo = __shfl_sync(0xffffffffu, xl, f > 0 ? f - 1 : 0);
                const float xhi = __shfl_sync(0xffffffffu, xl, f < 32 ? f : 31);
                if (f > 0) flo = xlo;
                if (f < 32) fhi = xhi;
            }
            if (lane == 0) { brlo[warp] = flo; brhi[warp] = fhi; }
        }
    }
    __syncthreads();
    if (warp > 1) return;
    // 3. FP64 refinement and certification, lane -> eigenvalue blockIdx.x * EPC + lane in both warps
    //    (every lane of both warps reaches the named barrier below: lanes without an eigenvalue
    //    repeat lane 0's)
    const bool valid = lane < EPC && blockIdx.x * EPC + lane < mb;
    const int ln = valid ? lane : 0;
    const int t = blockIdx.x * EPC + ln;
    const int pos = k0 - s + t;
    const double satol = DBL_EPSILON * sspan;
    const float flo = brlo[ln], fhi = brhi[ln];
    const double widen = 32.0 * FLT_EPSILON * sspan;
    const double blo = fmax(s_lo, (double)flo - widen), bhi = fmin(s_hi, (double)fhi + widen);
    double x = 0.5 * ((double)flo + (double)fhi);
    int npass = 0;
    for (int it = 0; it < 3; it++) {
        const double xn = x + newton_step_split(d, e2, M, x, warp, lane, npass++ & 1, s_newton);
        const bool inside = xn >= blo && xn <= bhi;  // else keep the last iterate
        const bool settled = !inside || fabs(xn - x) <= 4.0 * DBL_EPSILON * fabs(xn) + 2.0 * satol;
        if (inside) x = xn;
        if (__all_sync(0xffffffffu, settled)) break;
    }
    // certification: warp 0 counts at x - tol, warp 1 at x + tol, and both warps read both
    // counts, so they take the same decisions. While a lane fails (at most twice), both warps run
    // one more Newton step for the failing lanes and count again. (Barrier 6 is reused only
    // after a Newton step, whose barriers both warps pass after reading the counts.)
    double tol = 0.0;
    bool ok = false;
    for (int round = 0; round < 3; round++) {
        tol = 4.0 * DBL_EPSILON * fabs(x) + 2.0 * satol;
        const double xs[1] = {warp == 0 ? x - tol : x + tol};
        int cs1[1];
        sturm_counts<1>(d, e2, M, xs, cs1);
        s_cnt[warp][lane] = cs1[0];
        named_sync64<6>();                                        // warps 0 and 1, all lanes
        ok = s_cnt[0][lane] <= pos && s_cnt[1][lane] > pos;
        if (__all_sync(0xffffffffu, ok) || round == 2) break;
        const double xn = x + newton_step_split(d, e2, M, x, warp, lane, npass++ & 1, s_newton);
        if (!ok && xn >= blo && xn <= bhi) x = xn;
    }
    if (warp == 1) return;
    // lanes still uncertified: warp 0 resolves them one at a time by FP64 multisection over its
    // 32 lanes (31 subintervals per Sturm pass, about five bits, instead of one bit per pass of a
    // lane's bisection), on the widened FP32 bracket while its end counts enclose the position,
    // else on the Gershgorin interval
    unsigned fail = __ballot_sync(0xffffffffu, valid && !ok);
    while (fail) {
        const int src = __ffs(fail) - 1;
        fail &= fail - 1;
        const int ps = __shfl_sync(0xffffffffu, pos, src);
        double lo = __shfl_sync(0xffffffffu, blo, src), hi = __shfl_sync(0xffffffffu, bhi, src);
        bool gersh = false;
        for (int r = 0; r < 32; r++) {
            const double w = (hi - lo) * (1.0 / 31.0);
            const double xm[1] = {(lane == 31) ? hi : fma(w, (double)lane, lo)};
            int cm[1];
            sturm_counts<1>(d, e2, M, xm, cm);
            const unsigned above = __ballot_sync(0xffffffffu, cm[0] > ps);
            if ((above & 1u) || !(above >> 31)) {                // the ends do not enclose it
                if (gersh) break;
                lo = s_lo;
                hi = s_hi;
                gersh = true;
                continue;
            }
            const int f = __ffs(above) - 1;                       // first point above, >= 1
            const double nlo = __shfl_sync(0xffffffffu, xm[0], f - 1), nhi = __shfl_sync(0xffffffffu, xm[0], f);
            lo = nlo;
            hi = nhi;
            if (hi - lo <= 2.0 * DBL_EPSILON * fmax(fabs(lo), fabs(hi)) + satol) break;
        }
        if (lane == src) x = 0.5 * (lo + hi);
    }
    if (valid) sel_val[(size_t)b * mmax + t] = x * s_isc;
}

__device__ __forceinline__ double hash_unit(uint32_t a, uint32_t b, uint32_t c)
{
    uint64_t z = ((uint64_t)a << 42) ^ ((uint64_t)b << 21) ^ (uint64_t)c;
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    return ((double)(z >> 11) * 0x1.0p-53) * 2.0 - 1.0;   // (-1, 1)
}

// Bits of |x| and their comparison: for doubles of one sign the IEEE order is the integer order of
// the bit patterns, so pivot tests need no FP64 instruction (each costs a sub-partition's FP64
// pipe ~64 cycles on B300, the pace of a lane's whole dependent chain here).
__device__ __forceinline__ unsigned long long abs_bits(double x)
{
    return (unsigned long long)__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFull;
}

// Largest |z_i| exponent field of a lane's vector (element i at z[i * zst]), by integer max.
__device__ __forceinline__ int max_exponent(const double *z, size_t zst, int M)
{
    unsigned long long m = 0ull;
    for (int i = 0; i < M; i++) m = max(m, abs_bits(z[(size_t)i * zst]));
    return (int)(m >> 52);
}

// Grid (ceil(mmax / L), nb), L threads (L = 32, fewer for windows whose vectors would not fit in
// shared memory): lane t computes the unit eigenvector of T_b for the selected eigenvalue t by two
// inverse-iteration solves with a pivoted tridiagonal LU of T - lambda I (reciprocal pivots clamped
// to |pivot| >= eps ||T||). Members of a cluster (consecutive selected eigenvalues closer than
// gaptol) are computed one after another by the cluster's first lane and orthogonalised against
// each other (modified Gram-Schmidt) after every solve. The LU factors are written once per shift
// into global work arrays interleaved across lanes (element i of lane t at i * stride + t:
// coalesced), and only read by the solves; the vector z, which every sweep reads and rewrites,
// lives in shared memory (element i of lane t at i * L + t), so no load of z waits behind an L2
// round trip of the store before it. Windows too wide for 32 lanes' vectors in shared memory (ZG)
// keep z in a fifth global work array, interleaved like the factors, and every sweep over it loads
// a block of PB entries before it stores any, so a lane waits one L2 round trip per block instead
// of one per entry; the CTA then holds 32 lanes and the grid fits the GPU in one wave (with z in
// shared memory such windows ran 8 lanes per CTA, one CTA per SM, in eight waves).
// A lane's time is its count of FP64 instructions (~64 cycles each on its sub-partition), so: the
// first solve's forward elimination runs inside the factorisation, pivot tests compare bit
// patterns, a step computes only the taken branch, every lane starts from one random vector of the
// window (cluster members after the first from their own), and the vector is normalised once,
// after the second solve, with power-of-two rescaling by integer exponent tests guarding the range.
template <bool ZG>
__global__ void k_inverse_iter(const int32_t *__restrict__ plan, int32_t nb, int32_t Mmax,
                               int32_t mmax, const double *__restrict__ td,
                               const double *__restrict__ te, const double *__restrict__ sel_val,
                               double *__restrict__ sel_vec, double *__restrict__ work)
{
    constexpr int PB = 8;                                   // prefetch block of the solves
    const int b = blockIdx.y;
    const int mb = plan[nb + b], M = plan[3 * nb + b];
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    extern __shared__ double zsm[];
    const size_t stride = (size_t)nb * mmax;
    const size_t me = (size_t)b * mmax + t;
    // element i of the lane's vector at z[i * zst]: shared memory, or the fifth work array
    const size_t zst = ZG ? stride : (size_t)blockDim.x;
    double *z = ZG ? work + 4 * stride * Mmax + me : zsm + threadIdx.x;
    double *d = zsm + (ZG ? 0 : (size_t)blockDim.x * Mmax); // the window's T, shared by the lanes
    double *e = d + Mmax;
    double *rv = e + Mmax;                                  // the window's start vector
    __shared__ double tn_part[32];
    {
        const double *gd = td + (size_t)b * Mmax, *ge = te + (size_t)b * Mmax;
        double part = 0.0;
        for (int i = threadIdx.x; i < M; i += blockDim.x) {
            const double di = gd[i], ei = ge[i], em = (i > 0) ? ge[i - 1] : 0.0;
            d[i] = di;
            e[i] = ei;
            rv[i] = hash_unit(b, 0x5EED, i);
            part = fmax(part, fabs(di) + fabs(em) + (i + 1 < M ? fabs(ei) : 0.0));
        }
        tn_part[threadIdx.x] = part;
    }
    __syncthreads();
    double tnorm = 0.0;
    for (int q = 0; q < (int)blockDim.x; q++) tnorm = fmax(tnorm, tn_part[q]);
    if (t >= mb) return;
    const double *lam = sel_val + (size_t)b * mmax;
    const double gaptol = 1e-9 * fmax(tnorm, DBL_MIN);
    if (t > 0 && lam[t] - lam[t - 1] < gaptol) return;     // handled by the cluster's first lane
    double *__restrict__ u0 = work + me;                    // reciprocal pivots
    double *__restrict__ u1 = work + stride * Mmax + me;
    double *__restrict__ u2 = work + 2 * stride * Mmax + me;
    double *__restrict__ lm = work + 3 * stride * Mmax + me; // multipliers, sign bit = row swap
    const double pert = DBL_EPSILON * fmax(tnorm, DBL_MIN);
    const unsigned long long pert_bits = abs_bits(pert);
    // pivot clamped to |pivot| >= pert with its sign kept, by bit operations
    auto clamp_pivot = [&](double piv) {
        const unsigned long long pb = (unsigned long long)__double_as_longlong(piv);
        return ((pb & 0x7FFFFFFFFFFFFFFFull) >= pert_bits) ? piv
               : __longlong_as_double((long long)((pb & 0x8000000000000000ull) | pert_bits));
    };
    // z *= 2^-s when the largest exponent is far from 1 (keeps |z|^2 sums inside the FP64 range)
    auto rescale = [&]() {
        const int ex = max_exponent(z, zst, M) - 1023;
        if (ex > 400 || (ex < -400 && ex > -1023)) {
            const double f = ldexp(1.0, -ex);
            for (int i = 0; i < M; i++) z[i * zst] *= f;
        }
    };
    // dst[i] = z[i] * f for i < M (dst = z allowed), a block of PB loads before its stores
    auto scale_to = [&](double *dst, size_t dst_st, double f) {
        for (int i0 = 0; i0 < M; i0 += PB) {
            double zb[PB];
#pragma unroll
            for (int q2 = 0; q2 < PB; q2++) zb[q2] = (i0 + q2 < M) ? z[(size_t)(i0 + q2) * zst] : 0.0;
#pragma unroll
            for (int q2 = 0; q2 < PB; q2++)
                if (i0 + q2 < M) dst[(size_t)(i0 + q2) * dst_st] = zb[q2] * f;
        }
    };
    int last = t;
    while (last + 1 < mb && lam[last + 1] - lam[last] < gaptol) last++;
    for (int j = t; j <= last; j++) {
        const double x = lam[j];
        // start vector: the window's, or a cluster member's own (read by the elimination below)
        auto start = [&](int i) { return (j == t) ? rv[i] : hash_unit(b, j, i); };
        // pivoted LU of T - x I with the first solve's forward elimination: rows (p, q) = entries
        // at columns (i, i+1) of the pivot candidate, zi its right-hand side. The row-swap flag is
        // kept in the lowest mantissa bit of the stored multiplier (a 1-ulp change).
        double p = d[0] - x, q = (M > 1) ? e[0] : 0.0, zi = start(0);
#pragma unroll 4
        for (int i = 0; i + 1 < M; i++) {
            const double ei = e[i], an = d[i + 1] - x, en = (i + 2 < M) ? e[i + 1] : 0.0;
            const double zn = start(i + 1);
            const bool swp = abs_bits(p) < abs_bits(ei);
            const double rp = fast_rcp(clamp_pivot(swp ? ei : p));
            const double l = (swp ? p : ei) * rp;
            u0[i * stride] = rp;
            u1[i * stride] = swp ? an : q;
            u2[i * stride] = swp ? en : 0.0;
            const long long lb = __double_as_longlong(l);
            lm[i * stride] = __longlong_as_double(swp ? (lb | 1ll) : (lb & ~1ll));
            const double np = fma(-l, swp ? an : q, swp ? q : an);
            q = swp ? -l * en : en;
            p = np;
            z[i * zst] = swp ? zn : zi;
            zi = fma(-l, swp ? zn : zi, swp ? zi : zn);
        }
        u0[(size_t)(M - 1) * stride] = fast_rcp(clamp_pivot(p));
        u1[(size_t)(M - 1) * stride] = 0.0;      // read (times zero) by the back substitution
        u2[(size_t)(M - 1) * stride] = 0.0;
        z[(size_t)(M - 1) * zst] = zi;
        for (int it = 0; it < 2; it++) {
            if (it > 0) {
                // forward: replay the row operations on the right-hand side; the multipliers of a
                // block of PB rows are loaded together (one L2 round trip per block)
                double zf = z[0];
                for (int i0 = 0; i0 + 1 < M; i0 += PB) {
                    double lr[PB], zb[PB];
#pragma unroll
                    for (int q2 = 0; q2 < PB; q2++) {
                        const bool ok = i0 + q2 + 1 < M;
                        lr[q2] = ok ? lm[(size_t)(i0 + q2) * stride] : 0.0;
                        zb[q2] = ok ? z[(size_t)(i0 + q2 + 1) * zst] : 0.0;    // before this block's stores
                    }
#pragma unroll
                    for (int q2 = 0; q2 < PB; q2++) {
                        const int i = i0 + q2;
                        if (i + 1 < M) {
                            const double lraw = lr[q2];
                            const bool swp = (__double_as_longlong(lraw) & 1ll) != 0;
                            const double zn = zb[q2];
                            z[i * zst] = swp ? zn : zf;
                            zf = fma(-lraw, swp ? zn : zf, swp ? zf : zn);   // flag bit: <= 1 ulp of l
                        }
                    }
                }
                z[(size_t)(M - 1) * zst] = zf;
            }
            // back substitution with the three upper diagonals, factors loaded a block at a time
            double z1 = 0.0, z2 = 0.0;
            for (int i0 = M - 1; i0 >= 0; i0 -= PB) {
                double a0[PB], a1[PB], a2[PB], zb[PB];
#pragma unroll
                for (int q2 = 0; q2 < PB; q2++) {
                    const int i = i0 - q2;
                    const bool ok = i >= 0;
                    a0[q2] = ok ? u0[(size_t)i * stride] : 0.0;
                    a1[q2] = ok ? u1[(size_t)i * stride] : 0.0;
                    a2[q2] = ok ? u2[(size_t)i * stride] : 0.0;
                    zb[q2] = ok ? z[(size_t)i * zst] : 0.0;
                }
#pragma unroll
                for (int q2 = 0; q2 < PB; q2++) {
                    const int i = i0 - q2;
                    if (i >= 0) {
                        const double acc = fma(-a2[q2], z2, fma(-a1[q2], z1, zb[q2]));
                        const double zi2 = acc * a0[q2];
                        z[i * zst] = zi2;
                        z2 = z1;
                        z1 = zi2;
                    }
                }
            }
            rescale();
            const bool member = j > t;
            if (!member && it == 0) continue;            // one normalisation, after the second solve
            // orthogonalise against earlier cluster members, then normalise
            for (int c = t; c < j; c++) {
                const double *zc = sel_vec + ((size_t)b * mmax + c) * Mmax;
                double dot = 0.0;
                for (int i = 0; i < M; i++) dot = fma(zc[i], z[i * zst], dot);
                for (int i = 0; i < M; i++) z[i * zst] = fma(-dot, zc[i], z[i * zst]);
            }
            if (member) rescale();
            // four independent chains: a dependent FP64 instruction waits ~64 cycles on B300
            double n0 = 0.0, n1 = 0.0, n2 = 0.0, n3 = 0.0;
            int i4 = 0;
            for (; i4 + 3 < M; i4 += 4) {
                const double v0 = z[i4 * zst], v1 = z[(i4 + 1) * zst];
                const double v2 = z[(i4 + 2) * zst], v3 = z[(i4 + 3) * zst];
                n0 = fma(v0, v0, n0); n1 = fma(v1, v1, n1); n2 = fma(v2, v2, n2); n3 = fma(v3, v3, n3);
            }
            for (; i4 < M; i4++) { const double v = z[i4 * zst]; n0 = fma(v, v, n0); }
            const double nn = (n0 + n1) + (n2 + n3);
            if (!(nn > 0.0) || !(nn < INFINITY)) {
                for (int i = 0; i < M; i++) z[i * zst] = hash_unit(b, j + 7919, i + it);
                if (it == 1) scale_to(sel_vec + ((size_t)b * mmax + j) * Mmax, 1, 1.0);
                continue;
            }
            const double inr = rsqrt(nn);
            if (it == 1) {
                scale_to(sel_vec + ((size_t)b * mmax + j) * Mmax, 1, inr);    // the unit vector out
            } else {
                scale_to(z, zst, inr);                                        // a member's next solve
            }
        }
    }
}

__device__ __forceinline__ void cp_async8(double *dst, const double *src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src)
                 : "memory");
}

// z_j -= bk (v . z_j) v (entries k+1 .. M-1) for a warp's NVW vectors, lanes along the rows; the
// NVW dot products are summed over the lanes by one transpose-reduce (halving the values held per
// lane while the lane groups shrink), then broadcast from a lane holding each sum.
template <int NVW>
__device__ __forceinline__ void reflect(const double *__restrict__ v, double bk, double *const *z, int k, int M,
                                        int lane)
{
    double a[NVW];
#pragma unroll
    for (int j = 0; j < NVW; j++) a[j] = 0.0;
    for (int i = k + 1 + lane; i < M; i += 32) {
        const double vi = v[i];
#pragma unroll
        for (int j = 0; j < NVW; j++) a[j] = fma(vi, z[j][i], a[j]);
    }
    double f[NVW];
    if constexpr (NVW == 1) {
        double t = a[0];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        f[0] = bk * t;
    } else if constexpr (NVW == 2) {
        // lanes 0-15 end with the sum of vector 0, lanes 16-31 with that of vector 1
        const bool up = (lane & 16) != 0;
        double t = (up ? a[1] : a[0]) + __shfl_xor_sync(0xffffffffu, up ? a[0] : a[1], 16);
#pragma unroll
        for (int o = 8; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        const double fl = bk * t;
        f[0] = __shfl_sync(0xffffffffu, fl, 0);
        f[1] = __shfl_sync(0xffffffffu, fl, 16);
    } else {
        // lanes end with the sum of vector (lane >> 3) & 3: halve at offsets 16 and 8, then
        // butterflies over the lower three lane bits
        double b[4];
#pragma unroll
        for (int j = 0; j < 4; j++) b[j] = (j < NVW) ? a[j < NVW ? j : 0] : 0.0;
        {
            const bool up = (lane & 16) != 0;
            const double s0 = up ? b[0] : b[2], s1 = up ? b[1] : b[3];
            const double k0v = up ? b[2] : b[0], k1v = up ? b[3] : b[1];
            b[0] = k0v + __shfl_xor_sync(0xffffffffu, s0, 16);
            b[1] = k1v + __shfl_xor_sync(0xffffffffu, s1, 16);
        }
        {
            const bool up = (lane & 8) != 0;
            const double s0 = up ? b[0] : b[1], k0v = up ? b[1] : b[0];
            b[0] = k0v + __shfl_xor_sync(0xffffffffu, s0, 8);
        }
        b[0] += __shfl_xor_sync(0xffffffffu, b[0], 4);
        b[0] += __shfl_xor_sync(0xffffffffu, b[0], 2);
        b[0] += __shfl_xor_sync(0xffffffffu, b[0], 1);
        const double fl = bk * b[0];
#pragma unroll
        for (int j = 0; j < NVW; j++) f[j] = __shfl_sync(0xffffffffu, fl, 8 * j);
    }
    for (int i = k + 1 + lane; i < M; i += 32) {
        const double vi = v[i];
#pragma unroll
        for (int j = 0; j < NVW; j++) z[j][i] = fma(-f[j], vi, z[j][i]);
    }
}

// Back-transform y = H_0 H_1 ... H_{M-3} z of the selected eigenvectors z of T_b, then the sign
// rule, zero padding to length N, the shift eps and the step alpha, written straight into X.
// One-dimensional grid, 32 NW threads: window b owns ceil(m_b / vpc) consecutive CTAs, each taking
// up to vpc <= NW NV consecutive vectors of the window, warp w the vectors w, w+NW, ... (NV per
// warp, lanes along the rows). The work is the FP64 pipe's (2 (M - k) FMAs per reflector and
// vector), so the launch gives every SM at most one CTA; with NW = 8 two warps share each
// sub-partition (one's dot-reduce-update chain hides behind the other's FMAs) and a
// sub-partition holds at most three vectors (vpc <= 10). The reflectors pass through shared memory
// in double-buffered chunks of KC rows (cp.async, shared by the CTA's warps), and the NV dot
// products of a reflector are summed over the lanes by one transpose-reduce. A warp applies the
// reflectors to its real vectors only (the FP64 pipe is the bound: unused slots cost nothing).
template <int NV, int NW>
__global__ void __launch_bounds__(32 * NW, 1)
k_backtransform(const int32_t *__restrict__ plan, int32_t nb, int64_t N, int32_t Mmax, int32_t mmax,
                const double *__restrict__ refl, const double *__restrict__ tau,
                const double *__restrict__ sel_val, const double *__restrict__ sel_vec,
                const double *__restrict__ gersh, double alpha_theta, int vpc, int kc,
                double *__restrict__ X, double *__restrict__ eps, double *__restrict__ alpha)
{
    static_assert(NV >= 1 && NV <= 4, "at most four vectors per warp");
    // CTA c takes chunk c - first_b of window b, where window b owns ceil(m_b / vpc) chunks
    int b = -1, tbeg = 0;
    for (int q = 0, first = 0; q < nb; q++) {
        const int cnt = (plan[nb + q] + vpc - 1) / vpc;
        if ((int)blockIdx.x < first + cnt) { b = q; tbeg = ((int)blockIdx.x - first) * vpc; break; }
        first += cnt;
    }
    if (b < 0) return;                                    // whole CTA: beyond the last chunk
    const int k0 = plan[b], mb = plan[nb + b], s = plan[2 * nb + b], M = plan[3 * nb + b];
    const int nvc = min(vpc, mb - tbeg);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    extern __shared__ double smb[];
    double *zs = smb;                                     // [NW NV][Mmax] vector slots (slot w + NW j)
    double *ts = zs + (size_t)NW * NV * Mmax;             // [Mmax] tau
    double *rs = ts + Mmax;                               // [2][kc][Mmax] reflector chunks
    const double *brefl = refl + (size_t)b * Mmax * Mmax;
    for (int q = 0; q < NW * NV; q++) {
        const double *src = sel_vec + ((size_t)b * mmax + tbeg + q) * Mmax;
        for (int i = tid; i < M; i += blockDim.x) zs[(size_t)q * Mmax + i] = (q < nvc) ? src[i] : 0.0;
    }
    for (int i = tid; i < M; i += blockDim.x) ts[i] = tau[(size_t)b * Mmax + i];
    double *z[NV];
    int nvw = 0;                                          // the warp's vectors: slots 0 .. nvw-1
#pragma unroll
    for (int j = 0; j < NV; j++) {
        z[j] = zs + (size_t)(warp + NW * j) * Mmax;
        nvw += (warp + NW * j < nvc) ? 1 : 0;
    }
    const int nk = M - 2;                                 // reflectors k = M-3 .. 0
    const int nch = nk > 0 ? (nk + kc - 1) / kc : 0;
    auto issue = [&](int c) {
        double *dst = rs + (size_t)(c & 1) * kc * Mmax;
        const int khi = M - 3 - c * kc;
        for (int r = 0; r < kc; r++) {
            const int k = khi - r;
            if (k < 0) break;
            for (int i = k + 1 + tid; i < M; i += blockDim.x) cp_async8(dst + (size_t)r * Mmax + i, brefl + (size_t)k * Mmax + i);
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    if (nch > 0) issue(0);
    for (int c = 0; c < nch; c++) {
        if (c + 1 < nch) {
            issue(c + 1);
            asm volatile("cp.async.wait_group 1;" ::: "memory");
        } else {
            asm volatile("cp.async.wait_group 0;" ::: "memory");
        }
        __syncthreads();
        const double *cb = rs + (size_t)(c & 1) * kc * Mmax;
        const int khi = M - 3 - c * kc;
        for (int r = 0; r < kc; r++) {
            const int k = khi - r;
            if (k < 0) break;
            const double bk = ts[k];
            if (bk == 0.0) continue;
            const double *v = cb + (size_t)r * Mmax;
            if (nvw == NV) reflect<NV>(v, bk, z, k, M, lane);
            else if (NV > 1 && nvw == 1) reflect<1>(v, bk, z, k, M, lane);
            else if (NV > 2 && nvw == 2) reflect<(NV > 2 ? 2 : 1)>(v, bk, z, k, M, lane);
            else if (NV > 3 && nvw == 3) reflect<(NV > 3 ? 3 : 1)>(v, bk, z, k, M, lane);
            __syncwarp();
        }
        __syncthreads();                                  // chunk c's buffer is reloaded next
    }
    // sign rule: home component positive when |y_home| >= 0.1, else the largest component
    const double glo = gersh[2 * N], ghi = gersh[2 * N + 1];
#pragma unroll
    for (int j = 0; j < NV; j++) {
        const int lt = warp + NW * j;
        if (lt >= nvc) break;                             // warp-uniform
        const int t = tbeg + lt;
        const double *zz = z[j];
        const int home = k0 - s + t;
        double best = -1.0;
        int arg = M;
        for (int i = lane; i < M; i += 32) {
            const double av = fabs(zz[i]);
            if (av > best) { best = av; arg = i; }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const double ob = __shfl_xor_sync(0xffffffffu, best, o);
            const int oa = __shfl_xor_sync(0xffffffffu, arg, o);
            if (ob > best || (ob == best && oa < arg)) { best = ob; arg = oa; }
        }
        const double yh = zz[home];
        const double ref = (fabs(yh) >= 0.1) ? yh : zz[arg];
        const double flip = (ref < 0.0) ? -1.0 : 1.0;
        const int64_t kg = k0 + t;
        double *xr = X + kg * N;
        for (int64_t jj = lane; jj < N; jj += 32) {
            const int64_t li = jj - s;
            xr[jj] = (li >= 0 && li < M) ? flip * zz[li] : 0.0;
        }
        if (lane == 0) {
            const double lam = sel_val[(size_t)b * mmax + t];
            const double dmax = fmax(ghi - lam, lam - glo);
            const double av = alpha_theta / (dmax * dmax);
            const double cap = 1.0 - 0x1.0p-20;
            eps[kg] = lam;
            alpha[kg] = (av < cap) ? av : cap;
        }
    }
}

// Shared memory of k_backtransform<NV, NW> with chunks of kc reflectors.
size_t backtransform_smem(int Mmax, int nv, int nw, int kc)
{
    return ((size_t)nw * nv * Mmax + Mmax + (size_t)2 * kc * Mmax) * sizeof(double);
}

// Function attributes are process-wide while handles differ in window size, so every attribute
// is set to the device maximum (what a launch actually requests still sets its occupancy).
// Cluster size of the window reduction: B300 runs clusters of up to 16 CTAs (any size, 9-16 as
// non-portable), but a cluster must fit in one GPC, so how many clusters of a given size run at
// once depends on the GPC layout; the occupancy query answers it. Per-window time goes with the
// rows each CTA owns (its share of the FP64 work) plus a per-step barrier cost that grows with
// the cluster; windows beyond the co-resident count wait for a second wave. Chooses the size
// with the least waves x (rows per CTA + 3.3 x cluster size), rows in shared memory when they
// fit. The 3.3 is fitted to B300 timings of ten 384-row windows: 8, 9, 10 and 16 CTAs took 4.35,
// 4.22, 4.07 and 4.61 ms in one wave; 11, 12 and 14 fit nine clusters at a time and took 7.6-8.0.
cudaError_t select_tridiag_cluster(pfsm_handle_s *h, size_t smem_cap)
{
    const int Mx = h->Mmax, nb = h->nb;
    double best = 1e300;
    int best_cl = 16;
    bool best_smem = false;
    for (int cl = 16; cl >= 2; cl--) {
        const size_t R = (size_t)((Mx + cl - 1) / cl);
        const bool in_smem = tri_smem_bytes(Mx, cl, true) <= smem_cap;
        const size_t smem = tri_smem_bytes(Mx, cl, in_smem);
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)(nb * cl));
        cfg.blockDim = dim3(kTriLaThreads);
        cfg.dynamicSmemBytes = smem;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = cl;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        int active = 0;
        cudaError_t e = in_smem ? cudaOccupancyMaxActiveClusters(&active, k_tridiag<true>, &cfg)
                                : cudaOccupancyMaxActiveClusters(&active, k_tridiag<false>, &cfg);
        if (e != cudaSuccess || active < 1) {
            cudaGetLastError();
            continue;
        }
        const int waves = (nb + active - 1) / active;
        const double cost = waves * ((double)R + 3.3 * cl) * (in_smem ? 1.0 : 1.5);
        if (cost < best) { best = cost; best_cl = cl; best_smem = in_smem; }
    }
    if (best == 1e300) return cudaErrorInvalidConfiguration;
    h->cl = best_cl;
    h->rows_in_smem = best_smem;
    return cudaSuccess;
}

cudaError_t configure_kernels(pfsm_handle_s *h)
{
    (void)h;
    int dev = 0, cap = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&cap, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) != cudaSuccess) return e;
    // dynamic limit = opt-in maximum minus the kernel's own static shared memory
    auto set_max = [&](const void *fn) -> cudaError_t {
        cudaFuncAttributes fa;
        cudaError_t r = cudaFuncGetAttributes(&fa, fn);
        if (r != cudaSuccess) return r;
        return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, cap - (int)fa.sharedSizeBytes);
    };
    if ((e = set_max((const void *)k_tridiag<true>)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_tridiag<true>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1)) != cudaSuccess) return e;
    if ((e = set_max((const void *)k_tridiag<false>)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_tridiag<false>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1)) != cudaSuccess) return e;
    if ((e = set_max((const void *)k_tridiag_panel<8>)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_tridiag_panel<8>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1)) != cudaSuccess) return e;
    if ((e = set_max((const void *)k_tridiag_panel<24>)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_tridiag_panel<24>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1)) != cudaSuccess) return e;
    if ((e = set_max((const void *)k_bisect)) != cudaSuccess) return e;
    if ((e = set_max((const void *)k_inverse_iter<false>)) != cudaSuccess) return e;
    if ((e = set_max((const void *)k_inverse_iter<true>)) != cudaSuccess) return e;
    if ((e = set_max((const void *)k_backtransform<1, 4>)) != cudaSuccess) return e;
    if ((e = set_max((const void *)k_backtransform<2, 4>)) != cudaSuccess) return e;
    return set_max((const void *)k_backtransform<2, 8>);
}

cudaError_t launch_subeig(pfsm_handle_s *h, const double *A, cudaStream_t st)
{
    Workspace &w = h->ws;
    const int nb = h->nb, Mmax = h->Mmax, mmax = h->mmax, CL = h->cl;
    cudaError_t e0;
    // mixed forms: work that needs only A (the Eq. 11 operand split) joins the side stream from here
    // and runs beside the window reduction, which leaves SMs idle; it is enqueued after the
    // reduction's launch so that the reduction's clusters are placed first
    const bool side_e = h->side && h->prm.precision != PFSM_FP64 && !h->prm.fs_adaptive && h->prm.fs_iters > 0;
    if (side_e && (e0 = cudaEventRecord(h->fork_ev, st)) != cudaSuccess) return e0;
    // 1. tridiagonalisation: two stages (mixed forms, wide windows: k_band.cu), or one cluster
    //    per window
    if (h->tri_two_stage) {
        if ((e0 = launch_band_reduction(h, A, st)) != cudaSuccess) return e0;
    } else if (h->tri_blocked) {
        // blocked: one panel launch per kPanel columns, the trailing update as a batched digit
        // product A_ps[k1:, k1:] -= [V W] [W V]^T per window (FP64-accurate, tensor cores)
        const size_t smem = tri_panel_smem(Mmax, CL, h->tri_mcap);
        const int64_t srows = (int64_t)nb * Mmax;
        SliceBuf dP{w.tdP, srows, 2 * kPanel, OZ_SLICES, 0}, dQ{w.tdQ, srows, 2 * kPanel, OZ_SLICES, 0};
        for (int k0 = 0; k0 == 0 || k0 < Mmax - 2; k0 += kPanel) {
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3((unsigned)(nb * CL));
            cfg.blockDim = dim3(kTriThreads);
            cfg.dynamicSmemBytes = smem;
            cfg.stream = st;
            cudaLaunchAttribute attr[1];
            attr[0].id = cudaLaunchAttributeClusterDimension;
            attr[0].val.clusterDim.x = CL;
            attr[0].val.clusterDim.y = 1;
            attr[0].val.clusterDim.z = 1;
            cfg.attrs = attr;
            cfg.numAttrs = 1;
            cudaError_t e;
            if (h->tri_rpw == 8)
                e = counted(cudaLaunchKernelEx(&cfg, k_tridiag_panel<8>, A, h->N, (const int32_t *)w.plan, nb, Mmax,
                                               h->tri_mcap, k0, w.iiwork, w.refl, w.tau, w.td, w.te, w.VW, w.WV));
            else
                e = counted(cudaLaunchKernelEx(&cfg, k_tridiag_panel<24>, A, h->N, (const int32_t *)w.plan, nb, Mmax,
                                               h->tri_mcap, k0, w.iiwork, w.refl, w.tau, w.td, w.te, w.VW, w.WV));
            if (e != cudaSuccess) return e;
            const int k1 = k0 + kPanel;
            if (k1 >= Mmax - 2) break;                 // every window ended in this panel
            if ((e = launch_oz_split(w.VW, srows, 2 * kPanel, 2 * kPanel, dP, w.tdeP, st)) != cudaSuccess) return e;
            if ((e = launch_oz_split(w.WV, srows, 2 * kPanel, 2 * kPanel, dQ, w.tdeQ, st)) != cudaSuccess) return e;
            OzParams o{};
            o.rows = Mmax; o.cols = Mmax; o.C = w.iiwork; o.ldc = Mmax; o.sub = 1; o.status = w.status;
            o.zrow = Mmax; o.zc = (int64_t)Mmax * Mmax; o.row_base = k1; o.ext = w.plan + 3 * nb;
            if ((e = launch_gemm_oz(dP, w.tdeP, dQ, w.tdeQ, o, st, nb)) != cudaSuccess) return e;
        }
    } else {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)(nb * CL));
        cfg.blockDim = dim3(kTriLaThreads);
        cfg.dynamicSmemBytes = tri_smem_bytes(Mmax, CL, h->rows_in_smem);
        cfg.stream = st;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = CL;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        cudaError_t e;
        if (h->rows_in_smem)
            e = counted(cudaLaunchKernelEx(&cfg, k_tridiag<true>, A, h->N, (const int32_t *)w.plan, nb, Mmax,
                                   (double *)nullptr, w.refl, w.tau, w.td, w.te));
        else
            e = counted(cudaLaunchKernelEx(&cfg, k_tridiag<false>, A, h->N, (const int32_t *)w.plan, nb, Mmax,
                                   w.iiwork, w.refl, w.tau, w.td, w.te));
        if (e != cudaSuccess) return e;
    }
    if (side_e) {
        const int64_t ld = padded_ld(h->N);
        const SliceBuf sE{w.slE, h->N, ld, slices_for(h->prm.precision), slice_kind(h->prm.precision)};
        if ((e0 = cudaStreamWaitEvent(h->side, h->fork_ev, 0)) != cudaSuccess) return e0;
        if ((e0 = launch_split(A, h->N, h->N, h->N, sE, true, w.dA, h->side)) != cudaSuccess) return e0;
        const SliceBuf da{w.ozA, h->N, ld, OZ_SLICES, 0};      // A' digits for the Rayleigh product
        if ((e0 = launch_oz_split(A, h->N, h->N, h->N, da, w.ozeA, h->side, true, w.dA)) != cudaSuccess) return e0;
        h->a_split = true;
        if ((e0 = cudaEventRecord(h->join_ev, h->side)) != cudaSuccess) return e0;
        h->side_pending = true;
    }
    // mixed forms: the back-transform's steps that need only the reflectors run on the side
    // stream beside the eigenvalue and inverse-iteration kernels (one warp per SM)
    const bool side_bt = h->prm.precision != PFSM_FP64 && w.btG && h->side && !h->tri_two_stage;
    if (side_bt) {
        if ((e0 = cudaEventRecord(h->fork_ev, st)) != cudaSuccess) return e0;
        if ((e0 = cudaStreamWaitEvent(h->side, h->fork_ev, 0)) != cudaSuccess) return e0;
        if ((e0 = launch_backtransform_wy_reflectors(h, h->side)) != cudaSuccess) return e0;
        if ((e0 = cudaEventRecord(h->join_ev, h->side)) != cudaSuccess) return e0;
        h->side_pending = true;
    }
    // one eigenpair per lane, full warps (a warp-wide FP64 instruction costs the same with 1 or
    // 32 active lanes)
    const int tpb = 32;
    if (h->timing && (e0 = cudaEventRecord(h->sub_ev[0], st)) != cudaSuccess) return e0;
    // 2. eigenvalues
    {
        // eigenvalues per CTA: the fewest (>= 8) that keep the CTAs within one per SM
        int epc = 8;
        while (epc < 32 && (int64_t)nb * ((mmax + epc - 1) / epc) > (int64_t)sm_count()) epc++;
        dim3 grid((unsigned)((mmax + epc - 1) / epc), (unsigned)nb);
        k_bisect<<<grid, 32 * epc, (size_t)3 * Mmax * sizeof(double), st>>>(w.plan, nb, Mmax, mmax, w.td, w.te,
                                                                           w.sel_val);
        g_launches++;
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    if (h->timing && (e0 = cudaEventRecord(h->sub_ev[1], st)) != cudaSuccess) return e0;
    // 3. inverse iteration
    {
        // the lanes' vectors in shared memory when 32 lanes' fit, else in the fifth work array
        const bool zg = (size_t)(tpb + 3) * Mmax * sizeof(double) > kInvSmemCap;
        const int lanes = tpb;
        const size_t smem = (size_t)(zg ? 3 : lanes + 3) * Mmax * sizeof(double);
        dim3 grid((unsigned)((mmax + lanes - 1) / lanes), (unsigned)nb);
        if (zg)
            k_inverse_iter<true><<<grid, lanes, smem, st>>>(w.plan, nb, Mmax, mmax, w.td, w.te, w.sel_val, w.sel_vec,
                                                           w.iiwork);
        else
            k_inverse_iter<false><<<grid, lanes, smem, st>>>(w.plan, nb, Mmax, mmax, w.td, w.te, w.sel_val, w.sel_vec,
                                                            w.iiwork);
        g_launches++;
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    if (h->timing && (e0 = cudaEventRecord(h->sub_ev[2], st)) != cudaSuccess) return e0;
    // 4. back-transform + start vectors: the mixed forms apply the reflectors in compact-WY form
    //    with digit products on the tensor cores (k_bt_wy.cu), after the bulge-chasing reflectors
    //    when the reduction had two stages; the FP64 form one by one on the FP64 pipe
    if (h->tri_two_stage) return launch_band_backtransform(h, st);
    if (h->prm.precision != PFSM_FP64 && w.btG) return launch_backtransform_wy(h, st, side_bt);
    {
        // vectors per CTA: the fewest for which sum_b ceil(m_b / vpc) <= N / vpc + nb CTAs fit
        // one per SM; eight warps of up to two vectors (<= 3 per sub-partition for vpc <= 10) when
        // shared memory holds them, else four warps of NV <= 2; the reflector chunk KC as large as
        // shared memory allows (<= 16)
        const size_t cap = kInvSmemCap;
        const int64_t slots = std::max<int64_t>(1, (int64_t)sm_count() - nb);
        const int want = (int)std::max<int64_t>(1, (h->N + slots - 1) / slots);
        int nw = 8, nv = 2;
        if (want > 10 || backtransform_smem(Mmax, 2, 8, 1) > cap) {
            nw = 4;
            nv = backtransform_smem(Mmax, 2, 4, 1) <= cap ? 2 : 1;
        }
        int kc = 16;
        while (kc > 1 && backtransform_smem(Mmax, nv, nw, kc) > cap) kc >>= 1;
        const int vpc = std::min(want, nw == 8 ? 10 : nw * nv);
        dim3 grid((unsigned)((h->N + vpc - 1) / vpc + nb));
        const size_t smem = backtransform_smem(Mmax, nv, nw, kc);
        if (nw == 8)
            k_backtransform<2, 8><<<grid, 256, smem, st>>>(w.plan, nb, h->N, Mmax, mmax, w.refl, w.tau, w.sel_val,
                                                        w.sel_vec, w.gersh, h->prm.alpha_theta, vpc, kc, w.X, w.eps,
                                                        w.alpha);
        else if (nv == 2)
            k_backtransform<2, 4><<<grid, 128, smem, st>>>(w.plan, nb, h->N, Mmax, mmax, w.refl, w.tau, w.sel_val,
                                                        w.sel_vec, w.gersh, h->prm.alpha_theta, vpc, kc, w.X, w.eps,
                                                        w.alpha);
        else
            k_backtransform<1, 4><<<grid, 128, smem, st>>>(w.plan, nb, h->N, Mmax, mmax, w.refl, w.tau, w.sel_val,
                                                        w.sel_vec, w.gersh, h->prm.alpha_theta, vpc, kc, w.X, w.eps,
                                                        w.alpha);
        g_launches++;
        return cudaGetLastError();
    }
}

}  // namespace pfsm
