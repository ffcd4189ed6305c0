// Back-transformation of the selected window eigenvectors in the mixed forms (Section II: the
// eigenvectors y of each submatrix start Eq. 11), y = H_0 H_1 ... H_{M-3} z for the m selected
// eigenvectors z of the window's tridiagonal T, followed by the start-vector rules (sign, zero
// padding to length N, shift eps and step alpha).
//
// With H_k = I - beta_k v_k v_k^T, the product of the reflectors has the compact-WY form
//   H_0 ... H_{M-3} = I - V S^-1 V^T,   S = diag(1 / beta_k) + striu(V^T V)
// (V = [v_0 ... v_{M-3}], striu the strictly upper triangle; Schreiber and Van Loan 1989, in the
// form of Joffrain, Low, Quintana-Orti, van de Geijn and Van Zee 2006: for two reflectors
// S^-1 = [[b0, -b0 b1 v0.v1], [0, b1]] reproduces I - b0 v0 v0^T - b1 v1 v1^T + b0 b1 (v0.v1) v0 v1^T).
// A reflector with beta = 0 (column already reduced) has v = 0 and contributes nothing. The
// reflectors' lengths differ (|v_k|^2 = 2 / beta_k), and the digit products are accurate relative
// to the largest entry of each operand row, so every v_k is first scaled by a power of two
// 2^p_k ~ 1 / |v_k| and beta_k by 2^-2p_k: the same H_k exactly, with |2^p_k v_k| in [1/2, 2]. So
//   Y = Z - V W2,  S W2 = W1,  W1 = V^T Z
// and three of the four stages are dense products, done by the FP64-accurate digit product on the
// tensor cores, batched over the windows: G = V^T V (lower triangle), W1 = V^T Z and
// Y = Z - W2^T V^T (rows = vectors). Only the triangular solve with S stays on the FP64 pipe:
// M^2 m / 2 FMAs per window against the 2 M^2 m of applying the reflectors one by one.
//   k_bt_prep    zero the unused entries of the reflector rows (j <= k, j >= M, k >= M - 2) and
//                of the eigenvector rows, write V^T, and the per-window extents
//   k_bt_trsm    W2 = S^-1 W1 by columns of the right-hand side: one CTA per (window, chunk of
//                columns) holds its columns of the residual in shared memory and runs the
//                right-looking back substitution (rows of G staged by cp.async)
//   k_bt_finish  the start-vector rules of the FP64 back-transformation, one warp per vector
#include <algorithm>

#include "pfsm_internal.cuh"

namespace pfsm {

namespace {

constexpr int kTrsmThreads = 256;                // update threads of k_bt_trsm (plus one warp for w)
constexpr int kTrsmMaxCols = 32;                 // columns per CTA (one lane of the w warp each)
constexpr size_t kTrsmSmemCap = 160 * 1024;      // shared memory of one k_bt_trsm CTA
constexpr size_t kTrsmGBytes = 80 * 1024;        // of it, the double-buffered rows of G

__device__ __forceinline__ void cp_async8(double *dst, const double *src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src)
                 : "memory");
}

// rows of G per staged chunk: the largest power of two <= 8 whose double buffer fits kTrsmGBytes
int trsm_chunk_rows(int Mmax)
{
    int kc = 8;
    while (kc > 1 && (size_t)2 * kc * Mmax * sizeof(double) > kTrsmGBytes) kc >>= 1;
    return kc;
}

size_t trsm_smem(int Mmax, int cw, int kc)
{
    return ((size_t)Mmax * cw + (size_t)2 * kc * Mmax + (size_t)Mmax) * sizeof(double);
}

// p_k of the exact power-of-two rescaling of reflector k: 2^(2 p_k) within a factor 4 of
// beta_k / 2 = 1 / |v_k|^2 (0 for beta = 0, whose v is zero)
__device__ __forceinline__ int wy_scale_exp(double beta)
{
    return beta > 0.0 ? ilogb(0.5 * beta) / 2 : 0;
}

// x 2^p: the exponent field moved by integer addition (no FP64 instruction; B300 retires one FP64
// warp instruction per 16 cycles per SM) when x is normal and stays normal, else ldexp; 0 stays 0
__device__ __forceinline__ double scale_pow2(double x, int p)
{
    const long long u = __double_as_longlong(x);
    const int ex = (int)((u >> 52) & 0x7FF);
    if (ex > 0 && ex + p > 0 && ex + p < 2047) return __longlong_as_double(u + ((long long)p << 52));
    return ldexp(x, p);
}

}  // namespace

bool backtransform_wy_fits(int Mmax)
{
    return Mmax >= 1 && trsm_smem(Mmax, 1, trsm_chunk_rows(Mmax)) <= kTrsmSmemCap;
}

// Grid (ceil(Mmax / 32), ceil(rows / 32), nb), 256 threads. Reflector part (vectors = false, rows
// = Mmax): tile (ti, tj) of window b's reflector rows (row k = v_k, entries j; valid for k < M - 2,
// k < j < M) is scaled by 2^p_k and cleaned in place and written transposed into RT;
// ext = {M - 2, m_b, M} per window. Vector part (vectors = true, rows = mmax): the eigenvector rows
// t are cleaned (entries j >= M and rows t >= m_b set to zero).
__global__ void __launch_bounds__(256)
k_bt_prep(const int32_t *__restrict__ plan, int nb, int Mmax, int mmax, bool vectors,
          const double *__restrict__ tau, double *__restrict__ refl, double *__restrict__ RT,
          double *__restrict__ sel_vec, int32_t *__restrict__ ext)
{
    __shared__ double t[32][33];
    const int b = blockIdx.z;
    const int mb = plan[nb + b], M = plan[3 * nb + b];
    const int nk = M > 2 ? M - 2 : 0;
    const int ti = blockIdx.y, tj = blockIdx.x;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    if (vectors) {
        double *bs = sel_vec + (size_t)b * mmax * Mmax;
        for (int q = ty; q < 32; q += 8) {
            const int tt = ti * 32 + q, j = tj * 32 + tx;
            if (tt < mmax && j < Mmax && (tt >= mb || j >= M)) bs[(size_t)tt * Mmax + j] = 0.0;
        }
        return;
    }
    __shared__ int pk[32];
    double *br = refl + (size_t)b * Mmax * Mmax;
    if (threadIdx.x < 32) {
        const int k = ti * 32 + threadIdx.x;
        pk[threadIdx.x] = (k < nk) ? wy_scale_exp(tau[(size_t)b * Mmax + k]) : 0;
    }
    __syncthreads();
    for (int q = ty; q < 32; q += 8) {
        const int k = ti * 32 + q, j = tj * 32 + tx;
        double v = 0.0;
        if (k < Mmax && j < Mmax) {
            if (k < nk && j > k && j < M) v = scale_pow2(br[(size_t)k * Mmax + j], pk[q]);
            br[(size_t)k * Mmax + j] = v;
        }
        t[q][tx] = v;
    }
    __syncthreads();
    double *bt = RT + (size_t)b * Mmax * Mmax;
    for (int q = ty; q < 32; q += 8) {
        const int j = tj * 32 + q, k = ti * 32 + tx;            // RT[j][k] = refl[k][j]
        if (j < Mmax && k < Mmax) bt[(size_t)j * Mmax + k] = t[tx][q];
    }
    if (ti == 0 && tj == 0 && threadIdx.x == 0) {
        ext[b] = nk;
        ext[nb + b] = mb;
        ext[2 * nb + b] = M;
    }
}

// Grid (ceil(m / cw), nb), 288 threads: W2 = S^-1 W1 for the columns t in [c0, c0 + cw) of window
// b, S = diag(1 / beta) + striu(G) with G = V^T V (its lower triangle read: G[k][l], l < k, is row k).
// Right-looking back substitution: for k = nk - 1 .. 0, w_k = beta_k R_k, then R_l -= G[k][l] w_k
// for l < k. Update thread (rg, c) owns column c's rows l = rg (mod nrg) of R (shared memory) and
// applies each step to its rows below k - 1; a dedicated warp (lane = column) applies step k to
// row k - 1 and publishes w_{k-1}, so the w chain overlaps the updates and a step costs one
// barrier. Rows of G pass through shared memory in double-buffered chunks of kc rows (cp.async).
// The reflectors are the scaled ones of k_bt_prep: beta_k 2^-2p_k on the diagonal of S^-1.
// Writes W2^T (row t, entries k; zero for k >= nk and for t >= m_b).
__global__ void __launch_bounds__(kTrsmThreads + 32)
k_bt_trsm(const int32_t *__restrict__ ext, int nb, int Mmax, int mmax, int cw, int kc,
          const double *__restrict__ G, const double *__restrict__ tau, const double *__restrict__ W1,
          double *__restrict__ W2T)
{
    extern __shared__ double sm_trsm[];
    double *R = sm_trsm;                                  // [Mmax][cw]
    double *Gs = R + (size_t)Mmax * cw;                   // [2][kc][Mmax]
    double *bs = Gs + (size_t)2 * kc * Mmax;              // [Mmax] scaled beta
    __shared__ double W2s[2][kTrsmMaxCols];
    const int b = blockIdx.y;
    const int nk = ext[b], mb = ext[nb + b];
    const double *Gb = G + (size_t)b * Mmax * Mmax;
    const double *tb = tau + (size_t)b * Mmax;
    for (int k = threadIdx.x; k < nk; k += blockDim.x) {
        const double bk = tb[k];
        bs[k] = scale_pow2(bk, -2 * wy_scale_exp(bk));
    }
    // the grid is sized by the nominal slice width; a CTA takes chunks blockIdx.x, + gridDim.x, ...
    // of the window's mmax columns (chunks beyond m_b only get their rows zeroed)
    for (int ci = blockIdx.x; ci * cw < mmax; ci += gridDim.x) {
        const int c0 = ci * cw;
        const int nc = max(0, min(cw, mb - c0));
        double *W2Tb = W2T + ((size_t)b * mmax + c0) * Mmax;
        // zero the parts of this chunk's rows that the solve does not write
        for (int i = threadIdx.x; i < cw * Mmax; i += blockDim.x) {
            const int c = i / Mmax, k = i - c * Mmax;
            if (c0 + c < mmax && (c >= nc || k >= nk)) W2Tb[(size_t)c * Mmax + k] = 0.0;
        }
        if (nc == 0 || nk == 0) continue;                 // uniform over the CTA
        const double *W1b = W1 + (size_t)b * Mmax * mmax + c0;
        __syncthreads();                                  // the previous chunk is done with R, Gs, W2s
        for (int i = threadIdx.x; i < nk * nc; i += blockDim.x) {
            const int k = i / nc, c = i - k * nc;
            R[(size_t)k * cw + c] = W1b[(size_t)k * mmax + c];
        }
        // threads [0, kTrsmThreads) update rows; the last warp computes and publishes the next w
        const bool wwarp = (int)threadIdx.x >= kTrsmThreads;
        const int wl = (int)threadIdx.x - kTrsmThreads;   // its lane: column wl
        const int nrg = kTrsmThreads / nc;
        const int c = (int)threadIdx.x % nc, rg = (int)threadIdx.x / nc;
        const bool act = !wwarp && rg < nrg;
        const int nch = (nk + kc - 1) / kc;
        auto issue = [&](int ch) {                        // rows k = khi, khi - 1, ... of G, entries l < k
            double *dst = Gs + (size_t)(ch & 1) * kc * Mmax;
            const int khi = nk - 1 - ch * kc;
            for (int r = 0; r < kc; r++) {
                const int k = khi - r;
                if (k < 0) break;
                for (int l = threadIdx.x; l < k; l += blockDim.x)
                    cp_async8(dst + (size_t)r * Mmax + l, Gb + (size_t)k * Mmax + l);
            }
            asm volatile("cp.async.commit_group;" ::: "memory");
        };
        issue(0);
        __syncthreads();                                  // R and the scaled betas loaded
        if (wwarp && wl < nc) {                           // w of the last row
            const double wv = bs[nk - 1] * R[(size_t)(nk - 1) * cw + wl];
            W2s[(nk - 1) & 1][wl] = wv;
            W2Tb[(size_t)wl * Mmax + nk - 1] = wv;
        }
        for (int ch = 0; ch < nch; ch++) {
            if (ch + 1 < nch) {
                issue(ch + 1);
                asm volatile("cp.async.wait_group 1;" ::: "memory");
            } else {
                asm volatile("cp.async.wait_group 0;" ::: "memory");
            }
            __syncthreads();                              // chunk ch of G and the last w visible
            const double *gch = Gs + (size_t)(ch & 1) * kc * Mmax;
            const int khi = nk - 1 - ch * kc;
            for (int r = 0; r < kc; r++) {
                const int k = khi - r;
                if (k < 0) break;
                const double *grow = gch + (size_t)r * Mmax;
                if (wwarp) {
                    // row k - 1 receives its last update in this step: the w warp applies it and
                    // publishes w_{k-1} while the update threads work on rows l < k - 1
                    if (k >= 1 && wl < nc) {
                        const double wv = bs[k - 1] * fma(-grow[k - 1], W2s[k & 1][wl], R[(size_t)(k - 1) * cw + wl]);
                        W2s[(k - 1) & 1][wl] = wv;
                        W2Tb[(size_t)wl * Mmax + k - 1] = wv;
                    }
                } else if (act) {
                    const double wk = W2s[k & 1][c];
#pragma unroll 4
                    for (int l = rg; l < k - 1; l += nrg) R[(size_t)l * cw + c] = fma(-grow[l], wk, R[(size_t)l * cw + c]);
                }
                __syncthreads();
            }
        }
    }
}

// One warp per selected vector (window b = warp / mmax, vector t): y = row t of Y, then the
// start-vector rules of the FP64 back-transformation: the home component positive when
// |y_home| >= 0.1, else the largest component (lowest index on ties); y zero-padded into row
// k0 + t of X at columns s .. s + M - 1; eps = the window eigenvalue, alpha = min(theta / d^2,
// 1 - 2^-20) with d the larger distance to the Gershgorin ends.
__global__ void __launch_bounds__(256)
k_bt_finish(const int32_t *__restrict__ plan, int nb, int64_t N, int Mmax, int mmax, const double *__restrict__ Y,
            const double *__restrict__ sel_val, const double *__restrict__ gersh, double alpha_theta,
            double *__restrict__ X, double *__restrict__ eps, double *__restrict__ alpha)
{
    const int gw = (int)(blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5));
    const int lane = threadIdx.x & 31;
    const int b = gw / mmax, t = gw - b * mmax;
    if (b >= nb) return;
    const int k0 = plan[b], mb = plan[nb + b], s = plan[2 * nb + b], M = plan[3 * nb + b];
    if (t >= mb) return;
    const double *zz = Y + ((size_t)b * mmax + t) * Mmax;
    const int home = k0 - s + t;
    // |y_i| compared as bit patterns (the IEEE order of magnitudes); a NaN is never the largest
    auto mag = [](double x) -> long long {
        const long long a = __double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFll;
        return a > 0x7FF0000000000000ll ? -1ll : a;
    };
    long long best = -1;
    int arg = M;
    for (int i = lane; i < M; i += 32) {
        const long long av = mag(zz[i]);
        if (av > best) { best = av; arg = i; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const long long ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oa = __shfl_xor_sync(0xffffffffu, arg, o);
        if (ob > best || (ob == best && oa < arg)) { best = ob; arg = oa; }
    }
    if (arg >= M) arg = home;                             // every entry NaN
    const double yh = zz[home];
    const long long tenth = __double_as_longlong(0.1);
    const double ref = (mag(yh) >= tenth) ? yh : zz[arg];
    const unsigned long long flip = (__double_as_longlong(ref) < 0) ? 0x8000000000000000ull : 0ull;   // sign bit
    const int64_t kg = k0 + t;
    double *xr = X + kg * N;
    for (int64_t jj = lane; jj < N; jj += 32) {
        const int64_t li = jj - s;
        xr[jj] = (li >= 0 && li < M) ? __longlong_as_double((long long)((unsigned long long)__double_as_longlong(zz[li]) ^ flip))
                                     : 0.0;
    }
    if (lane == 0) {
        const double glo = gersh[2 * N], ghi = gersh[2 * N + 1];
        const double lam = sel_val[(size_t)b * mmax + t];
        const double dmax = fmax(ghi - lam, lam - glo);
        const double av = alpha_theta / (dmax * dmax);
        const double cap = 1.0 - 0x1.0p-20;
        eps[kg] = lam;
        alpha[kg] = (av < cap) ? av : cap;
    }
}

// Steps that need only the window reduction's reflectors: clean and scale them, V^T, the extents,
// the digits of V^T's rows and G = V^T V (lower triangle), per window.
cudaError_t launch_backtransform_wy_reflectors(pfsm_handle_s *h, cudaStream_t st)
{
    Workspace &w = h->ws;
    const int nb = h->nb, Mmax = h->Mmax, mmax = h->mmax;
    const int64_t ldk = padded_ld(Mmax);
    const int64_t nbM = (int64_t)nb * Mmax;
    SliceBuf dA{w.btDA, nbM, ldk, OZ_SLICES, 0};
    cudaError_t e;
    const unsigned nt = (unsigned)((Mmax + 31) / 32);
    k_bt_prep<<<dim3(nt, nt, (unsigned)nb), 256, 0, st>>>(w.plan, nb, Mmax, mmax, false, w.tau, w.refl, w.btRT,
                                                           w.sel_vec, w.btExt);
    g_launches++;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = launch_oz_split(w.refl, nbM, Mmax, Mmax, dA, w.btEA, st)) != cudaSuccess) return e;
    OzParams o{};
    o.rows = Mmax; o.cols = Mmax; o.C = w.btG; o.ldc = Mmax; o.lower_only = 1; o.status = w.status;
    o.zrow = Mmax; o.zc = (int64_t)Mmax * Mmax; o.ext = w.btExt;
    return launch_gemm_oz(dA, w.btEA, dA, w.btEA, o, st, nb);
}

// The rest, after the tridiagonal eigenvectors: reflector steps on this stream unless the side
// stream ran them (joined before W1).
cudaError_t launch_backtransform_wy(pfsm_handle_s *h, cudaStream_t st, bool reflectors_done)
{
    Workspace &w = h->ws;
    const int nb = h->nb, Mmax = h->Mmax, mmax = h->mmax;
    const int64_t ldk = padded_ld(Mmax);
    const int64_t nbM = (int64_t)nb * Mmax, nbm = (int64_t)nb * mmax;
    SliceBuf dA{w.btDA, nbM, ldk, OZ_SLICES, 0}, dB{w.btDB, nbm, ldk, OZ_SLICES, 0};
    int32_t *ext_k = w.btExt, *ext_m = w.btExt + nb, *ext_M = w.btExt + 2 * nb;
    cudaError_t e;
    if (!reflectors_done && (e = launch_backtransform_wy_reflectors(h, st)) != cudaSuccess) return e;
    // 1. clean the eigenvector rows; their digits (z_t, entries j)
    const unsigned nt = (unsigned)((Mmax + 31) / 32);
    k_bt_prep<<<dim3(nt, (unsigned)((mmax + 31) / 32), (unsigned)nb), 256, 0, st>>>(w.plan, nb, Mmax, mmax, true, w.tau,
                                                                                      w.refl, w.btRT, w.sel_vec, w.btExt);
    g_launches++;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = launch_oz_split(w.sel_vec, nbm, Mmax, Mmax, dB, w.btEB, st)) != cudaSuccess) return e;
    if ((e = join_side(h, st)) != cudaSuccess) return e;
    // 2. W1 = V^T Z (rows k, columns t), per window
    OzParams o{};
    o.rows = Mmax; o.cols = mmax; o.C = w.btW1; o.ldc = mmax; o.status = w.status;
    o.zrow = Mmax; o.zrow_q = mmax; o.zc = (int64_t)Mmax * mmax; o.ext = ext_k; o.ext_c = ext_m;
    if ((e = launch_gemm_oz(dA, w.btEA, dB, w.btEB, o, st, nb)) != cudaSuccess) return e;
    // 3. W2 = S^-1 W1 -> W2^T: columns per CTA so that the CTAs fill the SMs once, within shared memory
    {
        // sized by the nominal slice width ceil(N / nb): mmax is the widest a slice can become after
        // cluster snapping, usually far from what the plan gives
        const int mnom = (int)std::min<int64_t>(mmax, (h->N + nb - 1) / nb);
        const int kc = trsm_chunk_rows(Mmax);
        int cw = 1;
        while (cw < kTrsmMaxCols && (int64_t)nb * ((mnom + cw - 1) / cw) > (int64_t)sm_count()) cw++;
        while (cw > 1 && trsm_smem(Mmax, cw, kc) > kTrsmSmemCap) cw--;
        const dim3 grid((unsigned)((mnom + cw - 1) / cw), (unsigned)nb);
        k_bt_trsm<<<grid, kTrsmThreads + 32, trsm_smem(Mmax, cw, kc), st>>>(w.btExt, nb, Mmax, mmax, cw, kc, w.btG,
                                                                           w.tau, w.btW1, w.btW2T);
        g_launches++;
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    // 4. digits of W2^T (rows t, entries k) and of V (rows j, entries k)
    if ((e = launch_oz_split(w.btW2T, nbm, Mmax, Mmax, dB, w.btEB, st)) != cudaSuccess) return e;
    if ((e = launch_oz_split(w.btRT, nbM, Mmax, Mmax, dA, w.btEA, st)) != cudaSuccess) return e;
    // 5. Y = Z - W2^T V^T (rows t, entries j), per window
    if ((e = cudaMemcpyAsync(w.btY, w.sel_vec, (size_t)nbm * Mmax * sizeof(double), cudaMemcpyDeviceToDevice, st)) !=
        cudaSuccess)
        return e;
    o = OzParams{};
    o.rows = mmax; o.cols = Mmax; o.C = w.btY; o.ldc = Mmax; o.sub = 1; o.status = w.status;
    o.zrow = mmax; o.zrow_q = Mmax; o.zc = (int64_t)mmax * Mmax; o.ext = ext_m; o.ext_c = ext_M;
    if ((e = launch_gemm_oz(dB, w.btEB, dA, w.btEA, o, st, nb)) != cudaSuccess) return e;
    // 6. start vectors
    {
        const int64_t warps = nbm;
        k_bt_finish<<<(unsigned)((warps + 7) / 8), 256, 0, st>>>(w.plan, nb, h->N, Mmax, mmax, w.btY, w.sel_val,
                                                                 w.gersh, h->prm.alpha_theta, w.X, w.eps, w.alpha);
        g_launches++;
    }
    return cudaGetLastError();
}

cudaError_t launch_bt_finish(pfsm_handle_s *h, const double *Y, cudaStream_t st)
{
    Workspace &w = h->ws;
    const int64_t warps = (int64_t)h->nb * h->mmax;
    k_bt_finish<<<(unsigned)((warps + 7) / 8), 256, 0, st>>>(w.plan, h->nb, h->N, h->Mmax, h->mmax, Y, w.sel_val,
                                                             w.gersh, h->prm.alpha_theta, w.X, w.eps, w.alpha);
    g_launches++;
    return cudaGetLastError();
}

cudaError_t join_side(pfsm_handle_s *h, cudaStream_t st)
{
    if (!h->side_pending) return cudaSuccess;
    h->side_pending = false;
    return cudaStreamWaitEvent(st, h->join_ev, 0);
}

cudaError_t configure_bt_wy_kernels()
{
    return cudaFuncSetAttribute(k_bt_trsm, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTrsmSmemCap);
}

}  // namespace pfsm
