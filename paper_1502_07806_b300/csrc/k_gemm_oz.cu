// FP64-accurate products on the BF16 tensor cores (tcgen05 + TMEM, TMA-fed): the error-free
// splitting of Ozaki, Ogita, Oishi and Rump (2012), arranged for B300, where the DFMA pipe gives
// 1.2 TFLOP/s and the BF16 tensor cores about 1.8 PFLOP/s.
//
// Splitting (k_oz_split): every row r of an operand is scaled by its own power of two 2^-e_r so
// that |x| < 1, rounded to a 45-bit fixed-point integer q, and q is cut into S = 9 balanced base-32
// digits n_0 .. n_8 (n_s in [-16, 16) for s >= 1, |n_0| <= 32), each stored exactly as a BF16 value:
//   x = 2^e_r sum_s n_s 2^-5(s+1)   (to 2^-46 of the row's largest entry).
// Product (k_gemm_oz): C[r, c] = sum_L 2^(e_r + e_c - 5(L+2)) sum_{s+t=L} sum_k n_s[r,k] m_t[c,k].
// Every digit product has |n m| <= 2^10 and a level has at most S = 9 pairs, so a level summed over
// a K chunk of 1792 terms stays below 2^24 and the FP32 accumulation in tensor memory is EXACT.
// Levels L = 0 .. OZ_LEVELS-1 = 10 are kept. Every entry, however small, has O(1) low digits, so
// the products of a dropped level L add up like a random walk over K: about
// sqrt(K (pairs at L)) 2^(8 - 5(L+2)) / 3 relative to 2^(e_r + e_c). Stopping after L = 8 would
// leave sqrt(K) 2^-46 (1e-12 at K = 9072); stopping after L = 10 leaves about 1e-15 there, below
// the 2^-46 rounding of the operands themselves. Products that only need FP32-class accuracy
// ask for fewer levels (about sqrt(K) 2^(3 - 5(levels+1)) / 3). Each (level, K chunk) group is
// drained from TMEM into FP64 registers with its exact power-of-two scale while the tensor cores
// fill the other of two TMEM buffers.
//
// CTA: 192 threads, a 128 x 64 output tile. Warp 0: TMA loads of digit tiles (6-stage ring).
// Warp 1: TMEM owner and MMA issuer (M = 128, N = 64, K = 16). Warps 2-5: drain TMEM (one row each
// thread, 64 FP64 accumulators), then apply the epilogue, which can add an exact FP64 diagonal
// term C[r, c] += V[r, c] d[c] (for products with A = diag(d) + E whose digits cover E only, so
// that the error scales with the small off-diagonal part). All mbarrier waits are bounded.
#include "tc_common.cuh"

namespace pfsm {

namespace oz {

constexpr int BM = 128, BN = 64, STAGES = 6;
constexpr int A_BYTES = BM * 128, B_BYTES = BN * 128, STAGE_BYTES = A_BYTES + B_BYTES;
constexpr uint32_t TMEM_COLS = 128;          // two 64-column FP32 accumulators
constexpr int KCHUNK = 1792;                 // K terms per exact group: 1792 * 9 <= 16384
constexpr int BETA = 5;

}  // namespace oz

// ---- splitting -------------------------------------------------------------------------------

// One warp per row: exponent of the row's largest |entry| and the S digits of every entry.
// zero_diag: digits of the off-diagonal part (entry (r, r) taken as 0, its value stored in d[r]).
// Input in FP64 or FP32 (an FP32 operand's digits are exact: 24 bits fit in the 45-bit grid of its
// row unless the entry is below 2^-21 of the row's largest).
template <typename T>
__global__ void k_oz_split(const T *__restrict__ src, int64_t rows, int64_t cols, int64_t ld,
                           __nv_bfloat16 *__restrict__ dst, int64_t sl_ld, int64_t sstride,
                           int32_t *__restrict__ exps, int zero_diag, double *__restrict__ d)
{
    const int lane = threadIdx.x & 31;
    const int64_t r = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (r >= rows) return;
    const T *x = src + r * ld;
    auto val = [&](int64_t c) { return (zero_diag && c == r) ? 0.0 : (double)x[c]; };
    if (zero_diag && lane == 0 && d) d[r] = (double)x[r];
    double mx = 0.0;
    for (int64_t c = lane; c < cols; c += 32) mx = fmax(mx, fabs(val(c)));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    int e = 0;
    if (mx > 0.0) frexp(mx, &e);             // mx = f 2^e, f in [0.5, 1): |x| 2^-e < 1
    if (lane == 0) exps[r] = e;
    const double sc = ldexp(1.0, 5 * OZ_SLICES - e);
    __nv_bfloat16 *out = dst + r * sl_ld;
    for (int64_t c = lane; c < cols; c += 32) {
        long long q = __double2ll_rn(val(c) * sc);    // |q| <= 2^45
        int dig[OZ_SLICES];
#pragma unroll
        for (int s = OZ_SLICES - 1; s >= 1; s--) {    // balanced base-32 digits, low to high
            const int d = (int)(((q + 16) & 31) - 16);
            dig[s] = d;
            q = (q - d) >> 5;
        }
        dig[0] = (int)q;
#pragma unroll
        for (int s = 0; s < OZ_SLICES; s++) out[s * sstride + c] = __int2bfloat16_rn(dig[s]);
    }
}

// ---- product ---------------------------------------------------------------------------------

__global__ void __launch_bounds__(192, 1)
k_gemm_oz(const __grid_constant__ CUtensorMap mapP, const __grid_constant__ CUtensorMap mapQ, OzParams prm)
{
    using namespace tc;
    using namespace oz;
    const int z = blockIdx.z;
    const int row0 = prm.row_base + blockIdx.y * BM, col0 = prm.row_base + blockIdx.x * BN;
    const int rows_lim = prm.ext ? prm.ext[z] : prm.rows, cols_lim = prm.ext ? prm.ext[z] : prm.cols;
    if (row0 >= rows_lim || col0 >= cols_lim) return;              // tile outside this window
    if (prm.lower_only && col0 > row0 + BM - 1) return;           // whole tile above the diagonal
    const int64_t zr = (int64_t)z * prm.zrow;                      // operand row offset
    double *Cz = prm.C + (int64_t)z * prm.zc;
    extern __shared__ __align__(1024) uint8_t smraw[];
    const uint32_t raw = smem_u32(smraw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    uint8_t *gbase = smraw + (base - raw);
    uint64_t *bars = reinterpret_cast<uint64_t *>(gbase + STAGES * STAGE_BYTES);
    // bars: [0,S) full, [S,2S) empty, [2S,2S+2) accumulator full, [2S+2,2S+4) accumulator empty
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 2 * STAGES + 4);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
    int *ecol = reinterpret_cast<int *>(tmem_slot + 2);           // BN column exponents
    double *estage = reinterpret_cast<double *>(gbase + STAGES * STAGE_BYTES + 1024);   // 128 x (BN + 1)
    const uint32_t bar_base = smem_u32(bars);
    auto full_bar = [&](int s) { return bar_base + 8u * s; };
    auto empty_bar = [&](int s) { return bar_base + 8u * (STAGES + s); };
    auto accf_bar = [&](int b) { return bar_base + 8u * (2 * STAGES + b); };
    auto acce_bar = [&](int b) { return bar_base + 8u * (2 * STAGES + 2 + b); };
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    // 64-element K blocks; a lower-triangular P has no entries beyond column row0 + BM - 1
    const int nkb_total = prm.p_lower ? min(prm.kblocks, (row0 + BM + 63) / 64) : prm.kblocks;
    const int kb_per_chunk = KCHUNK / 64;
    const int nch = (nkb_total + kb_per_chunk - 1) / kb_per_chunk;
    const int S = OZ_SLICES;
    const int LV = (prm.levels > 0 && prm.levels < 2 * S - 1) ? prm.levels : OZ_LEVELS;   // levels 0 .. LV-1
    const int groups = LV * nch;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; s++) {
            mbar_init(full_bar(s), 1);
            mbar_init(empty_bar(s), 1);
        }
        for (int b = 0; b < 2; b++) {
            mbar_init(accf_bar(b), 1);
            mbar_init(acce_bar(b), 128);
        }
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&mapP) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&mapQ) : "memory");
    }
    for (int j = threadIdx.x; j < BN; j += blockDim.x)
        ecol[j] = (col0 + j < cols_lim) ? prm.eq[zr + col0 + j] : 0;
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(smem_u32(tmem_slot)), "r"(TMEM_COLS) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem_acc = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            int it = 0, issued = 0;
            bool stop = false;
            for (int g = 0; g < groups && !stop; g++) {
                const int L = g / nch, ch = g % nch;
                const int kbA = ch * kb_per_chunk, kbB = min(nkb_total, kbA + kb_per_chunk);
                for (int sa = (L >= S ? L - S + 1 : 0); sa <= L && sa < S && !stop; sa++) {
                    const int sb = L - sa;
                    for (int kb = kbA; kb < kbB; kb++, it++) {
                        const int s = it % STAGES, round = it / STAGES;
                        if (round > 0 && !mbar_wait(empty_bar(s), (round - 1) & 1)) {
                            set_status(prm.status, PFSM_ERR_TIMEOUT);
                            *abort_flag = 1;
                            stop = true;
                            break;
                        }
                        if (*abort_flag) { stop = true; break; }
                        const uint32_t a = base + s * STAGE_BYTES, b = a + A_BYTES;
                        mbar_expect_tx(full_bar(s), STAGE_BYTES);
                        tma_load_3d(a, &mapP, full_bar(s), kb * 64, (int)(zr + row0), sa);
                        tma_load_3d(b, &mapQ, full_bar(s), kb * 64, (int)(zr + col0), sb);
                        issued = it + 1;
                    }
                }
            }
            for (int i = (issued > STAGES ? issued - STAGES : 0); i < issued; i++)
                mbar_wait(full_bar(i % STAGES), (i / STAGES) & 1);
        }
        __syncwarp();
    } else if (warp == 1) {
        if (lane == 0) {
            int it = 0;
            bool ok = true;
            for (int g = 0; g < groups && ok; g++) {
                const int L = g / nch, ch = g % nch, buf = g & 1;
                if (g >= 2 && !mbar_wait(acce_bar(buf), ((g >> 1) - 1) & 1)) { ok = false; break; }
                fence_after();
                const uint32_t dacc = tmem_acc + 64u * buf;
                const int kbA = ch * kb_per_chunk, kbB = min(nkb_total, kbA + kb_per_chunk);
                bool first = true;
                for (int sa = (L >= S ? L - S + 1 : 0); sa <= L && sa < S && ok; sa++) {
                    for (int kb = kbA; kb < kbB; kb++, it++) {
                        const int s = it % STAGES;
                        if (!mbar_wait(full_bar(s), (it / STAGES) & 1) || *abort_flag) { ok = false; break; }
                        fence_after();
                        const uint32_t a = base + s * STAGE_BYTES, b = a + A_BYTES;
                        const uint64_t da = sw128_desc(a), db = sw128_desc(b);
#pragma unroll
                        for (int kk = 0; kk < 4; kk++) {
                            umma<0, BM, BN>(dacc, da + 2 * kk, db + 2 * kk, first ? 0u : 1u);
                            first = false;
                        }
                        umma_commit(empty_bar(s));
                    }
                }
                umma_commit(accf_bar(buf));   // this group's sum is complete when its MMAs are
            }
            if (!ok) {
                set_status(prm.status, PFSM_ERR_TIMEOUT);
                *abort_flag = 1;
                umma_commit(accf_bar(0));
                mbar_wait(accf_bar(0), 0);    // fences the MMAs issued so far (bounded)
            }
        }
        __syncwarp();
    } else {
        const int gq = warp & 3;
        const int r = row0 + 32 * gq + lane;
        // the levels are combined in float-float (hi + lo, about 48 bits) with Knuth's TwoSum: each
        // level sum is an exact FP32 integer and its scale an exact power of two, so a level costs
        // a few FP32 operations per entry instead of two FP64 ones (the FP64 pipe is 64 times
        // slower); one FP64 conversion per entry at the end
        float hi[BN], lo[BN];
#pragma unroll
        for (int j = 0; j < BN; j++) { hi[j] = 0.0f; lo[j] = 0.0f; }
        bool ok = true;
        for (int g = 0; g < groups; g++) {
            const int L = g / nch, buf = g & 1;
            bool got = mbar_wait(accf_bar(buf), (g >> 1) & 1);
            got = __all_sync(0xffffffffu, got) && !*abort_flag;
            if (!got) {
                ok = false;
                set_status(prm.status, PFSM_ERR_TIMEOUT);
                *abort_flag = 1;
                break;
            }
            fence_after();
            const float scale = __int_as_float((127 - oz::BETA * (L + 2)) << 23);   // 2^-5(L+2)
            uint32_t v[32];
#pragma unroll
            for (int half = 0; half < 2; half++) {
                tmem_ld32(tmem_acc + ((uint32_t)(32 * gq) << 16) + 64u * buf + 32 * half, v);
#pragma unroll
                for (int j = 0; j < 32; j++) {
                    const float x = __uint_as_float(v[j]) * scale;
                    const float h = hi[32 * half + j];
                    const float sum = h + x, bp = sum - h;
                    lo[32 * half + j] += (h - (sum - bp)) + (x - bp);
                    hi[32 * half + j] = sum;
                }
            }
            fence_before();
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(acce_bar(buf)) : "memory");
        }
        // epilogue through this warp's shared-memory staging block (32 rows x 64 columns), so
        // that the loads and stores of C (and of the exact diagonal term) are row-contiguous
        double(*eb)[BN + 1] = reinterpret_cast<double(*)[BN + 1]>(estage) + 32 * gq;
        const int R0 = row0 + 32 * gq;
        const int er = (ok && r < rows_lim) ? prm.ep[zr + r] : 0;
#pragma unroll
        for (int j = 0; j < BN; j++) eb[lane][j] = ldexp((double)hi[j] + (double)lo[j], er + ecol[j]);
        __syncwarp();
        if (ok) {
            for (int rr = 0; rr < 32; rr++) {
                const int gr = R0 + rr;
                if (gr >= rows_lim) break;
#pragma unroll
                for (int h = 0; h < BN / 32; h++) {
                    const int c = col0 + 32 * h + lane;
                    if (c < cols_lim && !(prm.lower_only && c > gr)) {
                        double res = eb[rr][32 * h + lane];
                        if (prm.dcol) res = fma(prm.Vp[(int64_t)gr * prm.ldv + c], prm.dcol[c], res);
                        const int64_t o = (int64_t)gr * prm.ldc + c;
                        if (prm.sub) Cz[o] -= res;
                        else Cz[o] = res;
                    }
                }
            }
        }
    }
    fence_before();
    __syncthreads();
    if (warp == 1) {
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_acc), "r"(oz::TMEM_COLS) : "memory");
    }
}

// ---- host side -------------------------------------------------------------------------------

namespace {
size_t oz_smem_bytes() { return (size_t)oz::STAGES * oz::STAGE_BYTES + 1024 + 1024 + (size_t)128 * (oz::BN + 1) * 8; }
}

cudaError_t configure_oz_kernels()
{
    return cudaFuncSetAttribute(k_gemm_oz, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)oz_smem_bytes());
}

cudaError_t launch_oz_split(const double *src, int64_t rows, int64_t cols, int64_t ld, const SliceBuf &dst,
                            int32_t *exps, cudaStream_t st, bool zero_diag, double *d)
{
    const unsigned blocks = (unsigned)((rows + 7) / 8);
    k_oz_split<double><<<blocks, 256, 0, st>>>(src, rows, cols, ld, reinterpret_cast<__nv_bfloat16 *>(dst.ptr),
                                               dst.ld, dst.ld * dst.rows, exps, zero_diag ? 1 : 0, d);
    g_launches++;
    return cudaGetLastError();
}

cudaError_t launch_oz_split_f32(const float *src, int64_t rows, int64_t cols, int64_t ld, const SliceBuf &dst,
                                int32_t *exps, cudaStream_t st)
{
    const unsigned blocks = (unsigned)((rows + 7) / 8);
    k_oz_split<float><<<blocks, 256, 0, st>>>(src, rows, cols, ld, reinterpret_cast<__nv_bfloat16 *>(dst.ptr),
                                              dst.ld, dst.ld * dst.rows, exps, 0, nullptr);
    g_launches++;
    return cudaGetLastError();
}

cudaError_t launch_gemm_oz(const SliceBuf &P, const int32_t *ep, const SliceBuf &Q, const int32_t *eq,
                           OzParams prm, cudaStream_t st, int batch)
{
    CUtensorMap mp, mq;
    cudaError_t e;
    if ((e = make_slice_map(&mp, P, oz::BM)) != cudaSuccess) return e;
    if ((e = make_slice_map(&mq, Q, oz::BN)) != cudaSuccess) return e;
    prm.kblocks = (int)(P.ld / 64);
    prm.ep = ep;
    prm.eq = eq;
    // batched: prm.rows / prm.cols give the grid extent from row_base (the largest window)
    const int ext_r = prm.rows - prm.row_base, ext_c = prm.cols - prm.row_base;
    if (ext_r <= 0 || ext_c <= 0) return cudaSuccess;
    dim3 grid((unsigned)((ext_c + oz::BN - 1) / oz::BN), (unsigned)((ext_r + oz::BM - 1) / oz::BM), (unsigned)batch);
    k_gemm_oz<<<grid, 192, oz_smem_bytes(), st>>>(mp, mq, prm);
    g_launches++;
    return cudaGetLastError();
}

}  // namespace pfsm
