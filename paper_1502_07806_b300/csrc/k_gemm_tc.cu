// Split-precision GEMM on the 5th-generation tensor cores (tcgen05 + TMEM, operands fed by TMA)
// for the products of Eq. 11 in the mixed forms.
//
//   C[r, c] = sum over slice pairs (a, b) of sum_k P_a[r, k] * Q_b[c, k]
//
// P and Q are FP64 matrices held as BF16 (3 slices) or TF32 (2 slices) pieces, x = sum_s x_s with
// each x_s the rounding of the remainder left by the earlier slices. Pairs of total order below
// the slice count are accumulated into ONE FP32 accumulator in tensor memory (6 products for
// BF16, 3 for TF32): the K loop runs over (pair, k-block). The epilogue converts to FP64 and
// applies the Eq. 11 algebra in FP64 (TC_EPI_* modes), and can write the BF16/TF32 slices of its
// own result, which are the operand of the next product. TC_EPI_STORE / TC_EPI_RSUB serve the
// FP32-accurate products of the mixed-form Gram-Schmidt.
//
// CTA: 192 threads, one 128x128 output tile. Warp 0 issues TMA loads (SWIZZLE_128B, 128-byte K
// rows) into a 6-stage ring; warp 1 owns the TMEM accumulator (128 columns) and issues
// tcgen05.mma (M=128, N=128, K=16 bf16 / 8 tf32) from one lane; warps 2-5 drain TMEM with
// tcgen05.ld (32 lanes each). Every mbarrier wait is bounded by %globaltimer: a wait that gives
// up records PFSM_ERR_TIMEOUT in the status word, the CTA skips the rest of its work, waits
// (bounded) for its copies in flight, frees its TMEM and exits.
#include "tc_common.cuh"

namespace pfsm {

namespace tc {

constexpr int BM = 128, BN = 128, STAGES = 6;
constexpr int TILE_BYTES = BM * 128;                 // 128 rows x 128 bytes
constexpr int STAGE_BYTES = 2 * TILE_BYTES;
constexpr uint32_t TMEM_COLS = 128;

}  // namespace tc

template <int KIND>
__global__ void __launch_bounds__(192, 1)
k_gemm_tc(const __grid_constant__ CUtensorMap mapP, const __grid_constant__ CUtensorMap mapQ, TcParams prm)
{
    using namespace tc;
    extern __shared__ __align__(1024) uint8_t smraw[];
    const uint32_t raw = smem_u32(smraw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    uint8_t *gbase = smraw + (base - raw);
    uint64_t *bars = reinterpret_cast<uint64_t *>(gbase + STAGES * STAGE_BYTES);
    // bars[0..S): full, [S..2S): empty, [2S]: accumulator ready
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 2 * STAGES + 1);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
    const uint32_t bar_base = smem_u32(bars);
    const uint32_t acc_bar = bar_base + 8u * (2 * STAGES);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int row0 = blockIdx.y * BM, col0 = blockIdx.x * BN;
    if (prm.lower_only && col0 > row0 + BM - 1) return;           // whole tile above the diagonal

    // K-block range (the first product only needs the columns its rows' windows cover)
    int kb0 = 0, kb1 = prm.kblocks;
    if (prm.krange) {
        const int t0 = 2 * blockIdx.y;
        const int t1 = min(t0 + 1, prm.nrowtiles64 - 1);
        const int kbeg = min(prm.krange[2 * t0], prm.krange[2 * t1]);
        const int kend = max(prm.krange[2 * t0 + 1], prm.krange[2 * t1 + 1]);
        kb0 = kbeg / prm.bk;
        kb1 = min(prm.kblocks, (kend + prm.bk - 1) / prm.bk);
        if (kb1 < kb0) kb1 = kb0;
    }
    const int nkb = kb1 - kb0;
    const int total = nkb * prm.npairs;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; s++) {
            mbar_init(bar_base + 8u * s, 1);
            mbar_init(bar_base + 8u * (STAGES + s), 1);
        }
        mbar_init(acc_bar, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&mapP) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&mapQ) : "memory");
    }
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
            int issued = 0;
            for (int it = 0; it < total; it++) {
                const int s = it % STAGES, round = it / STAGES;
                if (round > 0 && !mbar_wait(bar_base + 8u * (STAGES + s), (round - 1) & 1)) {
                    set_status(prm.status, PFSM_ERR_TIMEOUT);
                    *abort_flag = 1;
                    break;
                }
                if (*abort_flag) break;
                const int q = it / nkb, kb = kb0 + it % nkb;
                const uint32_t sa = base + s * STAGE_BYTES, sb = sa + TILE_BYTES;
                mbar_expect_tx(bar_base + 8u * s, STAGE_BYTES);
                tma_load_3d(sa, &mapP, bar_base + 8u * s, kb * prm.bk, row0, prm.pa[q]);
                tma_load_3d(sb, &mapQ, bar_base + 8u * s, kb * prm.bk, col0, prm.pb[q]);
                issued = it + 1;
            }
            // leave no copies in flight: wait (bounded) for the last stages filled
            for (int it = (issued > STAGES ? issued - STAGES : 0); it < issued; it++)
                mbar_wait(bar_base + 8u * (it % STAGES), (it / STAGES) & 1);
        }
        __syncwarp();
    } else if (warp == 1) {
        if (lane == 0) {
            bool ok = true;
            for (int it = 0; it < total; it++) {
                const int s = it % STAGES;
                if (!mbar_wait(bar_base + 8u * s, (it / STAGES) & 1) || *abort_flag) {
                    set_status(prm.status, PFSM_ERR_TIMEOUT);
                    *abort_flag = 1;
                    ok = false;
                    break;
                }
                fence_after();
                const uint32_t sa = base + s * STAGE_BYTES, sb = sa + TILE_BYTES;
                const uint64_t da = sw128_desc(sa), db = sw128_desc(sb);
#pragma unroll
                for (int kk = 0; kk < 4; kk++)   // 4 x 32 bytes of K per 128-byte row
                    umma<KIND>(tmem_acc, da + 2 * kk, db + 2 * kk, (it > 0 || kk > 0) ? 1u : 0u);
                umma_commit(bar_base + 8u * (STAGES + s));
            }
            // signals the epilogue; also tracks every issued MMA before TMEM is released
            umma_commit(acc_bar);
            if (!ok) mbar_wait(acc_bar, 0);
        }
        __syncwarp();
    } else {
        // epilogue: warp w reads TMEM lanes 32*(w % 4) .. +31, i.e. tile rows
        const int g = warp & 3;
        const int r = row0 + 32 * g + lane;
        const bool have_acc = total > 0;
        bool ok = true;
        if (have_acc) ok = mbar_wait(acc_bar, 0);
        ok = __all_sync(0xffffffffu, ok);
        if (!ok) {
            set_status(prm.status, PFSM_ERR_TIMEOUT);
            *abort_flag = 1;
        }
        fence_after();
        const bool row_ok = r < prm.rows;
        double er = 0.0, ar = 0.0;
        int win_lo = 0, win_hi = 0;
        if (row_ok) {
            if (prm.eps) er = prm.eps[r];
            if (prm.alpha) ar = prm.alpha[r];
            if (prm.epi == TC_EPI_Y0) {
                // window of the slice owning row r (largest b with k0[b] <= r)
                int lo = 0, hi = prm.nb - 1;
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (prm.plan[mid] <= r) lo = mid; else hi = mid - 1;
                }
                win_lo = prm.plan[2 * prm.nb + lo];
                win_hi = win_lo + prm.plan[3 * prm.nb + lo];
            }
        }
        for (int chunk = 0; chunk < BN / 32; chunk++) {
            uint32_t v[32];
            if (have_acc && ok) {
                tmem_ld32(tmem_acc + ((uint32_t)(32 * g) << 16) + 32 * chunk, v);
            } else {
#pragma unroll
                for (int j = 0; j < 32; j++) v[j] = 0u;
            }
            if (!row_ok || !ok) continue;
#pragma unroll
            for (int j = 0; j < 32; j++) {
                const int c = col0 + 32 * chunk + j;
                if (c < prm.cols) {
                    const double acc = (double)__uint_as_float(v[j]);
                    const int64_t o = (int64_t)r * prm.ldo + c;
                    double res;
                    if (prm.epi == TC_EPI_STORE) {
                        res = acc;
                    } else if (prm.epi == TC_EPI_Y0) {
                        res = (c >= win_lo && c < win_hi) ? 0.0 : acc;
                    } else if (prm.epi == TC_EPI_Z) {
                        res = acc + (prm.d[c] - er) * prm.V[o];
                        prm.X[o] -= ar * res;
                    } else if (prm.epi == TC_EPI_YN) {
                        res = prm.Yold[o] - ar * (acc + (prm.d[c] - er) * prm.V[o]);
                    } else {   // TC_EPI_RSUB
                        res = prm.V[o] - acc;
                    }
                    prm.out[o] = res;
                    if (prm.out_ns > 0)
                        store_slices<KIND>(prm.out_slices, prm.sl_stride, (int64_t)r * prm.sl_ld + c, prm.out_ns, res);
                }
            }
        }
    }
    fence_before();
    __syncthreads();
    if (warp == 1) {
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_acc), "r"(TMEM_COLS) : "memory");
    }
}

// ---- operand splitting ---------------------------------------------------------------------

// Slices of a rows x cols FP64 matrix (leading dimension ld) into slice matrices with leading
// dimension sl_ld; padding columns are left untouched (zero since allocation).
// zero_diag: split the off-diagonal part E = A - diag(A) and write diag(A) to d.
template <int KIND>
__global__ void k_split(const double *__restrict__ src, int64_t rows, int64_t cols, int64_t ld,
                        void *dst, int64_t sl_ld, int64_t sstride, int ns, int zero_diag,
                        double *__restrict__ d)
{
    const int64_t i = blockIdx.y;
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < cols; c += (int64_t)gridDim.x * blockDim.x) {
        double v = src[i * ld + c];
        if (zero_diag && c == i) {
            if (d) d[i] = v;
            v = 0.0;
        }
        tc::store_slices<KIND>(dst, sstride, i * sl_ld + c, ns, v);
    }
}

// ---- host side -------------------------------------------------------------------------------

namespace {

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                  const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                  const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn()
{
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)p;
    }
    return fn;
}

}  // namespace

// 3-D map over the slices: {ld (K), rows, ns}, box {128 bytes of K, box_rows rows, 1 slice}.
cudaError_t make_slice_map(CUtensorMap *map, const SliceBuf &b, int box_rows)
{
    EncodeTiledFn fn = encode_fn();
    if (!fn) return cudaErrorNotSupported;
    const int esz = b.kind == 0 ? 2 : 4;
    cuuint64_t dims[3] = {(cuuint64_t)b.ld, (cuuint64_t)b.rows, (cuuint64_t)b.ns};
    cuuint64_t strides[2] = {(cuuint64_t)b.ld * esz, (cuuint64_t)b.ld * b.rows * esz};
    cuuint32_t box[3] = {(cuuint32_t)(128 / esz), (cuuint32_t)box_rows, 1u};
    cuuint32_t estr[3] = {1u, 1u, 1u};
    CUresult r = fn(map, b.kind == 0 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3,
                    b.ptr, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

namespace {

size_t tc_smem_bytes() { return (size_t)tc::STAGES * tc::STAGE_BYTES + 1024 + 256; }

}  // namespace

cudaError_t configure_tc_kernels()
{
    cudaError_t e = cudaFuncSetAttribute(k_gemm_tc<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc_smem_bytes());
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_gemm_tc<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc_smem_bytes());
}

cudaError_t launch_split(const double *src, int64_t rows, int64_t cols, int64_t ld, const SliceBuf &dst,
                         bool zero_diag, double *d, cudaStream_t st)
{
    const int64_t bx = (cols + 255) / 256;
    dim3 grid((unsigned)(bx < 8 ? bx : 8), (unsigned)rows);
    if (dst.kind == 0)
        k_split<0><<<grid, 256, 0, st>>>(src, rows, cols, ld, dst.ptr, dst.ld, dst.ld * dst.rows, dst.ns, zero_diag, d);
    else
        k_split<1><<<grid, 256, 0, st>>>(src, rows, cols, ld, dst.ptr, dst.ld, dst.ld * dst.rows, dst.ns, zero_diag, d);
    g_launches++;
    return cudaGetLastError();
}

cudaError_t launch_gemm_tc(const SliceBuf &P, const SliceBuf &Q, TcParams prm, SliceBuf *out_sl, cudaStream_t st)
{
    CUtensorMap mp, mq;
    cudaError_t e;
    if ((e = make_slice_map(&mp, P, tc::BM)) != cudaSuccess) return e;
    if ((e = make_slice_map(&mq, Q, tc::BN)) != cudaSuccess) return e;
    prm.bk = P.kind == 0 ? 64 : 32;
    prm.kblocks = (int)(P.ld / prm.bk);
    int n = 0;   // slice pairs of total order below the slice count
    for (int ord = 0; ord < P.ns; ord++)
        for (int a = 0; a <= ord; a++) {
            prm.pa[n] = (int8_t)a;
            prm.pb[n] = (int8_t)(ord - a);
            n++;
        }
    prm.npairs = n;
    if (out_sl) {
        prm.out_slices = out_sl->ptr;
        prm.sl_ld = out_sl->ld;
        prm.sl_stride = out_sl->ld * out_sl->rows;
        prm.out_ns = out_sl->ns;
    } else {
        prm.out_ns = 0;
    }
    dim3 grid((unsigned)((prm.cols + tc::BN - 1) / tc::BN), (unsigned)((prm.rows + tc::BM - 1) / tc::BM));
    if (P.kind == 0)
        k_gemm_tc<0><<<grid, 192, tc_smem_bytes(), st>>>(mp, mq, prm);
    else
        k_gemm_tc<1><<<grid, 192, tc_smem_bytes(), st>>>(mp, mq, prm);
    g_launches++;
    return cudaGetLastError();
}

}  // namespace pfsm
