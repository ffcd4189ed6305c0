// Split-precision GEMM on the 5th-generation tensor cores (tcgen05 + TMEM, operands fed by TMA)
// for the products of Eq. 11 in the mixed forms, and the FP32-accurate products of the mixed-form
// Gram-Schmidt.
//
//   C[r, c] = sum over slice pairs (a, b) of sum_k P_a[r, k] * Q_b[c, k]
//
// P and Q are FP64 matrices held as BF16 (3 slices) or TF32 (2 slices) pieces, x = sum_s x_s with
// each x_s the rounding of the remainder left by the earlier slices. Pairs of total order below
// the slice count are accumulated into ONE FP32 accumulator in tensor memory (6 products for
// BF16, 3 for TF32). The epilogue applies the Eq. 11 algebra (TC_EPI_* modes) and can write the
// BF16/TF32 slices of its own result, the operand of the next product.
//
// Persistent CTAs (one per SM, 192 threads) walk the output tiles (128 x BN, BN = 64, 96 or 128:
// the width that fills the SMs best for the product's shape is measured once per shape class by
// tune_tc_tile). Warp 0 issues the TMA loads: one pipeline stage holds every slice of P and of Q
// for one 128-byte K block, so each slice tile is loaded once and feeds all the pairs that use
// it. Warp 1 owns a double-buffered TMEM accumulator (2 x 128 columns) and issues tcgen05.mma
// from one lane, so the MMAs of tile i + 1 run while warps 2-5 drain tile i. The epilogue keeps FP64 only where Eq. 11 accumulates
// (X -= alpha Z, Y_new = Y - alpha (...)) and does the rest in FP32, which is as accurate as the
// split product itself: B300's FP64 pipe (2 FMA/clk/SM) would otherwise outlast the MMAs.
// Every mbarrier wait is bounded by %globaltimer: a wait that gives up records PFSM_ERR_TIMEOUT
// in the status word; all roles then stop, the loads and MMAs in flight are waited for
// (bounded), TMEM is freed and the CTA exits.
#include <map>
#include <mutex>
#include <tuple>

#include "tc_common.cuh"

namespace pfsm {

namespace tc {

constexpr int BM = 128;
constexpr int TILE_BYTES = BM * 128;                 // P tile: 128 rows x 128 bytes
constexpr uint32_t TMEM_COLS = 256;                  // two accumulators, 128 columns apart
constexpr int EBP = 17;                              // epilogue staging row (16 columns + pad)

template <int KIND, int BN> struct Cfg {
    static_assert(BN % 32 == 0 && BN >= 64 && BN <= 128, "tile width");
    static constexpr int NS = KIND == 0 ? 3 : 2;     // slices per operand
    static constexpr int BK = KIND == 0 ? 64 : 32;   // K elements per 128-byte row
    static constexpr int KSTEP = KIND == 0 ? 16 : 8; // K per tcgen05.mma
    static constexpr int Q_TILE = BN * 128;          // Q tile: BN rows x 128 bytes
    static constexpr int STAGE_BYTES = NS * (TILE_BYTES + Q_TILE);
    static constexpr int STAGES = KIND == 0 ? 2 : 3;
    static constexpr int NPAIRS = NS * (NS + 1) / 2;
};

// Output tile t -> (tile row, tile column). Full products walk the tile grid in groups of
// kGroupRows tile rows, the group's rows innermost: the ~148 tiles in flight at a time then share
// a few tile rows of P and each tile column of Q is read from DRAM once per group, not once per
// tile row (at N = 9072 the operands' slices, ~0.5 GB each, are four times L2). Lower-only
// products of square outputs walk the lower triangle (column tile <= row tile) row by row.
constexpr int kGroupRows = 8;

__device__ __forceinline__ void tile_coords(int t, int nrowt, int ncolt, int lower, int &tr, int &tcl)
{
    if (!lower) {
        const int grp = t / (kGroupRows * ncolt), r_first = grp * kGroupRows;
        const int nr = min(kGroupRows, nrowt - r_first);
        const int loc = t - grp * kGroupRows * ncolt;
        tr = r_first + loc % nr;
        tcl = loc / nr;
        return;
    }
    int r = (int)((sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);
    while ((r + 1) * (r + 2) / 2 <= t) r++;
    while (r * (r + 1) / 2 > t) r--;
    tr = r;
    tcl = t - r * (r + 1) / 2;
}

}  // namespace tc

template <int KIND, int BN>
__global__ void __launch_bounds__(192, 1)
k_gemm_tc(const __grid_constant__ CUtensorMap mapP, const __grid_constant__ CUtensorMap mapQ, TcParams prm)
{
    using namespace tc;
    using C = Cfg<KIND, BN>;
    extern __shared__ __align__(1024) uint8_t smraw[];
    const uint32_t raw = smem_u32(smraw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    uint8_t *gbase = smraw + (base - raw);
    uint64_t *bars = reinterpret_cast<uint64_t *>(gbase + C::STAGES * C::STAGE_BYTES);
    // bars: [0,S) full, [S,2S) empty, [2S,2S+2) accumulator full, [2S+2,2S+4) accumulator empty,
    // [2S+4] all MMAs done
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 2 * C::STAGES + 5);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
    float *dhi = reinterpret_cast<float *>(tmem_slot + 4);     // per tile column: diag(A) split
    float *dlo = dhi + BN;
    double *ebuf = reinterpret_cast<double *>(dlo + BN);        // epilogue staging, 128 x EBP
    const uint32_t bar_base = smem_u32(bars);
    auto full_bar = [&](int s) { return bar_base + 8u * s; };
    auto empty_bar = [&](int s) { return bar_base + 8u * (C::STAGES + s); };
    auto accf_bar = [&](int b) { return bar_base + 8u * (2 * C::STAGES + b); };
    auto acce_bar = [&](int b) { return bar_base + 8u * (2 * C::STAGES + 2 + b); };
    const uint32_t done_bar = bar_base + 8u * (2 * C::STAGES + 4);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ncolt = (prm.cols + BN - 1) / BN, nrowt = (prm.rows + BM - 1) / BM;
    const int ntiles = prm.lower_only ? nrowt * (nrowt + 1) / 2 : nrowt * ncolt;

    // K-block range of a tile row (the first product only needs the columns its rows' windows cover)
    auto krange = [&](int tr, int &kb0, int &kb1) {
        kb0 = 0;
        kb1 = prm.kblocks;
        if (prm.krange) {
            const int t0 = 2 * tr;
            const int t1 = min(t0 + 1, prm.nrowtiles64 - 1);
            const int kbeg = min(prm.krange[2 * t0], prm.krange[2 * t1]);
            const int kend = max(prm.krange[2 * t0 + 1], prm.krange[2 * t1 + 1]);
            kb0 = kbeg / C::BK;
            kb1 = min(prm.kblocks, (kend + C::BK - 1) / C::BK);
            if (kb1 < kb0) kb1 = kb0;
        }
    };

    if (threadIdx.x == 0) {
        for (int s = 0; s < C::STAGES; s++) {
            mbar_init(full_bar(s), 1);
            mbar_init(empty_bar(s), 1);
        }
        for (int b = 0; b < 2; b++) {
            mbar_init(accf_bar(b), 1);
            mbar_init(acce_bar(b), 128);
        }
        mbar_init(done_bar, 1);
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
            int it = 0, issued = 0;
            bool stop = false;
            for (int t = blockIdx.x; t < ntiles && !stop; t += gridDim.x) {
                int tr, tcl, kb0, kb1;
                tile_coords(t, nrowt, ncolt, prm.lower_only, tr, tcl);
                krange(tr, kb0, kb1);
                for (int kb = kb0; kb < kb1; kb++, it++) {
                    const int s = it % C::STAGES, round = it / C::STAGES;
                    if (round > 0 && !mbar_wait(empty_bar(s), (round - 1) & 1)) {
                        set_status(prm.status, PFSM_ERR_TIMEOUT);
                        *abort_flag = 1;
                        stop = true;
                        break;
                    }
                    if (*abort_flag) { stop = true; break; }
                    const uint32_t st0 = base + s * C::STAGE_BYTES;
                    mbar_expect_tx(full_bar(s), C::STAGE_BYTES);
#pragma unroll
                    for (int a = 0; a < C::NS; a++) {
                        tma_load_3d(st0 + a * TILE_BYTES, &mapP, full_bar(s), kb * C::BK, tr * BM, a);
                        tma_load_3d(st0 + C::NS * TILE_BYTES + a * C::Q_TILE, &mapQ, full_bar(s), kb * C::BK,
                                    tcl * BN, a);
                    }
                    issued = it + 1;
                }
            }
            // leave no copies in flight: wait (bounded) for the last stages filled
            for (int i = (issued > C::STAGES ? issued - C::STAGES : 0); i < issued; i++)
                mbar_wait(full_bar(i % C::STAGES), (i / C::STAGES) & 1);
        }
        __syncwarp();
    } else if (warp == 1) {
        if (lane == 0) {
            int it = 0, lt = 0;
            bool ok = true;
            for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x, lt++) {
                int tr, tcl, kb0, kb1;
                tile_coords(t, nrowt, ncolt, prm.lower_only, tr, tcl);
                krange(tr, kb0, kb1);
                const int buf = lt & 1;
                if (lt >= 2 && !mbar_wait(acce_bar(buf), ((lt >> 1) - 1) & 1)) { ok = false; break; }
                fence_after();
                const uint32_t dacc = tmem_acc + 128u * buf;
                bool first = true;
                for (int kb = kb0; kb < kb1; kb++, it++) {
                    const int s = it % C::STAGES;
                    if (!mbar_wait(full_bar(s), (it / C::STAGES) & 1) || *abort_flag) { ok = false; break; }
                    fence_after();
                    const uint32_t st0 = base + s * C::STAGE_BYTES;
#pragma unroll
                    for (int ord = 0; ord < C::NS; ord++)
#pragma unroll
                        for (int a = 0; a <= ord; a++) {
                            const uint64_t da = sw128_desc(st0 + a * TILE_BYTES);
                            const uint64_t db = sw128_desc(st0 + C::NS * TILE_BYTES + (ord - a) * C::Q_TILE);
#pragma unroll
                            for (int kk = 0; kk < 4; kk++) {   // 4 x 32 bytes of K per 128-byte row
                                umma<KIND, BM, BN>(dacc, da + 2 * kk, db + 2 * kk, first ? 0u : 1u);
                                first = false;
                            }
                        }
                    umma_commit(empty_bar(s));
                }
                umma_commit(accf_bar(buf));   // this tile's sum is complete when its MMAs are
            }
            if (!ok) {
                set_status(prm.status, PFSM_ERR_TIMEOUT);
                *abort_flag = 1;
            }
            // track every issued MMA before TMEM is released (bounded)
            umma_commit(done_bar);
            mbar_wait(done_bar, 0);
        }
        __syncwarp();
    } else {
        // epilogue: warp w reads TMEM lanes 32*(w % 4) .. +31, i.e. tile rows
        const int g = warp & 3;
        const int et = threadIdx.x - 64;                 // 0 .. 127
        int lt = 0;
        for (int t = blockIdx.x; t < ntiles; t += gridDim.x, lt++) {
            int tr, tcl, kb0, kb1;
            tile_coords(t, nrowt, ncolt, prm.lower_only, tr, tcl);
            krange(tr, kb0, kb1);
            const int buf = lt & 1;
            const int row0 = tr * BM, col0 = tcl * BN;
            const int r = row0 + 32 * g + lane;
            // column data of this tile (the previous tile's readers are done: named barrier)
            asm volatile("bar.sync 1, 128;" ::: "memory");
            if (prm.d && et < BN) {
                const int c = col0 + et;
                const double dv = c < prm.cols ? prm.d[c] : 0.0;
                const float h = (float)dv;
                dhi[et] = h;
                dlo[et] = (float)(dv - (double)h);
            }
            asm volatile("bar.sync 1, 128;" ::: "memory");
            const bool got = mbar_wait(accf_bar(buf), (lt >> 1) & 1);
            if (!got) {
                set_status(prm.status, PFSM_ERR_TIMEOUT);
                *abort_flag = 1;
            }
            // one decision for all four epilogue warps (they meet at named barriers)
            int stop;
            asm volatile("{\n\t.reg .pred p, q;\n\tsetp.ne.s32 q, %1, 0;\n\t"
                         "bar.red.or.pred p, 1, 128, q;\n\tselp.s32 %0, 1, 0, p;\n\t}"
                         : "=r"(stop) : "r"((!got || *abort_flag) ? 1 : 0) : "memory");
            if (stop) break;
            fence_after();
            const bool have_acc = kb1 > kb0;
            const bool row_ok = r < prm.rows;
            float ehi = 0.0f, elo = 0.0f;
            double ar = 0.0;
            int win_lo = 0, win_hi = 0;
            if (row_ok) {
                if (prm.eps) {
                    const double ev = prm.eps[r];
                    ehi = (float)ev;
                    elo = (float)(ev - (double)ehi);
                }
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
            double(*eb)[EBP] = reinterpret_cast<double(*)[EBP]>(ebuf) + 32 * g;   // this warp's staging
            const int R0 = row0 + 32 * g;
            // coalesced access of the warp's 32 x 16 block: lanes 0-15 row 2i, lanes 16-31 row 2i+1
            auto in_block = [&](int rr, int c) { return R0 + rr < prm.rows && c < prm.cols && !(prm.lower_only && c > R0 + rr); };
            // all 16 loads of a lane in flight at once (one L2 round trip per block)
            auto load_block = [&](const double *src, int C0) {
#pragma unroll
                for (int i = 0; i < 16; i++) {
                    const int rr = 2 * i + (lane >> 4), cc = lane & 15, c = C0 + cc;
                    if (in_block(rr, c)) eb[rr][cc] = src[(int64_t)(R0 + rr) * prm.ldo + c];
                }
                __syncwarp();
            };
            auto store_block = [&](double *dst, int C0, bool slices) {
                __syncwarp();
#pragma unroll 4
                for (int i = 0; i < 16; i++) {
                    const int rr = 2 * i + (lane >> 4), cc = lane & 15, c = C0 + cc;
                    if (in_block(rr, c)) {
                        const double x = eb[rr][cc];
                        dst[(int64_t)(R0 + rr) * prm.ldo + c] = x;
                        if (slices)
                            store_slices_f32<KIND>(prm.out_slices, prm.sl_stride, (int64_t)(R0 + rr) * prm.sl_ld + c,
                                                   prm.out_ns, (float)x);
                    }
                }
                __syncwarp();
            };
            const bool sl = prm.out_ns > 0;
            for (int chunk = 0; chunk < BN / 32; chunk++) {
                uint32_t v[32];
                if (have_acc) {
                    tmem_ld32(tmem_acc + ((uint32_t)(32 * g) << 16) + 128u * buf + 32 * chunk, v);
                } else {
#pragma unroll
                    for (int j = 0; j < 32; j++) v[j] = 0u;
                }
                if (chunk == BN / 32 - 1) {     // accumulator drained: hand it back to the MMA warp
                    fence_before();
                    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(acce_bar(buf)) : "memory");
                }
#pragma unroll
                for (int h = 0; h < 2; h++) {
                    const int C0 = col0 + 32 * chunk + 16 * h;
                    if (prm.epi == TC_EPI_STORE || prm.epi == TC_EPI_Y0) {
#pragma unroll
                        for (int j = 0; j < 16; j++) {
                            const int c = C0 + j;
                            float x = __uint_as_float(v[16 * h + j]);
                            if (prm.epi == TC_EPI_Y0 && c >= win_lo && c < win_hi) x = 0.0f;
                            eb[lane][j] = (double)x;
                        }
                        store_block(prm.out, C0, sl);
                    } else if (prm.epi == TC_EPI_RSUB) {
                        load_block(prm.V, C0);
#pragma unroll
                        for (int j = 0; j < 16; j++) eb[lane][j] -= (double)__uint_as_float(v[16 * h + j]);
                        store_block(prm.out, C0, false);
                    } else {
                        // the accumulated operand (X for Z, Y_old for Y_new): each lane's own row,
                        // 16 contiguous doubles straight into registers, in flight together with
                        // the staged loads of V below (one L2 round trip for both)
                        double xo[16];
                        {
                            const double *xs = (prm.epi == TC_EPI_Z) ? prm.X : prm.Yold;
                            const int rw = R0 + lane;
#pragma unroll
                            for (int j = 0; j < 16; j++)
                                xo[j] = in_block(lane, C0 + j) ? xs[(int64_t)rw * prm.ldo + C0 + j] : 0.0;
                        }
                        // (A - eps_r I) applied to the FP64 operand's diagonal part, in FP32:
                        // (d_c - eps_r) from hi/lo pieces, times the operand rounded to FP32
                        float t[16];
                        load_block(prm.V, C0);
#pragma unroll
                        for (int j = 0; j < 16; j++) {
                            const int cl = C0 - col0 + j;
                            const float diff = (dhi[cl] - ehi) + (dlo[cl] - elo);
                            t[j] = fmaf(diff, (float)eb[lane][j], __uint_as_float(v[16 * h + j]));
                        }
                        __syncwarp();
#pragma unroll
                        for (int j = 0; j < 16; j++) eb[lane][j] = fma(-ar, (double)t[j], xo[j]);
                        if (prm.epi == TC_EPI_Z) {                       // X -= alpha Z in FP64
                            store_block(prm.X, C0, false);
#pragma unroll
                            for (int j = 0; j < 16; j++) eb[lane][j] = (double)t[j];
                            store_block(prm.out, C0, sl);
                        } else {   // TC_EPI_YN: Y - alpha (E Z + (D - eps) Z), accumulated in FP64
                            store_block(prm.out, C0, sl);
                        }
                    }
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

cudaError_t make_slice_map64(CUtensorMap *map, const SliceBuf &b, int box_rows, int box_slices)
{
    EncodeTiledFn fn = encode_fn();
    if (!fn) return cudaErrorNotSupported;
    const int esz = b.kind == 0 ? 2 : 4;
    cuuint64_t dims[3] = {(cuuint64_t)b.ld, (cuuint64_t)b.rows, (cuuint64_t)b.ns};
    cuuint64_t strides[2] = {(cuuint64_t)b.ld * esz, (cuuint64_t)b.ld * b.rows * esz};
    cuuint32_t box[3] = {(cuuint32_t)(64 / esz), (cuuint32_t)box_rows, (cuuint32_t)box_slices};
    cuuint32_t estr[3] = {1u, 1u, 1u};
    CUresult r = fn(map, b.kind == 0 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3,
                    b.ptr, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

namespace {

template <int KIND, int BN>
size_t tc_smem_bytes()
{
    return (size_t)tc::Cfg<KIND, BN>::STAGES * tc::Cfg<KIND, BN>::STAGE_BYTES + 1024 + 256 + 2 * BN * 4 +
           128 * tc::EBP * 8;
}

}  // namespace

int sm_count()
{
    static int n = 0;
    if (!n) {
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) n = 148;
    }
    return n;
}

cudaError_t configure_tc_kernels()
{
    cudaError_t e = cudaSuccess;
    auto set = [&](const void *fn, size_t bytes) {
        if (e == cudaSuccess) e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    };
    set((const void *)k_gemm_tc<0, 64>, tc_smem_bytes<0, 64>());
    set((const void *)k_gemm_tc<0, 96>, tc_smem_bytes<0, 96>());
    set((const void *)k_gemm_tc<0, 128>, tc_smem_bytes<0, 128>());
    set((const void *)k_gemm_tc<1, 64>, tc_smem_bytes<1, 64>());
    set((const void *)k_gemm_tc<1, 96>, tc_smem_bytes<1, 96>());
    set((const void *)k_gemm_tc<1, 128>, tc_smem_bytes<1, 128>());
    return e;
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
    // tile width: the caller's (tuned) choice, 128 for lower-triangle products (square tiles)
    const int bn = (prm.lower_only || (prm.bn != 64 && prm.bn != 96)) ? 128 : prm.bn;
    if ((e = make_slice_map(&mp, P, tc::BM)) != cudaSuccess) return e;
    if ((e = make_slice_map(&mq, Q, bn)) != cudaSuccess) return e;
    if (P.kind != Q.kind || P.ns != (P.kind == 0 ? 3 : 2) || Q.ns != P.ns || P.ld != Q.ld) return cudaErrorInvalidValue;
    if (prm.lower_only && prm.rows != prm.cols) return cudaErrorInvalidValue;
    prm.bk = P.kind == 0 ? 64 : 32;
    prm.kblocks = (int)(P.ld / prm.bk);
    prm.npairs = P.ns * (P.ns + 1) / 2;
    if (out_sl) {
        if (out_sl->ns != P.ns || out_sl->kind != P.kind) return cudaErrorInvalidValue;
        prm.out_slices = out_sl->ptr;
        prm.sl_ld = out_sl->ld;
        prm.sl_stride = out_sl->ld * out_sl->rows;
        prm.out_ns = out_sl->ns;
    } else {
        prm.out_ns = 0;
    }
    const int nrowt = (prm.rows + tc::BM - 1) / tc::BM, ncolt = (prm.cols + bn - 1) / bn;
    const int ntiles = prm.lower_only ? nrowt * (nrowt + 1) / 2 : nrowt * ncolt;
    if (ntiles == 0) return cudaSuccess;
    const unsigned grid = (unsigned)(ntiles < sm_count() ? ntiles : sm_count());
#define PFSM_TC_LAUNCH(K_, B_) k_gemm_tc<K_, B_><<<grid, 192, tc_smem_bytes<K_, B_>(), st>>>(mp, mq, prm)
    if (P.kind == 0) {
        if (bn == 64) PFSM_TC_LAUNCH(0, 64);
        else if (bn == 96) PFSM_TC_LAUNCH(0, 96);
        else PFSM_TC_LAUNCH(0, 128);
    } else {
        if (bn == 64) PFSM_TC_LAUNCH(1, 64);
        else if (bn == 96) PFSM_TC_LAUNCH(1, 96);
        else PFSM_TC_LAUNCH(1, 128);
    }
#undef PFSM_TC_LAUNCH
    g_launches++;
    return cudaGetLastError();
}

// Tile-width autotuner: every candidate width is timed (CUDA events, private stream, after one
// warm-up launch, best of three) on a plain product C = P Q^T of the caller's shape, with the
// caller's slice buffers as operands and `scratch` (rows x cols doubles) as output, and the
// fastest width is kept per (device, slice kind, shape class). The operands' contents do not
// matter for the timing. Runs synchronously; returns 128 if a candidate fails to launch.
int tune_tc_tile(const SliceBuf &P, const SliceBuf &Q, int rows, int cols, double *scratch)
{
    static std::mutex mu;
    static std::map<std::tuple<int, int, int, int, int64_t>, int> cache;
    int dev = 0;
    cudaGetDevice(&dev);
    const auto key = std::make_tuple(dev, P.kind, (rows + 63) / 64, (cols + 63) / 64, (P.ld + 63) / 64);
    {
        std::lock_guard<std::mutex> lk(mu);
        auto it = cache.find(key);
        if (it != cache.end()) return it->second;
    }
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int best = 128;
    float best_ms = 1e30f;
    int32_t *status = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) == cudaSuccess && cudaEventCreate(&e0) == cudaSuccess &&
        cudaEventCreate(&e1) == cudaSuccess && cudaMalloc((void **)&status, sizeof(int32_t)) == cudaSuccess &&
        cudaMemsetAsync(status, 0, sizeof(int32_t), st) == cudaSuccess) {
        const int cands[3] = {128, 96, 64};
        for (int bn : cands) {
            TcParams p{};
            p.rows = rows; p.cols = cols; p.epi = TC_EPI_STORE; p.out = scratch; p.ldo = cols;
            p.status = status; p.bn = bn;
            if (launch_gemm_tc(P, Q, p, nullptr, st) != cudaSuccess) continue;
            float ms = 1e30f;
            bool ok = true;
            for (int r = 0; r < 3 && ok; r++) {
                float t = 0.0f;
                ok = cudaEventRecord(e0, st) == cudaSuccess && launch_gemm_tc(P, Q, p, nullptr, st) == cudaSuccess &&
                     cudaEventRecord(e1, st) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess &&
                     cudaEventElapsedTime(&t, e0, e1) == cudaSuccess;
                if (ok && t < ms) ms = t;
            }
            if (ok && ms < best_ms) { best_ms = ms; best = bn; }
        }
        int32_t hs = 0;
        cudaMemcpyAsync(&hs, status, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
        cudaStreamSynchronize(st);
        if (hs != 0) best = 128;
    }
    cudaGetLastError();
    if (status) cudaFree(status);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st) cudaStreamDestroy(st);
    std::lock_guard<std::mutex> lk(mu);
    cache[key] = best;
    return best;
}

}  // namespace pfsm
