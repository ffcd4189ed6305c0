// FP64-accurate products on the BF16 tensor cores (tcgen05 + TMEM, TMA-fed): the error-free
// splitting of Ozaki, Ogita, Oishi and Rump (2012), arranged for B300, where the DFMA pipe gives
// 1.2 TFLOP/s and the BF16 tensor cores about 1.75 PFLOP/s.
//
// Splitting (k_oz_split): every row r of an operand is scaled by its own power of two 2^-e_r so
// that |x| < 1, rounded to a 48-bit fixed-point integer q (|q| <= 2^48), and q is cut into S = 7
// balanced base-128 digits n_0 .. n_6 (n_s in [-64, 64) for s >= 1, |n_0| <= 64), each an integer
// that BF16 holds exactly:
//   x = 2^e_r sum_s n_s 2^-(6 + 7 s)   (to 2^-49 of the row's largest entry).
// Product (k_gemm_oz): C[r, c] = sum_L 2^(e_r + e_c - 12 - 7 L) sum_{s+t=L} sum_k n_s[r,k] m_t[c,k].
// Every digit product has |n m| <= 2^12 and level L <= 6 has L + 1 pairs, so a level summed over a
// K chunk of 512 terms stays below 7 * 2^21 < 2^24 and the FP32 accumulation in tensor memory is
// EXACT. Levels L = 0 .. OZ_LEVELS-1 = 6 are kept (all 28 pairs with s + t <= 6). Every entry,
// however small, has O(1) low digits, so the products of the first dropped level L add up like a
// random walk over K: about sqrt((L + 1) K) 2^-7L / 3 relative to 2^(e_r + e_c) -- for L = 7
// (the default) about sqrt(K) 2^-49, the size of the operands' own rounding. Products that only
// need FP32-class accuracy ask for fewer levels (5 levels: about sqrt(6 K) 2^-35 / 3).
//
// CTA: 192 threads, a 128 x 32 output tile. All levels accumulate at once, each in its own
// 32-column FP32 accumulator in tensor memory, in one of two 256-column buffers that alternate
// between exact K chunks (the drain of one chunk overlaps the MMAs of the next). A pipeline stage
// (3 of them) holds every digit slice of P and of Q for one 32-element (64-byte, 64-byte-swizzled)
// K block, 70 KB loaded by two TMA copies. Q's slice tiles sit back to back in the stage, one SW64
// layout of 7 x 32 rows, and level L's accumulator at columns 32 L, so P slice s times Q slices
// 0 .. LV-1-s is ONE MMA (N = 32 (LV - s)) whose output columns are exactly the accumulators of
// levels s .. LV-1: 7 MMAs per 16 K for 28 slice pairs, each reading the 4 KB P tile once. The
// s = 0 MMA covers every level, so it alone carries the "overwrite" flag at a chunk's start.
// Warp 0: TMA. Warp 1: TMEM owner and MMA issuer. Warps 2-5: at the end of each exact K chunk,
// drain the level sums (one row per thread) into float-float registers with exact power-of-two
// scales; finally one FP64 conversion per entry and row-contiguous stores through shared memory.
// The epilogue can add an exact FP64 diagonal term C[r, c] += V[r, c] d[c] (for products with
// A = diag(d) + E whose digits cover E only). All mbarrier waits are bounded.
#include "fp64_util.cuh"
#include "tc_common.cuh"

namespace pfsm {

namespace oz {

constexpr int BM = 128, BN = 32, KB = 32;         // tile, K block (32 BF16 = 64 bytes)
constexpr int P_TILE = BM * 64, Q_TILE = BN * 64;  // bytes per slice per K block
constexpr int STAGES = 3;
constexpr int MAX_STAGE_BYTES = OZ_SLICES * (P_TILE + Q_TILE);
constexpr uint32_t TMEM_COLS = 512;               // two buffers of 256 columns, level L at 32 L
constexpr uint32_t BUF_COLS = 256;
constexpr int KCHUNK = 512;                       // K terms per exact level sum
constexpr int kGroupRows = 8;                     // row tiles per group of the tile walk
constexpr int BETA = 7;                           // bits per digit
constexpr int QBITS = BETA * OZ_SLICES - 1;       // fixed-point bits of q (48)
static_assert(OZ_LEVELS <= OZ_SLICES && OZ_LEVELS <= 8, "the s = 0 MMA must span every level");
static_assert(OZ_LEVELS * BN <= (int)BUF_COLS, "levels of one buffer exceed its columns");
static_assert(KCHUNK % KB == 0 && (double)KCHUNK * OZ_LEVELS * 4096.0 < 16777216.0,
              "a level sum over one K chunk must stay exact in FP32");

}  // namespace oz

// ---- splitting -------------------------------------------------------------------------------

// One warp per row: exponent of the row's largest |entry| and the S digits of every entry.
// zero_diag: digits of the off-diagonal part (entry (r, r) taken as 0, its value stored in d[r]).
// Input in FP64 or FP32 (an FP32 operand's digits are exact: 24 bits fit in the 48-bit grid of its
// row unless the entry is below 2^-24 of the row's largest).
// B300 retires one FP64 warp instruction per 16 cycles per SM, and the integer pipe two per cycle,
// so each entry costs one FP64 instruction: the row maximum compares bit patterns (IEEE order of
// magnitudes is the integer order of non-negative bit patterns), q = rn(x 2^(QBITS - e)) comes
// from one FMA with 1.5 2^52 (the sum's low significand bits are q, rounded to nearest even: the
// same integer as the product and conversion), and with q' = q + sum_i 64 128^i the balanced
// digits are the 7-bit fields of q' minus 64 (bit-field extracts on 32-bit halves), whose BF16
// values come from FP32 adds.
__device__ __forceinline__ unsigned long long oz_bits(double x) { return (unsigned long long)__double_as_longlong(x); }

// BF16 bits of (field - 64) for a 7-bit field: 1.5 2^23 + field is exact, and so is the BF16 of
// the (<= 7 significant bits) difference
__device__ __forceinline__ unsigned short oz_digit_bf16(uint32_t field)
{
    const float f = __int_as_float(0x4B400000 | (int)field) - 12582976.0f;   // 1.5 2^23 + 64
    return (unsigned short)(__float_as_uint(f) >> 16);
}

// The digits of one row of `cols` entries (lane `lane` of one warp): exponent e of the row's
// largest |entry| into *eout and the S digit slices of entry c at out[c + s * sstride]; columns
// cols .. fill_to - 1 get zero digits. diag_col >= 0: that entry is taken as 0 (its value stored
// in *dval when dval is given).
// f 2^e as a double for a float f: sign, exponent and significand moved by integer operations
// (B300's FP64 pipe retires one warp instruction per 16 cycles per SM, and the float-to-double
// conversion and ldexp run on it); zeros directly, the rare subnormal, infinite or out-of-range
// cases by the conversion and ldexp. Equal to ldexp((double)f, e) for every input.
__device__ __forceinline__ double oz_f2d_scaled(float f, int e)
{
    const uint32_t u = __float_as_uint(f);
    if ((u << 1) == 0u) return __longlong_as_double((long long)(u >> 31) << 63);
    const int ex = (int)((u >> 23) & 0xFFu);
    const int dex = ex - 127 + 1023 + e;
    if (ex == 0 || ex == 255 || dex <= 0 || dex >= 2047) return ldexp((double)f, e);
    return __longlong_as_double((long long)(((unsigned long long)(u >> 31) << 63) | ((unsigned long long)dex << 52) |
                                            ((unsigned long long)(u & 0x7FFFFFu) << 29)));
}

// An exact FP32 integer |v| < 2^22 (a level sum of at most 64-term digit products) as an int32:
// adding 1.5 2^23 leaves it, exactly, in the low significand bits.
__device__ __forceinline__ int oz_lvl_i32(uint32_t raw)
{
    return __float_as_int(__uint_as_float(raw) + 12582912.0f) - 0x4B400000;
}

// T = sum_L v_L 128^(LV-1-L) over the raw level sums of column j: with K <= 64, |v_L| <=
// (L + 1) 64^2 K = (L + 1) 2^18, so |T| < 2^61 and the sum is exact in 64-bit integers. Seven
// levels go in int32 pairs (v_{L+1} + 128 v_L stays below 2^28) before the 64-bit adds.
template <int N>
__device__ __forceinline__ long long oz_levels_i64(const uint32_t (&v)[OZ_LEVELS][N], int j, int LV)
{
    if (LV == 7 && OZ_LEVELS == 7) {
        const int i0 = oz_lvl_i32(v[0][j]), i1 = oz_lvl_i32(v[1][j]), i2 = oz_lvl_i32(v[2][j]);
        const int i3 = oz_lvl_i32(v[3][j]), i4 = oz_lvl_i32(v[4][j]), i5 = oz_lvl_i32(v[5][j]);
        const int i6 = oz_lvl_i32(v[6][j]);
        const int p = i6 + i5 * 128, q = i4 + i3 * 128, r = i2 + i1 * 128;
        return (long long)i0 * (1ll << 42) + (long long)r * (1ll << 28) + (long long)q * (1ll << 14) + (long long)p;
    }
    long long t = 0;
#pragma unroll
    for (int L = 0; L < OZ_LEVELS; L++)
        if (L < LV) t = t * 128 + oz_lvl_i32(v[L][j]);
    return t;
}

template <typename T>
__device__ __forceinline__ void oz_split_row(const T *__restrict__ x, int64_t cols, int64_t fill_to, int64_t diag_col,
                                             double *dval, unsigned short *__restrict__ out, int64_t sstride,
                                             int32_t *eout, int lane)
{
    static_assert(OZ_SLICES == 7 && oz::BETA == 7, "digit fields are laid out for seven 7-bit digits");
    const bool zero_diag = diag_col >= 0;
    auto val = [&](int64_t c) -> double { return (zero_diag && c == diag_col) ? 0.0 : (double)x[c]; };
    if (zero_diag && lane == 0 && dval) *dval = (double)x[diag_col];
    unsigned long long mb = 0ull;
    for (int64_t c = lane; c < cols; c += 32) {
        unsigned long long b;
        if (sizeof(T) == 8) b = oz_bits((double)x[c]) & 0x7FFFFFFFFFFFFFFFull;
        else b = (unsigned long long)(__float_as_uint((float)x[c]) & 0x7FFFFFFFu);
        mb = max(mb, (zero_diag && c == diag_col) ? 0ull : b);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mb = max(mb, __shfl_xor_sync(0xffffffffu, mb, o));
    // e with max|x| = f 2^e, f in [1/2, 1) (frexp); e = 0 for a zero row
    int e = 0;
    if (sizeof(T) == 8) {
        const int ex = (int)(mb >> 52);
        if (ex > 0) e = ex - 1022;
        else if (mb != 0ull) e = -1010 - __clzll((long long)mb);                // subnormal
    } else {
        const int ex = (int)(mb >> 23);
        if (ex > 0) e = ex - 126;
        else if (mb != 0ull) e = -117 - __clz((int)mb);
    }
    if (lane == 0) *eout = e;
    // one digit row: q from t = x 2^(QBITS - e) + 1.5 2^52 (|x 2^(QBITS - e)| < 2^QBITS <= 2^51, so
    // the sum is rounded to an integer held in the low significand bits)
    constexpr double kMagic = 6755399441055744.0;                     // 1.5 2^52
    constexpr long long kBias = 64ll * (((1ll << 42) - 1) / 127);     // sum_{i < 6} 64 128^i
    // the seven BF16 digits of t (low half: slice 6 .. high: slice 0), as 16-bit patterns
    auto digits = [&](double t, uint32_t (&d)[OZ_SLICES]) {
        const long long q = (long long)(oz_bits(t) - oz_bits(kMagic)) + kBias;
        const uint32_t lo = (uint32_t)q, hi = (uint32_t)((unsigned long long)q >> 32);
        d[6] = oz_digit_bf16(lo & 127u);
        d[5] = oz_digit_bf16((lo >> 7) & 127u);
        d[4] = oz_digit_bf16((lo >> 14) & 127u);
        d[3] = oz_digit_bf16((lo >> 21) & 127u);
        d[2] = oz_digit_bf16(__funnelshift_r(lo, hi, 28) & 127u);
        d[1] = oz_digit_bf16((hi >> 3) & 127u);
        d[0] = oz_digit_bf16((uint32_t)(((int)hi >> 10) + 64));      // top digit q' >> 42, |n_0| <= 64
    };
    // two adjacent entries per lane, their digits stored as one 32-bit word per slice (row starts
    // and slice strides are even); past the row's end the pair's second entry is zero, whose zero
    // digits land in the row's padding, which the products read as zero K terms anyway
    auto emit2 = [&](int64_t c, double t0, double t1) {
        uint32_t d0[OZ_SLICES], d1[OZ_SLICES];
        digits(t0, d0);
        digits(t1, d1);
#pragma unroll
        for (int sl = 0; sl < OZ_SLICES; sl++)
            *reinterpret_cast<uint32_t *>(out + c + sl * sstride) = d0[sl] | (d1[sl] << 16);
    };
    const int sh = oz::QBITS - e;
    if (sh <= 1000) {                                                 // 2^sh is a double: one FMA
        const double sc = ldexp(1.0, sh);
        for (int64_t c = 2 * lane; c < cols; c += 64)
            emit2(c, fma(val(c), sc, kMagic), (c + 1 < cols) ? fma(val(c + 1), sc, kMagic) : kMagic);
    } else {                                                          // rows below 2^-952: two factors
        const double sc1 = ldexp(1.0, sh / 2), sc2 = ldexp(1.0, sh - sh / 2);
        for (int64_t c = 2 * lane; c < cols; c += 64)
            emit2(c, fma(val(c) * sc1, sc2, kMagic), (c + 1 < cols) ? fma(val(c + 1) * sc1, sc2, kMagic) : kMagic);
    }
    for (int64_t c = cols + lane; c < fill_to; c += 32)
#pragma unroll
        for (int s = 0; s < OZ_SLICES; s++) out[c + s * sstride] = 0;
}

template <typename T>
__global__ void k_oz_split(const T *__restrict__ src, int64_t rows, int64_t cols, int64_t ld,
                           __nv_bfloat16 *__restrict__ dst, int64_t sl_ld, int64_t sstride,
                           int32_t *__restrict__ exps, int zero_diag, double *__restrict__ d)
{
    const int lane = threadIdx.x & 31;
    const int64_t r = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (r >= rows) return;
    oz_split_row<T>(src + r * ld, cols, cols, zero_diag ? r : -1, d ? d + r : nullptr,
                    reinterpret_cast<unsigned short *>(dst + r * sl_ld), sstride, exps + r, lane);
}

// Batched over windows (blockIdx.y = window z): with n = ext[z] - ext_off, rows i in [0, n) (or
// [0, rows_fixed) when rows_fixed > 0, or [0, rext[z]) when rext is given) of the n-column block
// whose first entry is
// src + z * src_z + row0 * ld + col0 (ld the row stride), into digit rows
// z * dst_zrow + dst_row0 + i with K index = column - col0; columns n .. fill_to - 1 of each row
// get zero digits (the K padding the products read). zero_diag: entry (i, i) of the block is taken
// as 0 and its value stored in dout[digit row].
__global__ void k_oz_split_win(const double *__restrict__ src, int64_t src_z, int64_t ld, int64_t row0, int64_t col0,
                               const int32_t *__restrict__ ext, int ext_off, int rows_fixed,
                               const int32_t *__restrict__ rext, int zero_diag, double *__restrict__ dout,
                               int64_t fill_to,
                               __nv_bfloat16 *__restrict__ dst, int64_t dst_zrow, int64_t dst_row0, int64_t sl_ld,
                               int64_t sstride, int32_t *__restrict__ exps)
{
    const int z = blockIdx.y;
    const int lane = threadIdx.x & 31;
    const int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int64_t n = max(0, ext[z] - ext_off);                      // the window's extent
    const int64_t nrows = rows_fixed > 0 ? rows_fixed : (rext ? rext[z] : n);
    if (i >= nrows) return;
    const double *x = src + (int64_t)z * src_z + (row0 + i) * ld + col0;
    const int64_t drow = (int64_t)z * dst_zrow + dst_row0 + i;
    oz_split_row<double>(x, n, fill_to, zero_diag ? i : -1, zero_diag ? dout + drow : nullptr,
                         reinterpret_cast<unsigned short *>(dst + drow * sl_ld), sstride, exps + drow, lane);
}

// ---- product ---------------------------------------------------------------------------------

__global__ void __launch_bounds__(192, 1)
k_gemm_oz(const __grid_constant__ CUtensorMap mapP, const __grid_constant__ CUtensorMap mapQ, OzParams prm)
{
    using namespace tc;
    using namespace oz;
    const int z = blockIdx.z;
    // CTAs start in blockIdx order; the tiles are walked in groups of kGroupRows tile rows, the
    // group's rows innermost, so the CTAs resident together share a few row tiles of P and each
    // column tile of Q is read from DRAM once per group instead of once per row tile
    int ty, tx;
    {
        const int gx = gridDim.x, lin = blockIdx.y * gx + blockIdx.x;
        const int grp = lin / (kGroupRows * gx), r_first = grp * kGroupRows;
        const int nr = min(kGroupRows, (int)gridDim.y - r_first);
        const int loc = lin - grp * kGroupRows * gx;
        ty = r_first + loc % nr;
        tx = loc / nr;
    }
    const int row0 = prm.row_base + ty * BM;
    const int col0 = (prm.cols_from_zero ? 0 : prm.row_base) + prm.col_off + tx * BN;
    const int rows_lim = prm.ext ? prm.ext[z] : prm.rows;
    const int cols_lim = prm.ext_c ? prm.ext_c[z] : (prm.ext ? prm.ext[z] : prm.cols);
    if (row0 >= rows_lim || col0 >= cols_lim) return;              // tile outside this window
    if (prm.lower_only && col0 > row0 + BM - 1) return;           // whole tile above the diagonal
    const int64_t zr = (int64_t)z * prm.zrow;                      // operand row offsets
    const int64_t zq = (int64_t)z * (prm.zrow_q ? prm.zrow_q : prm.zrow);
    double *Cz = prm.C + (int64_t)z * prm.zc;
    const int LV = (prm.levels > 0 && prm.levels < OZ_LEVELS) ? prm.levels : OZ_LEVELS;   // levels 0 .. LV-1
    const int NSL = LV;                                            // slices that take part (s, t < LV)
    const int stage_bytes = NSL * (P_TILE + Q_TILE);
    extern __shared__ __align__(1024) uint8_t smraw[];
    const uint32_t raw = smem_u32(smraw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    uint8_t *gbase = smraw + (base - raw);
    uint64_t *bars = reinterpret_cast<uint64_t *>(gbase + STAGES * MAX_STAGE_BYTES);
    // bars: [0, S) full, [S, 2S) empty, then per TMEM buffer "chunk summed" x2, "chunk drained"
    // x2, and "all MMAs done"
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 2 * STAGES + 5);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
    int *ecol = reinterpret_cast<int *>(tmem_slot + 2);           // BN column exponents
    const uint32_t bar_base = smem_u32(bars);
    auto full_bar = [&](int s) { return bar_base + 8u * s; };
    auto empty_bar = [&](int s) { return bar_base + 8u * (STAGES + s); };
    auto accf_bar = [&](int b) { return bar_base + 8u * (2 * STAGES + b); };
    auto acce_bar = [&](int b) { return bar_base + 8u * (2 * STAGES + 2 + b); };
    const uint32_t done_bar = bar_base + 8u * (2 * STAGES + 4);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    // 32-element K blocks kb_lo .. kb_lo + nkb - 1: a lower-triangular P has no entries beyond
    // column row0 + BM - 1; with krange64 only the K range of the tile's rows (union of the ranges
    // of its two 64-row tiles) is read
    int kb_lo = 0, kb_hi = prm.p_lower ? min(prm.kblocks, (row0 + BM + KB - 1) / KB) : prm.kblocks;
    if (prm.krange64) {
        const int t0 = row0 / 64, t1 = min(t0 + 1, prm.nrowtiles64 - 1);
        const int kbeg = min(prm.krange64[2 * t0], prm.krange64[2 * t1]);
        const int kend = max(prm.krange64[2 * t0 + 1], prm.krange64[2 * t1 + 1]);
        kb_lo = min(kbeg / KB, kb_hi);
        kb_hi = max(kb_lo, min(kb_hi, (kend + KB - 1) / KB));
    }
    const int nkb = kb_hi - kb_lo;
    const int kb_per_chunk = KCHUNK / KB;
    const int nch = (nkb + kb_per_chunk - 1) / kb_per_chunk;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; s++) {
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
    for (int j = threadIdx.x; j < BN; j += blockDim.x)
        ecol[j] = (col0 + j < cols_lim) ? prm.eq[zq + col0 + j] : 0;
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(smem_u32(tmem_slot)), "r"(TMEM_COLS) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem_acc = *tmem_slot;
    auto stageP = [&](int s, int sl) { return base + s * MAX_STAGE_BYTES + sl * P_TILE; };
    auto stageQ = [&](int s, int sl) { return base + s * MAX_STAGE_BYTES + NSL * P_TILE + sl * Q_TILE; };

    if (warp == 0) {
        if (lane == 0) {
            int issued = 0;
            for (int kb = 0; kb < nkb; kb++) {
                const int s = kb % STAGES, round = kb / STAGES;
                if (round > 0 && !mbar_wait(empty_bar(s), (round - 1) & 1)) {
                    set_status(prm.status, PFSM_ERR_TIMEOUT);
                    *abort_flag = 1;
                    break;
                }
                if (*abort_flag) break;
                mbar_expect_tx(full_bar(s), stage_bytes);
                tma_load_3d(stageP(s, 0), &mapP, full_bar(s), (kb_lo + kb) * KB, (int)(zr + row0), 0);
                tma_load_3d(stageQ(s, 0), &mapQ, full_bar(s), (kb_lo + kb) * KB, (int)(zq + col0), 0);
                issued = kb + 1;
            }
            for (int i = (issued > STAGES ? issued - STAGES : 0); i < issued; i++)
                mbar_wait(full_bar(i % STAGES), (i / STAGES) & 1);
        }
        __syncwarp();
    } else if (warp == 1) {
        if (lane == 0) {
            bool ok = true;
            for (int ch = 0; ch < nch && ok; ch++) {
                const int buf = ch & 1;
                // the buffer's previous chunk (ch - 2) must be drained before it is overwritten
                if (ch >= 2 && !mbar_wait(acce_bar(buf), ((ch >> 1) - 1) & 1)) { ok = false; break; }
                fence_after();
                const uint32_t dbuf = tmem_acc + BUF_COLS * buf;
                const int kbA = ch * kb_per_chunk, kbB = min(nkb, kbA + kb_per_chunk);
                for (int kb = kbA; kb < kbB && ok; kb++) {
                    const int s = kb % STAGES;
                    if (!mbar_wait(full_bar(s), (kb / STAGES) & 1) || *abort_flag) { ok = false; break; }
                    fence_after();
                    for (int h = 0; h < 2; h++) {                  // the two 16-element halves
                        for (int sa = 0; sa < NSL; sa++) {
                            const uint32_t acc = (kb == kbA && h == 0 && sa == 0) ? 0u : 1u;
                            umma_bf16_n(dbuf + 32u * sa, sw64_desc(stageP(s, sa)) + 2 * h,
                                        sw64_desc(stageQ(s, 0)) + 2 * h, BN * (LV - sa), acc);
                        }
                    }
                    umma_commit(empty_bar(s));
                }
                umma_commit(accf_bar(buf));  // this chunk's level sums are complete with its MMAs
            }
            if (!ok) {
                set_status(prm.status, PFSM_ERR_TIMEOUT);
                *abort_flag = 1;
            }
            umma_commit(done_bar);          // tracks every MMA issued before TMEM is released
            mbar_wait(done_bar, 0);
        }
        __syncwarp();
    } else {
        const int gq = warp & 3;
        const int r = row0 + 32 * gq + lane;
        // float-float (hi + lo, ~48 bits) with Knuth's TwoSum: each level sum is an exact FP32
        // integer and its scale an exact power of two, so a level costs a few FP32 operations
        float hi[BN], lo[BN];
#pragma unroll
        for (int j = 0; j < BN; j++) { hi[j] = 0.0f; lo[j] = 0.0f; }
        bool ok = true;
        for (int ch = 0; ch < nch; ch++) {
            const int buf = ch & 1;
            bool got = mbar_wait(accf_bar(buf), (ch >> 1) & 1);
            got = __all_sync(0xffffffffu, got) && !*abort_flag;
            if (!got) {
                ok = false;
                set_status(prm.status, PFSM_ERR_TIMEOUT);
                *abort_flag = 1;
                break;
            }
            fence_after();
            for (int L = 0; L < LV; L++) {
                const float scale = __int_as_float((127 - 12 - BETA * L) << 23);   // 2^-(12 + 7 L)
                uint32_t v[32];
                tmem_ld32(tmem_acc + ((uint32_t)(32 * gq) << 16) + BUF_COLS * buf + 32u * L, v);
#pragma unroll
                for (int j = 0; j < 32; j++) {
                    const float x = __uint_as_float(v[j]) * scale;
                    const float sum = hi[j] + x, bp = sum - hi[j];
                    lo[j] += (hi[j] - (sum - bp)) + (x - bp);
                    hi[j] = sum;
                }
            }
            fence_before();
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(acce_bar(buf)) : "memory");
        }
        // every MMA has completed (last chunk waited) and every stage consumed: the stage
        // memory now holds this warp's staging block (32 rows x 32 columns), so that the loads and
        // stores of C (and of the exact diagonal term) are row-contiguous
        double(*eb)[BN + 1] = reinterpret_cast<double(*)[BN + 1]>(gbase) + 32 * gq;
        const int R0 = row0 + 32 * gq;
        const int er = (ok && r < rows_lim) ? prm.ep[zr + r] : 0;
#pragma unroll
        for (int j = 0; j < BN; j++) eb[lane][j] = oz_f2d_scaled(hi[j], er + ecol[j]) + oz_f2d_scaled(lo[j], er + ecol[j]);
        __syncwarp();
        if (ok) {
            // every global load of the lane's 32 rows (C for a subtracting product, V for the
            // diagonal term) issued before the first store, so they are in flight together instead
            // of one dependent round trip per row
            const int c = col0 + lane;
            const bool cok = c < cols_lim;
            const int64_t zvo = (int64_t)z * prm.zv, zdo = (int64_t)z * prm.zd;
            const int64_t vcs = prm.vcs ? prm.vcs : 1;
            const bool dterm = prm.dcol || prm.drow;
            const double dc = (prm.dcol && cok) ? prm.dcol[zdo + c] : 0.0;
            double cv[32], dv[32];
#pragma unroll
            for (int rr = 0; rr < 32; rr++) {
                const int gr = R0 + rr;
                const bool v = gr < rows_lim && cok && !(prm.lower_only && c > gr);
                cv[rr] = (v && prm.sub) ? Cz[(int64_t)gr * prm.ldc + c] : 0.0;
                dv[rr] = (v && dterm) ? prm.Vp[zvo + (int64_t)gr * prm.ldv + c * vcs] : 0.0;
            }
#pragma unroll
            for (int rr = 0; rr < 32; rr++) {
                const int gr = R0 + rr;
                if (gr < rows_lim && cok && !(prm.lower_only && c > gr)) {
                    double res = eb[rr][lane];
                    if (prm.win_plan) {
                        // zero inside the window of the slice owning row gr (largest b, k0[b] <= gr)
                        int lo = 0, hi = prm.win_nb - 1;
                        while (lo < hi) {
                            const int mid = (lo + hi + 1) >> 1;
                            if (prm.win_plan[mid] <= gr) lo = mid; else hi = mid - 1;
                        }
                        const int ws = prm.win_plan[2 * prm.win_nb + lo];
                        if (c >= ws && c < ws + prm.win_plan[3 * prm.win_nb + lo]) res = 0.0;
                    }
                    if (prm.dcol) res = fma(dv[rr], dc, res);
                    if (prm.drow) res = fma(dv[rr], prm.drow[zdo + gr], res);
                    const int64_t o = (int64_t)gr * prm.ldc + c;
                    Cz[o] = prm.sub ? cv[rr] - res : res;
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

// ---- small-K products over column strips --------------------------------------------------------
// The same digit product for K <= 64 (the rank-64 trailing updates of the two-stage reduction and
// its panel back-transformation), where k_gemm_oz's per-tile costs dominate: every 128 x 32 tile
// would reload 112 KB of P digits for 28 KB of Q digits and allocate its own tensor memory. Here a
// CTA keeps its 128-row tile of P digits (all K blocks) in shared memory and walks a strip of up to
// `strip` column tiles: Q digits through a two-stage ring, the level sums of tile t in TMEM buffer
// t & 1 (levels at columns 32 L), so the drain and the C update of a tile overlap the MMAs of the
// next. K <= 64 < one exact 512-term chunk, so every tile is one exact level sum. Warp roles as in
// k_gemm_oz (0: TMA, 1: TMEM owner and MMA issuer), sixteen drain warps (2-17); every wait bounded.
namespace ozs {
constexpr int MAXKB = 2;                                  // K <= 64
constexpr int QST = 2;                                    // Q ring stages
constexpr int P_BYTES = MAXKB * OZ_SLICES * oz::P_TILE;   // 112 KB
constexpr int QSTAGE = MAXKB * OZ_SLICES * oz::Q_TILE;    // 28 KB
constexpr int EPI_WARPS = 16;                            // drain warps: 4 per TMEM lane quarter
constexpr int CW = oz::BN * 4 / EPI_WARPS;                // columns per drain warp (8)
constexpr int THREADS = 64 + 32 * EPI_WARPS;
constexpr int EB_BYTES = EPI_WARPS * 32 * (CW + 1) * 8;  // per-warp 32 x CW staging block
static_assert(CW == 8, "the drain loads one 8-column TMEM group per level");
}  // namespace ozs

__global__ void __launch_bounds__(ozs::THREADS, 1)
k_gemm_oz_strip(const __grid_constant__ CUtensorMap mapP, const __grid_constant__ CUtensorMap mapQ, OzParams prm,
                int strip)
{
    using namespace tc;
    using namespace oz;
    const int z = blockIdx.z;
    const int row0 = prm.row_base + blockIdx.y * BM;
    const int cbase = (prm.cols_from_zero ? 0 : prm.row_base) + prm.col_off;
    const int rows_lim = prm.ext ? prm.ext[z] : prm.rows;
    const int cols_lim = prm.ext_c ? prm.ext_c[z] : (prm.ext ? prm.ext[z] : prm.rows);
    const int ct0 = blockIdx.x * strip;
    if (row0 >= rows_lim) return;
    // column tiles of this strip inside the window
    int nt = 0;
    while (nt < strip && cbase + (ct0 + nt) * BN < cols_lim) nt++;
    if (nt == 0) return;
    const int64_t zr = (int64_t)z * prm.zrow;
    const int64_t zq = (int64_t)z * (prm.zrow_q ? prm.zrow_q : prm.zrow);
    double *Cz = prm.C + (int64_t)z * prm.zc;
    const int LV = (prm.levels > 0 && prm.levels < OZ_LEVELS) ? prm.levels : OZ_LEVELS;
    const int NSL = LV;
    const int nkb = prm.kblocks;                                  // 1 or 2
    extern __shared__ __align__(1024) uint8_t smraw[];
    const uint32_t raw = smem_u32(smraw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    uint8_t *gbase = smraw + (base - raw);
    const uint32_t pbase = base, qbase = base + ozs::P_BYTES;
    double *ebuf = reinterpret_cast<double *>(gbase + ozs::P_BYTES + ozs::QST * ozs::QSTAGE);
    uint64_t *bars = reinterpret_cast<uint64_t *>(gbase + ozs::P_BYTES + ozs::QST * ozs::QSTAGE + ozs::EB_BYTES);
    // bars: pfull, qfull[2], qempty[2], accf[2], acce[2], done
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 10);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
    const uint32_t bb = smem_u32(bars);
    const uint32_t pfull = bb;
    auto qfull = [&](int s) { return bb + 8u * (1 + s); };
    auto qempty = [&](int s) { return bb + 8u * (3 + s); };
    auto accf = [&](int b) { return bb + 8u * (5 + b); };
    auto acce = [&](int b) { return bb + 8u * (7 + b); };
    const uint32_t done_bar = bb + 8u * 9;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        mbar_init(pfull, 1);
        for (int q = 0; q < ozs::QST; q++) {
            mbar_init(qfull(q), 1);
            mbar_init(qempty(q), 1);
        }
        for (int b = 0; b < 2; b++) {
            mbar_init(accf(b), 1);
            mbar_init(acce(b), 32 * ozs::EPI_WARPS);
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
    auto pslice = [&](int kb, int sl) { return pbase + (uint32_t)((kb * NSL + sl) * P_TILE); };
    auto qslice = [&](int st, int kb, int sl) {
        return qbase + (uint32_t)(st * ozs::QSTAGE + (kb * NSL + sl) * Q_TILE);
    };

    if (warp == 0) {
        if (lane == 0) {
            mbar_expect_tx(pfull, nkb * NSL * P_TILE);
            for (int kb = 0; kb < nkb; kb++) tma_load_3d(pslice(kb, 0), &mapP, pfull, kb * KB, (int)(zr + row0), 0);
            int issued = 0;
            for (int t = 0; t < nt; t++) {
                const int st = t % ozs::QST, round = t / ozs::QST;
                if (round > 0 && !mbar_wait(qempty(st), (round - 1) & 1)) {
                    set_status(prm.status, PFSM_ERR_TIMEOUT);
                    *abort_flag = 1;
                    break;
                }
                if (*abort_flag) break;
                const int col0 = cbase + (ct0 + t) * BN;
                mbar_expect_tx(qfull(st), nkb * NSL * Q_TILE);
                for (int kb = 0; kb < nkb; kb++)
                    tma_load_3d(qslice(st, kb, 0), &mapQ, qfull(st), kb * KB, (int)(zq + col0), 0);
                issued = t + 1;
            }
            // every copy this warp issued has landed before the CTA can exit
            mbar_wait(pfull, 0);
            for (int i = (issued > ozs::QST ? issued - ozs::QST : 0); i < issued; i++)
                mbar_wait(qfull(i % ozs::QST), (i / ozs::QST) & 1);
        }
        __syncwarp();
    } else if (warp == 1) {
        if (lane == 0) {
            bool ok = mbar_wait(pfull, 0);
            for (int t = 0; t < nt && ok; t++) {
                const int buf = t & 1, st = t % ozs::QST;
                if (t >= 2 && !mbar_wait(acce(buf), ((t >> 1) - 1) & 1)) { ok = false; break; }
                if (!mbar_wait(qfull(st), (t / ozs::QST) & 1) || *abort_flag) { ok = false; break; }
                fence_after();
                const uint32_t dbuf = tmem_acc + BUF_COLS * buf;
                for (int kb = 0; kb < nkb; kb++)
                    for (int h = 0; h < 2; h++)
                        for (int sa = 0; sa < NSL; sa++) {
                            const uint32_t acc = (kb == 0 && h == 0 && sa == 0) ? 0u : 1u;
                            umma_bf16_n(dbuf + 32u * sa, sw64_desc(pslice(kb, sa)) + 2 * h,
                                        sw64_desc(qslice(st, kb, 0)) + 2 * h, BN * (LV - sa), acc);
                        }
                umma_commit(qempty(st));
                umma_commit(accf(buf));
            }
            if (!ok) {
                set_status(prm.status, PFSM_ERR_TIMEOUT);
                *abort_flag = 1;
            }
            umma_commit(done_bar);
            mbar_wait(done_bar, 0);
        }
        __syncwarp();
    } else {
        // drain warps 2 .. 17: TMEM lane quarter gq = warp & 3 (the quarter a warp may read) and
        // column slice hc (8 of the tile's 32 columns), four warps per SM sub-partition so that
        // some drain while others wait on memory. Each entry's level sums are combined exactly in
        // 64-bit integers and rounded once to FP64; the C update is the only FP64 operation.
        using ozs::CW;
        const int gq = warp & 3, hc = (warp - 2) >> 2;
        const int r = row0 + 32 * gq + lane;
        const int er = (r < rows_lim) ? prm.ep[zr + r] : 0;
        const int escale = -12 - BETA * (LV - 1);                 // scale of T's unit
        double(*eb)[CW + 1] = reinterpret_cast<double(*)[CW + 1]>(ebuf) + 32 * (warp - 2);
        const int R0 = row0 + 32 * gq;
        constexpr int RP = 32 / CW;                               // rows per C instruction (4)
        const int rsub = lane / CW, cl = lane % CW;               // C update: rows RP q + rsub, column cl
        for (int t = 0; t < nt; t++) {
            const int buf = t & 1;
            const int c = cbase + (ct0 + t) * BN + CW * hc + cl;
            const bool cok = c < cols_lim;
            const int ec = cok ? prm.eq[zq + c] : 0;
            // this warp alone updates its 32 x CW block of C: its loads go out before the wait for
            // the tile's MMAs, so their latency overlaps it
            double cv[32 / RP];
#pragma unroll
            for (int q = 0; q < 32 / RP; q++) {
                const int gr = R0 + RP * q + rsub;
                cv[q] = (prm.sub && gr < rows_lim && cok) ? Cz[(int64_t)gr * prm.ldc + c] : 0.0;
            }
            bool got = mbar_wait(accf(buf), (t >> 1) & 1);
            got = __all_sync(0xffffffffu, got) && !*abort_flag;
            if (!got) {
                set_status(prm.status, PFSM_ERR_TIMEOUT);
                *abort_flag = 1;
                break;
            }
            fence_after();
            const uint32_t ta = tmem_acc + ((uint32_t)(32 * gq) << 16) + BUF_COLS * buf + (uint32_t)(CW * hc);
            uint32_t v[OZ_LEVELS][8];
#pragma unroll
            for (int L = 0; L < OZ_LEVELS; L++)
                if (L < LV) tmem_ld8_nowait(ta + 32u * L, v[L]);
            tmem_wait_ld();
#pragma unroll
            for (int L = 0; L < OZ_LEVELS; L++)
                if (L < LV) tmem_regs_after_wait(v[L]);
            fence_before();                                       // every TMEM read of the tile done
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(acce(buf)) : "memory");
#pragma unroll
            for (int j = 0; j < CW; j++) {
                const int es = er + __shfl_sync(0xffffffffu, ec, j) + escale;
                eb[lane][j] = oz_i64_to_f64_scaled(oz_levels_i64(v, j, LV), es);
            }
            __syncwarp();
#pragma unroll
            for (int q = 0; q < 32 / RP; q++) {
                const int gr = R0 + RP * q + rsub;
                const double res = eb[RP * q + rsub][cl];
                if (gr < rows_lim && cok) Cz[(int64_t)gr * prm.ldc + c] = prm.sub ? cv[q] - res : res;
            }
            __syncwarp();
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
size_t oz_smem_bytes() { return (size_t)oz::STAGES * oz::MAX_STAGE_BYTES + 1024 + 512; }
}

size_t oz_strip_smem_bytes() { return (size_t)ozs::P_BYTES + ozs::QST * ozs::QSTAGE + ozs::EB_BYTES + 1024 + 256; }

cudaError_t configure_oz_kernels()
{
    cudaError_t e = cudaFuncSetAttribute(k_gemm_oz, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)oz_smem_bytes());
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_gemm_oz_strip, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)oz_strip_smem_bytes());
}

cudaError_t launch_oz_split(const double *src, int64_t rows, int64_t cols, int64_t ld, const SliceBuf &dst,
                            int32_t *exps, cudaStream_t st, bool zero_diag, double *d)
{
    const unsigned blocks = (unsigned)((rows + 1) / 2);   // two rows per CTA: small CTAs balance the SMs
    k_oz_split<double><<<blocks, 64, 0, st>>>(src, rows, cols, ld, reinterpret_cast<__nv_bfloat16 *>(dst.ptr),
                                               dst.ld, dst.ld * dst.rows, exps, zero_diag ? 1 : 0, d);
    g_launches++;
    return cudaGetLastError();
}

cudaError_t launch_oz_split_win(const double *src, int64_t src_z, int64_t ld, int64_t row0, int64_t col0,
                                const int32_t *ext, int ext_off, int rows_fixed, const int32_t *rext, int max_rows,
                                int nb, const SliceBuf &dst, int64_t dst_zrow, int64_t dst_row0, int32_t *exps,
                                cudaStream_t st, double *diag_out)
{
    if (max_rows <= 0) return cudaSuccess;
    dim3 grid((unsigned)((max_rows + 1) / 2), (unsigned)nb);
    k_oz_split_win<<<grid, 64, 0, st>>>(src, src_z, ld, row0, col0, ext, ext_off, rows_fixed, rext,
                                        diag_out ? 1 : 0, diag_out, dst.ld,
                                        reinterpret_cast<__nv_bfloat16 *>(dst.ptr), dst_zrow, dst_row0, dst.ld,
                                        dst.ld * dst.rows, exps);
    g_launches++;
    return cudaGetLastError();
}

cudaError_t launch_oz_split_f32(const float *src, int64_t rows, int64_t cols, int64_t ld, const SliceBuf &dst,
                                int32_t *exps, cudaStream_t st)
{
    const unsigned blocks = (unsigned)((rows + 1) / 2);
    k_oz_split<float><<<blocks, 64, 0, st>>>(src, rows, cols, ld, reinterpret_cast<__nv_bfloat16 *>(dst.ptr),
                                              dst.ld, dst.ld * dst.rows, exps, 0, nullptr);
    g_launches++;
    return cudaGetLastError();
}

cudaError_t launch_gemm_oz(const SliceBuf &P, const int32_t *ep, const SliceBuf &Q, const int32_t *eq,
                           OzParams prm, cudaStream_t st, int batch)
{
    CUtensorMap mp, mq;
    cudaError_t e;
    const int nsl = (prm.levels > 0 && prm.levels < OZ_LEVELS) ? prm.levels : OZ_LEVELS;
    if (P.ns != OZ_SLICES || Q.ns != OZ_SLICES || P.kind != 0 || Q.kind != 0 || P.ld != Q.ld || P.ld % oz::KB)
        return cudaErrorInvalidValue;
    if ((e = make_slice_map64(&mp, P, oz::BM, nsl)) != cudaSuccess) return e;
    if ((e = make_slice_map64(&mq, Q, oz::BN, nsl)) != cudaSuccess) return e;
    prm.kblocks = (int)(P.ld / oz::KB);
    prm.ep = ep;
    prm.eq = eq;
    // batched: prm.rows / prm.cols give the grid extent from row_base (the largest window)
    const int ext_r = prm.rows - prm.row_base;
    const int ext_c = prm.cols - (prm.cols_from_zero ? 0 : prm.row_base) - prm.col_off;
    if (ext_r <= 0 || ext_c <= 0) return cudaSuccess;
    dim3 grid((unsigned)((ext_c + oz::BN - 1) / oz::BN), (unsigned)((ext_r + oz::BM - 1) / oz::BM), (unsigned)batch);
    k_gemm_oz<<<grid, 192, oz_smem_bytes(), st>>>(mp, mq, prm);
    g_launches++;
    return cudaGetLastError();
}

cudaError_t launch_gemm_oz_strip(const SliceBuf &P, const int32_t *ep, const SliceBuf &Q, const int32_t *eq,
                                 OzParams prm, cudaStream_t st, int batch, int strip)
{
    CUtensorMap mp, mq;
    cudaError_t e;
    const int nsl = (prm.levels > 0 && prm.levels < OZ_LEVELS) ? prm.levels : OZ_LEVELS;
    if (P.ns != OZ_SLICES || Q.ns != OZ_SLICES || P.kind != 0 || Q.kind != 0 || P.ld != Q.ld || P.ld % oz::KB ||
        P.ld > ozs::MAXKB * oz::KB || prm.lower_only || prm.p_lower || prm.dcol || prm.drow || prm.win_plan ||
        prm.krange64 || strip < 1)
        return cudaErrorInvalidValue;
    if ((e = make_slice_map64(&mp, P, oz::BM, nsl)) != cudaSuccess) return e;
    if ((e = make_slice_map64(&mq, Q, oz::BN, nsl)) != cudaSuccess) return e;
    prm.kblocks = (int)(P.ld / oz::KB);
    prm.ep = ep;
    prm.eq = eq;
    const int ext_r = prm.rows - prm.row_base;
    const int ext_c = prm.cols - (prm.cols_from_zero ? 0 : prm.row_base) - prm.col_off;
    if (ext_r <= 0 || ext_c <= 0) return cudaSuccess;
    const int nct = (ext_c + oz::BN - 1) / oz::BN;
    dim3 grid((unsigned)((nct + strip - 1) / strip), (unsigned)((ext_r + oz::BM - 1) / oz::BM), (unsigned)batch);
    k_gemm_oz_strip<<<grid, ozs::THREADS, oz_strip_smem_bytes(), st>>>(mp, mq, prm, strip);
    g_launches++;
    return cudaGetLastError();
}

}  // namespace pfsm
