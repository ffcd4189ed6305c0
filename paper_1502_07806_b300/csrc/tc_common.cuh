// tcgen05 / TMA / mbarrier helpers shared by the tensor-core kernels (inline PTX, sm_103a).
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>

#include "pfsm_internal.cuh"

namespace pfsm {

namespace tc {

constexpr uint64_t kWaitNs = 2000000000ull;          // 2 s per wait before giving up

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t globaltimer()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait for the phase of parity `parity` to complete.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity)
{
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = globaltimer();
    while (!mbar_try_wait(bar, parity))
        if (globaltimer() - t0 > kWaitNs) return false;
    return true;
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap *map, uint32_t bar, int x, int y, int z)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
        ::"r"(dst), "l"((uint64_t)map), "r"(x), "r"(y), "r"(z), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor of a K-major operand tile with 128-byte swizzle: 8-row groups
// 1024 B apart (stride byte offset), descriptor version 1.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;                 // leading byte offset (unused for this layout)
    d |= (uint64_t)(1024 >> 4) << 32;       // stride byte offset
    d |= (uint64_t)1 << 46;                 // version
    d |= (uint64_t)2 << 61;                 // SWIZZLE_128B
    return d;
}

// The same for 64-byte K rows with 64-byte swizzle (layout type 4): 8-row groups 512 B apart.
__device__ __forceinline__ uint64_t sw64_desc(uint32_t saddr)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;                 // leading byte offset (unused for this layout)
    d |= (uint64_t)(512 >> 4) << 32;        // stride byte offset
    d |= (uint64_t)1 << 46;                 // version
    d |= (uint64_t)4 << 61;                 // SWIZZLE_64B
    return d;
}

// Instruction descriptor: FP32 accumulator, A/B element format (BF16 = 1, TF32 = 2), both
// operands K-major, N (bits 17-22 hold N/8), M (bits 24-28 hold M/16).
template <int KIND, int M_, int N_>
__host__ __device__ constexpr uint32_t idesc()
{
    return (1u << 4) | ((KIND == 0 ? 1u : 2u) << 7) | ((KIND == 0 ? 1u : 2u) << 10) |
           ((uint32_t)(N_ >> 3) << 17) | ((uint32_t)(M_ >> 4) << 24);
}

template <int KIND, int M_ = 128, int N_ = 128>
__device__ __forceinline__ void umma(uint32_t dtmem, uint64_t a, uint64_t b, uint32_t accum)
{
    if (KIND == 0)
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
            ::"r"(dtmem), "l"(a), "l"(b), "r"(idesc<0, M_, N_>()), "r"(accum));
    else
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}"
            ::"r"(dtmem), "l"(a), "l"(b), "r"(idesc<1, M_, N_>()), "r"(accum));
}

// kind::f16 MMA (BF16 operands) with M = 128 and N given at run time (a multiple of 16 in
// [16, 256]): N / 8 goes into bits 17-22 of the instruction descriptor.
__device__ __forceinline__ void umma_bf16_n(uint32_t dtmem, uint64_t a, uint64_t b, int n, uint32_t accum)
{
    const uint32_t id = idesc<0, 128, 0>() | ((uint32_t)(n >> 3) << 17);
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
        ::"r"(dtmem), "l"(a), "l"(b), "r"(id), "r"(accum));
}

__device__ __forceinline__ void umma_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// 8 consecutive TMEM columns of the warp's 32 lanes; the caller waits (tmem_wait_ld) before use,
// so several loads can be in flight together
__device__ __forceinline__ void tmem_ld8_nowait(uint32_t taddr, uint32_t (&r)[8])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// After tmem_wait_ld: ties the loaded registers to a point behind the wait, so that no use of them
// can be scheduled between the load and the wait
__device__ __forceinline__ void tmem_regs_after_wait(uint32_t (&r)[8])
{
    asm volatile(""
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]));
}

__device__ __forceinline__ float to_tf32(float x)
{
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

// FP64 bit pattern u rounded to 53 - DROP significant bits by integer operations: ties to even
// (RNA false) or away from zero (RNA true). A carry out of the significand moves into the
// exponent, which is the correctly rounded result; +-0 stay +-0.
template <int DROP, bool RNA>
__device__ __forceinline__ unsigned long long round_sig(unsigned long long u)
{
    const unsigned long long half = RNA ? (1ull << (DROP - 1)) : ((1ull << (DROP - 1)) - 1ull + ((u >> DROP) & 1ull));
    return (u + half) & ~((1ull << DROP) - 1ull);
}

// The slices of v by the conversion instructions (FP64 pipe), for values whose slices leave the
// normal FP32 exponent range. Not inlined, so that the compiler cannot predicate it into the
// common path.
template <int KIND>
__device__ __noinline__ void store_slices_exact(void *base, int64_t sstride, int64_t o, int ns, double v)
{
    double rem = v;
    for (int s = 0; s < ns; s++) {
        if (KIND == 0) {
            const __nv_bfloat16 b = __double2bfloat16(rem);
            reinterpret_cast<__nv_bfloat16 *>(base)[s * sstride + o] = b;
            rem -= (double)__bfloat162float(b);
        } else {
            const float t = to_tf32((float)rem);
            reinterpret_cast<float *>(base)[s * sstride + o] = t;
            rem -= (double)t;
        }
    }
}

// Writes the `ns` KIND slices of v at slice-matrix element offset `o`: slice s is the BF16 (KIND 0)
// or TF32 (KIND 1, via FP32) rounding of v minus the slices before it. B300 retires one FP64 warp
// instruction per 16 cycles per SM, and the conversions to and from FP64 run on that pipe, so
// the roundings are done on the FP64 bit pattern with integer operations (the same round-to-
// nearest-even, and for TF32 the FP32 rounding followed by ties-away, as the conversion
// instructions) and only the exact residual v - slice is an FP64 instruction. An element with a
// slice outside the normal FP32 exponent range takes store_slices_exact instead.
template <int KIND>
__device__ __forceinline__ void store_slices(void *base, int64_t sstride, int64_t o, int ns, double v)
{
    constexpr int MAXS = 3;
    uint32_t bits[MAXS] = {0u, 0u, 0u};
    bool ok = true;
    double rem = v;
#pragma unroll
    for (int s = 0; s < MAXS; s++) {
        if (s < ns) {
            const unsigned long long u = (unsigned long long)__double_as_longlong(rem);
            const int ex = (int)((u >> 52) & 0x7FF);
            ok = ok && ((ex >= 897 && ex <= 1149) || (u << 1) == 0ull);   // 2^-126 <= |rem| < 2^127, or 0
            const unsigned long long r = (KIND == 0) ? round_sig<45, false>(u)           // 8 bits
                                                     : round_sig<42, true>(round_sig<29, false>(u));   // FP32, 11 bits
            const unsigned int re = (unsigned int)((r >> 52) & 0x7FF);
            if (KIND == 0) {
                const unsigned int sg = (unsigned int)(r >> 48) & 0x8000u;
                bits[s] = re ? (sg | ((re - 896u) << 7) | (unsigned int)((r >> 45) & 0x7F)) : sg;
            } else {
                const unsigned int sg = (unsigned int)(r >> 32) & 0x80000000u;
                bits[s] = re ? (sg | ((re - 896u) << 23) | (unsigned int)((r >> 29) & 0x7FFFFF)) : sg;
            }
            if (s + 1 < ns) rem -= __longlong_as_double((long long)r);
        }
    }
    if (!ok) {
        store_slices_exact<KIND>(base, sstride, o, ns, v);
        return;
    }
#pragma unroll
    for (int s = 0; s < MAXS; s++) {
        if (s < ns) {
            if (KIND == 0) reinterpret_cast<unsigned short *>(base)[s * sstride + o] = (unsigned short)bits[s];
            else reinterpret_cast<uint32_t *>(base)[s * sstride + o] = bits[s];
        }
    }
}

// Writes the slices of an FP32 value (all arithmetic in FP32: the pieces of a 24-bit significand).
template <int KIND>
__device__ __forceinline__ void store_slices_f32(void *base, int64_t sstride, int64_t o, int ns, float v)
{
    float rem = v;
    for (int s = 0; s < ns; s++) {
        if (KIND == 0) {
            const __nv_bfloat16 b = __float2bfloat16_rn(rem);
            reinterpret_cast<__nv_bfloat16 *>(base)[s * sstride + o] = b;
            rem -= __bfloat162float(b);
        } else {
            const float t = to_tf32(rem);
            reinterpret_cast<float *>(base)[s * sstride + o] = t;
            rem -= t;
        }
    }
}

}  // namespace tc

// 3-D TMA map over row-major slices: {ld (K), rows, ns}, box {128 bytes of K, box_rows, 1}.
cudaError_t make_slice_map(CUtensorMap *map, const SliceBuf &b, int box_rows);
// The same with 64-byte K rows, 64-byte swizzle and `box_slices` slices per copy.
cudaError_t make_slice_map64(CUtensorMap *map, const SliceBuf &b, int box_rows, int box_slices);

}  // namespace pfsm
