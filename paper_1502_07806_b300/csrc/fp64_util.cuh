// FP64 helpers shared by the window eigensolve kernels (B300 issues one FP64 warp instruction
// per 16 cycles per SM and a dependent one every ~64 cycles, so the IEEE divide and square-root
// sequences, about ten dependent FP64 instructions each, are avoided on serial paths).
#pragma once

#include <cuda_runtime.h>

namespace pfsm {

// 1/p and 1/sqrt(d) for d, p > 0 of any FP64 magnitude without the IEEE FP64 divide / square
// root sequences (each ~10 dependent FP64 instructions of ~64 cycles on B300): the exponent is
// split off (so the FP32 seed never under- or overflows), then an FP32 estimate and two Newton
// steps, y <- y (2 - p y) and y <- y (3 - d y^2) / 2, give about 1 ulp.
__device__ __forceinline__ double scaled_rcp(double p)
{
    int e;
    const double m = frexp(p, &e);                     // p = m 2^e, m in [0.5, 1)
    double y = (double)__frcp_rn((float)m);
    y = y * fma(-m, y, 2.0);
    y = y * fma(-m, y, 2.0);
    return ldexp(y, -e);
}

__device__ __forceinline__ double scaled_rsqrt(double d)
{
    int e;
    double m = frexp(d, &e);
    if (e & 1) { m *= 2.0; e -= 1; }                  // d = m 2^e, e even, m in [0.5, 2)
    double y = (double)rsqrtf((float)m);
    y = y * fma(-0.5 * m, y * y, 1.5);
    y = y * fma(-0.5 * m, y * y, 1.5);
    return ldexp(y, -e / 2);
}

// Reciprocal without an IEEE FP64 division (~640 cycles dependent on B300) and without F2F
// conversions (they run on the FP64 pipe): the FP32 approximate reciprocal of p's leading 24 bits,
// both conversions done by integer operations on the bit patterns, then two Newton steps
// y <- y (2 - p y) (relative error 2^-22 -> 2^-44 -> rounding), about 1 ulp. |p| outside
// [2^-125, 2^126) takes the FP64 division.
__device__ __forceinline__ double fast_rcp(double p)
{
    const int hi = __double2hiint(p);
    const unsigned lo = (unsigned)__double2loint(p);
    const int ev = (hi >> 20) & 0x7FF;
    if ((unsigned)(ev - 898) > 250u) return 1.0 / p;
    const float pf = __uint_as_float(((unsigned)hi & 0x80000000u) | ((unsigned)(ev - 896) << 23) |
                                     ((unsigned)(hi & 0xFFFFF) << 3) | (lo >> 29));
    float rf;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(rf) : "f"(pf));
    const unsigned rb = __float_as_uint(rf);
    double y = __hiloint2double((int)((rb & 0x80000000u) | ((((rb >> 23) & 0xFFu) + 896u) << 20) |
                                      ((rb & 0x7FFFFFu) >> 3)),
                                (int)(rb << 29));
    y = y * fma(-p, y, 2.0);
    y = y * fma(-p, y, 2.0);
    return y;
}

// 1/sqrt(d) for d > 0 without F2F conversions or exponent splitting (both take FP64-pipe
// instructions): the FP32 approximate inverse square root of d's leading 24 bits, conversions from
// and to FP64 by integer operations on the bit patterns, then two Newton steps y <- y (3/2 - d y^2 / 2)
// (relative error 2^-22 -> 2^-43 -> rounding). d outside [2^-125, 2^124) takes scaled_rsqrt.
__device__ __forceinline__ double fast_rsqrt(double d)
{
    const int hi = __double2hiint(d);
    const unsigned lo = (unsigned)__double2loint(d);
    const int ev = (hi >> 20) & 0x7FF;
    if ((unsigned)(ev - 898) > 248u || hi < 0) return scaled_rsqrt(d);
    const float df = __uint_as_float(((unsigned)(ev - 896) << 23) | ((unsigned)(hi & 0xFFFFF) << 3) | (lo >> 29));
    float rf;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(rf) : "f"(df));
    const unsigned rb = __float_as_uint(rf);
    double y = __hiloint2double((int)(((((rb >> 23) & 0xFFu) + 896u) << 20) | ((rb & 0x7FFFFFu) >> 3)), (int)(rb << 29));
    const double hd = 0.5 * d;
    y = y * fma(-hd, y * y, 1.5);
    y = y * fma(-hd, y * y, 1.5);
    return y;
}

// t 2^e rounded to FP64 (to nearest, ties to even) by integer operations: the FP64 pipe, which
// the C update needs, is 1/64 of the integer rate.
__device__ __forceinline__ double oz_i64_to_f64_scaled(long long t, int e)
{
    if (t == 0) return 0.0;
    const unsigned long long sgn = (unsigned long long)t & 0x8000000000000000ull;
    unsigned long long m = sgn ? 0ull - (unsigned long long)t : (unsigned long long)t;
    const int lz = __clzll((long long)m);
    m <<= lz;                                                     // leading one at bit 63
    const unsigned long long rr = m + (0x3FFull + ((m >> 11) & 1ull));
    const int carry = rr < m ? 1 : 0;                             // rounded up to 2^64
    const int ex = 1023 + 63 - lz + e + carry;
    if (ex <= 0 || ex >= 2047) {                                  // subnormal or overflowing result:
        double x = (double)t;                                     // exact powers of two, no call
        for (int k = 0; k < 3; k++) {
            const int ek = max(-1022, min(1023, e));
            x *= __longlong_as_double((long long)(ek + 1023) << 52);
            e -= ek;
        }
        return x;
    }
    const unsigned long long mant = carry ? 0ull : ((rr >> 11) & 0xFFFFFFFFFFFFFull);
    return __longlong_as_double((long long)(sgn | ((unsigned long long)ex << 52) | mant));
}

}  // namespace pfsm
