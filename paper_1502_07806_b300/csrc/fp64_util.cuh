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

}  // namespace pfsm
