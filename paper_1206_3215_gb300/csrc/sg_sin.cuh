// sin u for the sine-Gordon passes (Eq. 3).
//
// FP32: Cody-Waite reduction modulo pi/2 and Taylor polynomials on
// [-pi/4, pi/4].  pi/2 = C1 + C2 + C3 (three floats, 72 bits together, from
// the double-double value of pi/2 below) is subtracted with fused
// multiply-adds, so the reduced argument is accurate to a few ulp while
// |k| < 2^20 (|u| < 1.6e6).  The omitted Taylor terms r^11/11! and r^12/12!
// are below 2e-9 on the interval.  A non-finite u gives NaN (no loop and no
// library slow path in the pass's code).  FP64 calls the math library.
#pragma once
#include <cuda_runtime.h>

namespace pss {

namespace sgsin {
constexpr double HI = 1.5707963267948966, LO = 6.123233995736766e-17;  // pi/2 = HI + LO
constexpr float C1 = float(HI);
constexpr float C2 = float(HI - double(C1));
constexpr float C3 = float((HI - double(C1) - double(C2)) + LO);
}  // namespace sgsin

#ifndef PSS_SG_LIBM_SIN
#define PSS_SG_LIBM_SIN 0
#endif

__device__ __forceinline__ float sg_sin(float x)
{
    if constexpr (PSS_SG_LIBM_SIN) return sinf(x);
    const float k = rintf(x * float(2.0 / 3.14159265358979323846));
    float r = __fmaf_rn(-k, sgsin::C1, x);
    r = __fmaf_rn(-k, sgsin::C2, r);
    r = __fmaf_rn(-k, sgsin::C3, r);
    const float r2 = r * r;
    const float sn = __fmaf_rn(r * r2, -1.0f / 6 + r2 * (1.0f / 120 + r2 * (-1.0f / 5040 + r2 * (1.0f / 362880))), r);
    const float cs = 1.0f + r2 * (-0.5f + r2 * (1.0f / 24 + r2 * (-1.0f / 720 + r2 * (1.0f / 40320 + r2 * (-1.0f / 3628800)))));
    const int q = int(k) & 3;
    const float v = (q & 1) ? cs : sn;
    return (q & 2) ? -v : v;
}
__device__ __forceinline__ double sg_sin(double x) { return sin(x); }

}  // namespace pss
