// atan and atanh of a ratio N / D for the FP32 SIE deflection (Sec. 2.1,
// Eqs. 2-3: alpha_x carries atan(e x' / (psi + s)), alpha_y carries
// atanh(e y' / (psi + q^2 s))).  Both take the numerator and the positive
// denominator separately, so the quotient that forms the argument is also
// the one the argument reduction needs.  The polynomial cores are minimax
// fits (lensed_minimax.cuh, written by gen_minimax.py); MUFU supplies the
// reciprocal and, for atanh beyond 1/2, the base-2 logarithm.
#pragma once

#include "lensed_minimax.cuh"

namespace lensed {

__device__ __forceinline__ float trig_rcp(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float trig_lg2(float x)
{
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// pi / 2 and ln(2) / 2 as float pairs (value + residual)
constexpr float kHalfPiHi = 1.57079637e+00f, kHalfPiLo = -4.37113901e-08f;
constexpr float kHalfLn2Hi = 3.46573591e-01f, kHalfLn2Lo = -9.52327162e-10f;

// atan(n / d) for d >= 0 (0 when n = d = 0).  t = min(|n|, d) / max(|n|, d)
// lies in [0, 1]; atan(t) = t + t^3 Q(t^2), and pi/2 - atan(t) when |n| > d
// (the subtraction from the leading float of pi/2 is exact there, since
// atan(t) <= pi/4).  Odd in n.
__device__ __forceinline__ float atan_ratio(float n, float d)
{
    const float an = fabsf(n);
    const float hi = fmaxf(an, d), lo = fminf(an, d);
    const float t = hi > 0.f ? lo * trig_rcp(hi) : 0.f;
    const float u = t * t;
    float r = fmaf(t * u, minimax_atan_q(u), t);
    if (an > d) r = (kHalfPiHi - r) + kHalfPiLo;
    return copysignf(r, n);
}

// atanh(n / d) for |n| < d (0 when d = 0).  z = n / d; for |z| <= 1/2,
// atanh(z) = z + z^3 Q(z^2); beyond, (1/2) ln((d + n) / (d - n)), whose
// value (> 0.549 in magnitude) keeps the logarithm's absolute error small
// against it.  Odd in n.
__device__ __forceinline__ float atanh_ratio(float n, float d)
{
    const float z = d > 0.f ? n * trig_rcp(d) : 0.f;
    const float u = z * z;
    if (u <= 0.25f) {
        return fmaf(z * u, minimax_atanh_q(u), z);
    }
    const float L = trig_lg2((d + n) * trig_rcp(d - n));
    return fmaf(kHalfLn2Hi, L, kHalfLn2Lo * L);
}

}  // namespace lensed
