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

// atan(n / d) for d >= 0 (0 when n = d = 0), for one ray (V = float) or a
// pair (V = float2).  t = min(|n|, d) / max(|n|, d) lies in [0, 1];
// atan(t) = t + t^3 Q(t^2), and pi/2 - atan(t) when |n| > d (the subtraction
// from the leading float of pi/2 is exact there, since atan(t) <= pi/4).
// Odd in n.
template <class V>
__device__ __forceinline__ V atan_ratio(V n, V d)
{
    const V lo = vmap(n, d, [](float a, float b) { return fminf(fabsf(a), b); });
    const V rh = vmap(n, d, [](float a, float b) {
        const float hi = fmaxf(fabsf(a), b);
        return hi > 0.f ? trig_rcp(hi) : 0.f;
    });
    const V t = vmul(lo, rh);
    const V u = vmul(t, t);
    const V r = vfma(vmul(t, u), minimax_atan_q(u), t);
    const V rc = vadd(vsub(vsplat<V>(kHalfPiHi), r), vsplat<V>(kHalfPiLo));
    return vmap(n, d, r, rc, [](float a, float b, float r0, float r1) {
        return copysignf(fabsf(a) > b ? r1 : r0, a);
    });
}

// atanh(n / d) for |n| < d (0 when d = 0), for one ray or a pair.  z = n / d;
// for |z| <= 1/2, atanh(z) = z + z^3 Q(z^2); beyond, (1/2) ln((d + n) / (d - n)),
// whose value (> 0.549 in magnitude) keeps the logarithm's absolute error
// small against it.  Each lane takes its own form; a pair computes a form
// only if one of its lanes needs it.  Odd in n.
__device__ __forceinline__ bool all_le(float u, float c) { return u <= c; }
__device__ __forceinline__ bool all_le(float2 u, float c) { return u.x <= c && u.y <= c; }
__device__ __forceinline__ bool all_gt(float u, float c) { return u > c; }
__device__ __forceinline__ bool all_gt(float2 u, float c) { return u.x > c && u.y > c; }
template <class V>
__device__ __forceinline__ V atanh_ratio(V n, V d)
{
    const V rd = vmap(d, [](float b) { return b > 0.f ? trig_rcp(b) : 0.f; });
    const V z = vmul(n, rd);
    const V u = vmul(z, z);
    const bool near_all = all_le(u, 0.25f), far_all = !near_all && all_gt(u, 0.25f);
    V P = z, Lg = z;
    if (!far_all) P = vfma(vmul(z, u), minimax_atanh_q(u), z);
    if (!near_all) {
        const V q = vmul(vadd(d, n), vmap(vsub(d, n), [](float b) { return trig_rcp(b); }));
        const V L = vmap(q, [](float a) { return trig_lg2(a); });
        Lg = vfma(vsplat<V>(kHalfLn2Hi), L, vmul(vsplat<V>(kHalfLn2Lo), L));
    }
    if (near_all) return P;
    if (far_all) return Lg;
    return vmap(u, P, Lg, u, [](float uu, float p, float l, float) { return uu <= 0.25f ? p : l; });
}

}  // namespace lensed
