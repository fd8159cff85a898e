// Generated by gen_minimax.py (Lawson minimax fits; do not edit).
// atan(t) = t + t^3 Qa(t^2) on [0, 1]; atanh(z) = z + z^3 Qh(z^2) on [0, 1/2].
// Each function evaluates Q(u) by Horner's rule in fused multiply-adds, for
// one ray (V = float) or a pair of rays (V = float2, packed instructions).
#pragma once

#include "lensed_vec2.cuh"

namespace lensed {
template <class V>
__device__ __forceinline__ V minimax_atan_q(V u)
{
    V q = vsplat<V>(2.920640865e-03f);
    q = vfma(q, u, vsplat<V>(-1.636772417e-02f));
    q = vfma(q, u, vsplat<V>(4.321153462e-02f));
    q = vfma(q, u, vsplat<V>(-7.552187145e-02f));
    q = vfma(q, u, vsplat<V>(1.066599190e-01f));
    q = vfma(q, u, vsplat<V>(-1.421105266e-01f));
    q = vfma(q, u, vsplat<V>(1.999377310e-01f));
    q = vfma(q, u, vsplat<V>(-3.333315253e-01f));
    return q;
}
template <class V>
__device__ __forceinline__ V minimax_atanh_q(V u)
{
    V q = vsplat<V>(1.766911596e-01f);
    q = vfma(q, u, vsplat<V>(5.135826021e-02f));
    q = vfma(q, u, vsplat<V>(1.182372943e-01f));
    q = vfma(q, u, vsplat<V>(1.422276199e-01f));
    q = vfma(q, u, vsplat<V>(2.000251859e-01f));
    q = vfma(q, u, vsplat<V>(3.333330154e-01f));
    return q;
}
}  // namespace lensed
