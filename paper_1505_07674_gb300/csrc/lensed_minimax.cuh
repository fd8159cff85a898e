// Generated by gen_minimax.py (Lawson minimax fits; do not edit).
// atan(t) = t + t^3 Qa(t^2) on [0, 1]; atanh(z) = z + z^3 Qh(z^2) on [0, 1/2].
// Each function evaluates Q(u) by Horner's rule in fused multiply-adds.
#pragma once

namespace lensed {
__device__ __forceinline__ float minimax_atan_q(float u)
{
    float q = 2.920640865e-03f;
    q = fmaf(q, u, -1.636772417e-02f);
    q = fmaf(q, u, 4.321153462e-02f);
    q = fmaf(q, u, -7.552187145e-02f);
    q = fmaf(q, u, 1.066599190e-01f);
    q = fmaf(q, u, -1.421105266e-01f);
    q = fmaf(q, u, 1.999377310e-01f);
    q = fmaf(q, u, -3.333315253e-01f);
    return q;
}
__device__ __forceinline__ float minimax_atanh_q(float u)
{
    float q = 1.766911596e-01f;
    q = fmaf(q, u, 5.135826021e-02f);
    q = fmaf(q, u, 1.182372943e-01f);
    q = fmaf(q, u, 1.422276199e-01f);
    q = fmaf(q, u, 2.000251859e-01f);
    q = fmaf(q, u, 3.333330154e-01f);
    return q;
}
}  // namespace lensed
