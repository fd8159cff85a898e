// Lane-wise FP32 arithmetic on one ray (float) or on two rays at once
// (float2): sm_100-family GPUs execute a float2 multiply-add, add or multiply
// as one packed instruction (FFMA2 / FADD2 / FMUL2), two rays per issue slot.
// Every operation of both forms rounds once, to nearest, and is never fused
// with a neighbour by the compiler, so a ray's value is the same bits whether
// it is traced alone or as half of a pair.  Operations without a packed form
// (special functions, comparisons, minima) run per lane through vmap.
#pragma once

namespace lensed {

__device__ __forceinline__ float vfma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ float2 vfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float vmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float2 vmul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float vadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float2 vadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
// a - b with one rounding (for pairs: b * -1 is exact, so fma(b, -1, a) is
// the correctly rounded difference, signed zeros included)
__device__ __forceinline__ float vsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float2 vsub(float2 a, float2 b)
{
    return __ffma2_rn(b, make_float2(-1.f, -1.f), a);
}

// a uniform value in every lane
template <class V>
__device__ __forceinline__ V vsplat(float s);
template <>
__device__ __forceinline__ float vsplat<float>(float s)
{
    return s;
}
template <>
__device__ __forceinline__ float2 vsplat<float2>(float s)
{
    return make_float2(s, s);
}

// f applied to each lane
template <class F>
__device__ __forceinline__ float vmap(float a, F f)
{
    return f(a);
}
template <class F>
__device__ __forceinline__ float2 vmap(float2 a, F f)
{
    return make_float2(f(a.x), f(a.y));
}
template <class F>
__device__ __forceinline__ float vmap(float a, float b, F f)
{
    return f(a, b);
}
template <class F>
__device__ __forceinline__ float2 vmap(float2 a, float2 b, F f)
{
    return make_float2(f(a.x, b.x), f(a.y, b.y));
}
template <class F>
__device__ __forceinline__ float vmap(float a, float b, float c, float d, F f)
{
    return f(a, b, c, d);
}
template <class F>
__device__ __forceinline__ float2 vmap(float2 a, float2 b, float2 c, float2 d, F f)
{
    return make_float2(f(a.x, b.x, c.x, d.x), f(a.y, b.y, c.y, d.y));
}

// smallest lane
__device__ __forceinline__ float vminlane(float a) { return a; }
__device__ __forceinline__ float vminlane(float2 a) { return fminf(a.x, a.y); }

// G rays' values: G / 2 pairs and, for odd G, one single ray (the last)
template <int G>
struct Rays {
    static constexpr int NP = G / 2;
    float2 p[NP > 0 ? NP : 1];
    float t;
    __device__ __forceinline__ float get(int k) const
    {
        return k < 2 * NP ? ((k & 1) ? p[k >> 1].y : p[k >> 1].x) : t;
    }
    __device__ __forceinline__ void set(int k, float v)
    {
        if (k < 2 * NP) {
            if (k & 1) p[k >> 1].y = v;
            else p[k >> 1].x = v;
        } else {
            t = v;
        }
    }
    __device__ __forceinline__ void fill(float v)
    {
#pragma unroll
        for (int j = 0; j < NP; ++j) p[j] = make_float2(v, v);
        t = v;
    }
};

// f(pair values...) for every pair of rays, then f(ray values...) for the
// odd one: f is a generic callable over float2 and float
template <int G, class F, class... R>
__device__ __forceinline__ void for_rays(F &&f, R &...r)
{
#pragma unroll
    for (int j = 0; j < G / 2; ++j) f(r.p[j]...);
    if (G & 1) f(r.t...);
}

}  // namespace lensed
