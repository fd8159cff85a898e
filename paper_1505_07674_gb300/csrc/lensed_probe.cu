// Throughput probes for the roofline: measured FP32 FMA and MUFU (ex2)
// rates of the GPU, against which the ray kernels' achieved rates are read.
#include <cuda_runtime.h>

#include "lensed_internal.cuh"
#include "lensed_sie_trig.cuh"

namespace lensed {

__device__ __forceinline__ float probe_ex2(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// 8 independent FMA (or MUFU ex2) chains per thread, iters rounds; the result
// is stored so nothing is elided.
__global__ void k_probe_fma(int iters, float seed, float *__restrict__ sink)
{
    float a[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = seed + threadIdx.x * 1e-7f + k;
    const float b = 0.999999f, c = 1e-7f;
    for (int it = 0; it < iters; ++it)
#pragma unroll
        for (int k = 0; k < 8; ++k) a[k] = fmaf(a[k], b, c);
    float t = 0.f;
#pragma unroll
    for (int k = 0; k < 8; ++k) t += a[k];
    if (t == 12345.f) sink[blockIdx.x] = t;
}

__global__ void k_probe_mufu(int iters, float seed, float *__restrict__ sink)
{
    float a[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = seed * 1e-3f + threadIdx.x * 1e-9f + k * 1e-4f;
    for (int it = 0; it < iters; ++it)
#pragma unroll
        for (int k = 0; k < 8; ++k) a[k] = probe_ex2(a[k]) - 1.f;
    float t = 0.f;
#pragma unroll
    for (int k = 0; k < 8; ++k) t += a[k];
    if (t == 12345.f) sink[blockIdx.x] = t;
}

// The FP32 SIE's atan and atanh of n[i] / d[i] (lensed_sie_trig.cuh) beside
// CUDA's atanf / atanhf of the rounded quotient, for accuracy tests.
__global__ void k_probe_trig(const float *__restrict__ n, const float *__restrict__ d,
                             long long count, float *__restrict__ out)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
         i += (long long)gridDim.x * blockDim.x) {
        const float a = n[i], b = d[i];
        const float z = b > 0.f ? a / b : 0.f;
        out[i] = atan_ratio(a, b);
        out[count + i] = atanh_ratio(a, b);
        out[2 * count + i] = atanf(z);
        out[3 * count + i] = atanhf(z);
    }
}

void launch_trig_probe(const float *n, const float *d, long long count, float *out,
                       cudaStream_t st)
{
    if (count <= 0) return;
    const long long want = (count + 255) / 256;
    const unsigned grid = (unsigned)(want < 4096 ? want : 4096);
    k_probe_trig<<<grid, 256, 0, st>>>(n, d, count, out);
}

void launch_probe(int mufu, int blocks, int threads, int iters, float *sink, cudaStream_t st)
{
    if (mufu)
        k_probe_mufu<<<blocks, threads, 0, st>>>(iters, 0.5f, sink);
    else
        k_probe_fma<<<blocks, threads, 0, st>>>(iters, 0.5f, sink);
}

}  // namespace lensed
