// Log-likelihood surrogate network: BF16 tensor-core training and inference.
//
//   h1 = silu(x W1^T + b1), h2 = silu(h1 W2^T + b2), h3 = silu(h2 W3^T + b3),
//   y = h3 . w4 + b4;  loss = mean((y - t)^2) / 2.
//
// The likelihood driver uses it to pre-screen nested-sampling proposals; the
// exact likelihood decides every accepted point.  The paper has no such
// component.
//
// Every matrix product runs through k_gemm_tc: C[M][N] = A[M][K] B[N][K]^T
// with BF16 operands staged in shared memory by cp.async (double-buffered,
// 128 x 64 output tile per 128-thread block) and multiplied by tcgen05.mma
// into an FP32 accumulator in tensor memory, with fused epilogues: bias +
// SiLU (forward), times SiLU'(z) (backward), or plain FP32.  Gradients of the
// weights are products over the batch, so the batch-major activations and
// output gradients are transposed (k_transpose) to make the batch the
// contraction axis.  Reductions (bias gradients, output layer, loss) run in a
// fixed order, so a training step is deterministic.  Adam keeps FP32 master
// weights and refreshes the BF16 copies after each step.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <string>
#include <vector>

#include "lensed.h"

namespace lensed {
// lensed_runtime.cu: the test hook lensed_debug_fail_alloc and its count of
// live device buffers
bool alloc_failure_injected();
void note_buffers(int delta);
}

namespace {

typedef __nv_bfloat16 bf16;


thread_local std::string g_mlp_error;

int mfail(int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_mlp_error = buf;
    return code;
}

#define MCUDA(call)                                                                         \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess)                                                              \
            return mfail(e_ == cudaErrorMemoryAllocation ? LENSED_E_NOMEM : LENSED_E_CUDA,  \
                         "%s: %s", #call, cudaGetErrorString(e_));                          \
    } while (0)

__device__ __forceinline__ float silu(float z) { return z / (1.f + __expf(-z)); }
__device__ __forceinline__ float silu_grad(float z)
{
    const float s = 1.f / (1.f + __expf(-z));
    return s * (1.f + z * (1.f - s));
}

// 16-byte global -> shared copy; src_bytes = 0 fills the destination with
// zeros (rows beyond M or N).
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem, int src_bytes)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem),
                 "r"(src_bytes));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }

enum { EPI_F32 = 0, EPI_BIAS_SILU = 1, EPI_DSILU = 2 };

// Every product is C = A B^T, A: [M][lda] bf16 (K used), B: [N][ldb] bf16;
// K % 32 == 0, lda, ldb multiples of 8.  Epilogues:
//   EPI_F32        Cf[m][n] = acc
//   EPI_BIAS_SILU  z = acc + bias[n]; Zout[m][n] = z (if Zout); Hout = bf16(silu(z))
//   EPI_DSILU      d = acc * silu'(Zin[m][n]); Zout[m][n] = d; Hout = bf16(d)
// ---------------------------------------------------------------------------
// The product on the 5th-generation tensor cores, with the 128 x 128 FP32
// accumulator tile in tensor memory.  K is consumed in slices of 64 through a
// ring of kStages shared-memory buffers: all threads stage a slice of A (128
// rows) and B (128 rows) by cp.async in the canonical K-major layout without
// swizzle (core matrices of 8 rows x 16 bytes; the next core matrix along K
// 128 bytes on, along M/N 1024 bytes on; chunks beyond K or beyond M/N are
// zero-filled), and one thread issues the slice's four tcgen05.mma (K = 16
// each) and commits them to the buffer's mbarrier.  A buffer is refilled only
// after the mbarrier shows that the products reading it have completed, so
// the copies of the next slices overlap the tensor-core work.  The epilogue
// reads the accumulators with tcgen05.ld (warp w owns rows 32w..32w+31) into
// shared memory and applies the fused operation with coalesced row stores.
// Every wait on an mbarrier is bounded: on expiry the block records the
// failure in *err, waits (bounded, with the full limit) for its own
// tensor-core work, frees its tensor memory and returns.  `spin` is the poll
// limit of the pipeline waits (kSpinLimit unless a test lowers it to drive
// the expiry path).
constexpr int TM = 128, TN = 128, TK = 64, kStages = 3;
constexpr uint32_t kTmemCols = TN;          // one FP32 column per output column
constexpr int kSpinLimit = 1 << 24;         // mbarrier polls before giving up
constexpr int kStageA = TM * TK, kStageB = TN * TK;  // bf16 elements per buffer
constexpr size_t kGemmSmem = (size_t)kStages * (kStageA + kStageB) * sizeof(bf16);
static_assert((size_t)TM * (TN + 1) * sizeof(float) <= kGemmSmem, "epilogue tile must fit the ring");

__device__ __forceinline__ uint32_t saddr(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor: start, leading (K) and stride (M/N) byte
// offsets, descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

// Instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, N = TN, M = TM.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TN >> 3) << 17) |
                            ((uint32_t)(TM >> 4) << 24);

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int limit)
{
    for (int it = 0; it < limit; ++it) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            " selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

template <int EPI>
__global__ void __launch_bounds__(128)
    k_gemm_tc(const bf16 *__restrict__ A, int lda, const bf16 *__restrict__ B, int ldb, int M,
              int N, int K, float *__restrict__ Cf, int ldc, const float *__restrict__ bias,
              const float *__restrict__ Zin, float *__restrict__ Zout, bf16 *__restrict__ Hout,
              int *__restrict__ err, int spin, int kchunk)
{
    extern __shared__ __align__(128) unsigned char g_smem[];
    if (kchunk > 0) {
        // split-K (EPI_F32 only): block z contracts K range [z kchunk, (z+1) kchunk)
        // into its own [M][ldc] slab of Cf; a fixed-order sum follows
        const int kz = blockIdx.z * kchunk;
        A += kz;
        B += kz;
        K = min(kchunk, K - kz);
        Cf += (size_t)blockIdx.z * M * ldc;
    }
    bf16 *As = reinterpret_cast<bf16 *>(g_smem);
    bf16 *Bs = As + kStages * kStageA;
    __shared__ __align__(8) unsigned long long s_bar[kStages];
    __shared__ uint32_t s_tmem;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.y * TM, n0 = blockIdx.x * TN;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(saddr(&s_tmem)), "r"(kTmemCols) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int b = 0; b < kStages; ++b)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(&s_bar[b])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;

    // 16-byte chunk (row r, K chunk j) of a slice -> its core-matrix slot
    auto load = [&](int stage, int k0) {
        bf16 *a = As + stage * kStageA, *b = Bs + stage * kStageB;
#pragma unroll
        for (int it = 0; it < (TM * TK / 8) / 128; ++it) {
            const int ch = tid + it * 128, r = ch >> 3, j = ch & 7;
            const int gm = m0 + r, gk = k0 + j * 8;
            const bool in = gm < M && gk < K;
            cp_async16(a + (r >> 3) * 512 + j * 64 + (r & 7) * 8,
                       A + (size_t)min(gm, M - 1) * lda + (in ? gk : 0), in ? 16 : 0);
        }
#pragma unroll
        for (int it = 0; it < (TN * TK / 8) / 128; ++it) {
            const int ch = tid + it * 128, r = ch >> 3, j = ch & 7;
            const int gn = n0 + r, gk = k0 + j * 8;
            const bool in = gn < N && gk < K;
            cp_async16(b + (r >> 3) * 512 + j * 64 + (r & 7) * 8,
                       B + (size_t)min(gn, N - 1) * ldb + (in ? gk : 0), in ? 16 : 0);
        }
    };

    const int nk = (K + TK - 1) / TK;
    bool ok = true;
    int issued = 0;  // slices whose products were committed
    for (int s = 0; s < kStages - 1; ++s) {
        if (s < nk) load(s, s * TK);
        cp_async_commit();
    }
    for (int kt = 0; kt < nk && ok; ++kt) {
        const int stage = kt % kStages;
        asm volatile("cp.async.wait_group %0;" ::"n"(kStages - 2) : "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            tc_fence_after();
            const uint32_t a0 = saddr(As + stage * kStageA), b0 = saddr(Bs + stage * kStageB);
#pragma unroll
            for (int s = 0; s < TK / 16; ++s) {
                const uint64_t ad = smem_desc(a0 + s * 256, 128, 1024);
                const uint64_t bd = smem_desc(b0 + s * 256, 128, 1024);
                const uint32_t acc = (kt > 0 || s > 0) ? 1u : 0u;
                asm volatile(
                    "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                    " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
                    ::"r"(tmem), "l"(ad), "l"(bd), "r"(kIdesc), "r"(acc)
                    : "memory");
            }
            asm volatile(
                "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                ::"r"(saddr(&s_bar[stage])) : "memory");
        }
        issued = kt + 1;
        // refill the buffer of slice kt - 1 with slice kt + kStages - 1 once
        // the products that read it are done
        const int next = kt + kStages - 1;
        if (next < nk) {
            bool w = true;
            if (kt >= 1)
                w = mbar_wait(saddr(&s_bar[(kt - 1) % kStages]),
                              (uint32_t)(((kt - 1) / kStages) & 1), spin);
            // one decision for the whole block, so no thread leaves the
            // loop while another waits at its barrier
            if (!__syncthreads_and(w)) {
                ok = false;
                if (tid == 0) atomicExch(err, 1);
            }
            if (ok) load(next % kStages, next * TK);
        }
        cp_async_commit();
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    // the last slice's commit covers every earlier product (always the full
    // limit: tensor memory is freed only after the block's products are done)
    const bool done = __syncthreads_and(
        issued > 0 && mbar_wait(saddr(&s_bar[(issued - 1) % kStages]),
                                (uint32_t)(((issued - 1) / kStages) & 1), kSpinLimit));
    if ((!done || !ok) && tid == 0) atomicExch(err, 1);
    // epilogue: accumulators -> shared memory (the ring is free now), then
    // coalesced row-wise stores with the fused operation
    float *stile = reinterpret_cast<float *>(g_smem);  // [TM][TN + 1]
    if (done && ok) {
        tc_fence_after();
#pragma unroll 1
        for (int c0 = 0; c0 < TN; c0 += 16) {
            if (n0 + c0 >= N) break;
            uint32_t v[16];
            const uint32_t ta = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, "
                "%9, %10, %11, %12, %13, %14, %15}, [%16];"
                : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]),
                  "=r"(v[6]), "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]),
                  "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
                : "r"(ta));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            float *dst = stile + (size_t)(warp * 32 + lane) * (TN + 1) + c0;
#pragma unroll
            for (int e = 0; e < 16; ++e) dst[e] = __uint_as_float(v[e]);
        }
    }
    __syncthreads();
    if (done && ok) {
        const int ncol = min(TN, N - n0);
        for (int idx = tid; idx < TM * TN; idx += 128) {
            const int r = idx / TN, c = idx - (idx / TN) * TN;
            const int row = m0 + r, n = n0 + c;
            if (row >= M || c >= ncol) continue;
            const float acc = stile[(size_t)r * (TN + 1) + c];
            const size_t o = (size_t)row * ldc + n;
            if (EPI == EPI_F32) {
                Cf[o] = acc;
            } else if (EPI == EPI_BIAS_SILU) {
                const float z = acc + bias[n];
                if (Zout) Zout[o] = z;
                Hout[o] = __float2bfloat16(silu(z));
            } else {
                const float d = acc * silu_grad(Zin[o]);
                Zout[o] = d;
                Hout[o] = __float2bfloat16(d);
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(kTmemCols) : "memory");
    }
}

// [R][C] bf16 -> [C][R] bf16 (32 x 32 tiles through shared memory)
__global__ void k_transpose(const bf16 *__restrict__ in, int R, int C, bf16 *__restrict__ out)
{
    __shared__ bf16 t[32][33];
    const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const int r = r0 + k, c = c0 + threadIdx.x;
        if (r < R && c < C) t[k][threadIdx.x] = in[(size_t)r * C + c];
    }
    __syncthreads();
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const int c = c0 + k, r = r0 + threadIdx.x;
        if (r < R && c < C) out[(size_t)c * R + r] = t[threadIdx.x][k];
    }
}

// inputs [B][n_in] fp32 -> [Bp][kin] bf16, zero padded
__global__ void k_pack(const float *__restrict__ X, int B, int n_in, int Bp, int kin,
                       bf16 *__restrict__ Xb)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)Bp * kin) return;
    const int r = (int)(i / kin), c = (int)(i % kin);
    Xb[i] = __float2bfloat16(r < B && c < n_in ? X[(size_t)r * n_in + c] : 0.f);
}

// y[m] = h3[m] . w4 + b4 (one warp per row, fixed-order lane sums)
__global__ void k_out(const bf16 *__restrict__ H3, int H, const float *__restrict__ w4,
                      const float *__restrict__ b4, int B, float *__restrict__ y)
{
    const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (row >= B) return;
    float s = 0.f;
    for (int k = lane; k < H; k += 32) s += __bfloat162float(H3[(size_t)row * H + k]) * w4[k];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) y[row] = s + b4[0];
}

// Backward of the output layer: dy = (y - t)/B (zero on padding rows),
// dZ3 = dy w4 silu'(Z3); loss terms r^2/(2B) per row.
__global__ void k_out_back(const float *__restrict__ y, const float *__restrict__ t, int B, int Bp,
                           int H, const float *__restrict__ w4, const float *__restrict__ Z3,
                           float *__restrict__ dy, float *__restrict__ lossrow,
                           float *__restrict__ dZf, bf16 *__restrict__ dZb)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)Bp * H) return;
    const int m = (int)(i / H), k = (int)(i % H);
    const float r = m < B ? y[m] - t[m] : 0.f;
    const float d = r / (float)B;
    if (k == 0) {
        dy[m] = d;
        lossrow[m] = 0.5f * r * r / (float)B;
    }
    const float g = d * w4[k] * silu_grad(Z3[i]);
    dZf[i] = g;
    dZb[i] = __float2bfloat16(g);
}

// Column sums out[n] = sum_m w[m] in[m][n] (w = 1 when NULL) in two passes
// with a fixed order: block (x, y) sums rows [y R, (y+1) R) of 32 columns
// (8 row lanes per column, then the 8 lane sums in order) into part[y][n];
// k_colsum_final adds the parts in order.
constexpr int kColParts = 64;

template <typename T>
__global__ void __launch_bounds__(256)
    k_colsum_part(const T *__restrict__ in, const float *__restrict__ w, int M, int N, int R,
                  float *__restrict__ part)
{
    __shared__ float t[8][33];
    const int n = blockIdx.x * 32 + threadIdx.x;
    const int m0 = blockIdx.y * R, m1 = min(M, m0 + R);
    float s = 0.f;
    if (n < N)
        for (int m = m0 + threadIdx.y; m < m1; m += 8) {
            const float v = (float)in[(size_t)m * N + n];
            s = w ? fmaf(v, w[m], s) : s + v;
        }
    t[threadIdx.y][threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.y == 0 && n < N) {
        float r = 0.f;
#pragma unroll
        for (int k = 0; k < 8; ++k) r += t[k][threadIdx.x];
        part[(size_t)blockIdx.y * N + n] = r;
    }
}

__global__ void k_colsum_final(const float *__restrict__ part, int S, int N,
                               float *__restrict__ out)
{
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    float s = 0.f;
    for (int z = 0; z < S; ++z) s += part[(size_t)z * N + n];
    out[n] = s;
}

// out[0] = sum of n values: 1024 threads, strided lane sums, then a fixed
// shared-memory tree
__global__ void __launch_bounds__(1024) k_sum(const float *__restrict__ in, int n,
                                              float *__restrict__ out)
{
    __shared__ float t[1024];
    float s = 0.f;
    for (int i = threadIdx.x; i < n; i += 1024) s += in[i];
    t[threadIdx.x] = s;
    __syncthreads();
    for (int w = 512; w > 0; w >>= 1) {
        if (threadIdx.x < w) t[threadIdx.x] += t[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = t[0];
}

// copy the first c columns of [R][ld] into [R][c]
__global__ void k_copy_cols(const float *__restrict__ in, int R, int ld, int c,
                            float *__restrict__ out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= R * c) return;
    out[i] = in[(size_t)(i / c) * ld + (i % c)];
}

__global__ void k_adam(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                       float *__restrict__ v, int n, float lr, float c1, float c2)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = 0.9f * m[i] + 0.1f * gi;
    const float vi = 0.999f * v[i] + 0.001f * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + 1e-8f);
}

// bf16 weight copies from the fp32 master: W1 into [H][kin] (zero padded),
// W2, W3 as they are
__global__ void k_refresh(const float *__restrict__ p, int n_in, int kin, int H,
                          bf16 *__restrict__ W1b, bf16 *__restrict__ W2b, bf16 *__restrict__ W3b)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int n1 = H * kin, n2 = H * H;
    if (i < n1) {
        const int r = i / kin, c = i % kin;
        W1b[i] = __float2bfloat16(c < n_in ? p[r * n_in + c] : 0.f);
    }
    const size_t o2 = (size_t)H * n_in + H;
    const size_t o3 = o2 + (size_t)H * H + H;
    if (i < n2) {
        W2b[i] = __float2bfloat16(p[o2 + i]);
        W3b[i] = __float2bfloat16(p[o3 + i]);
    }
}

template <typename T>
struct Buf {
    T *p = nullptr;
    size_t n = 0;
    ~Buf() { release(); }
    void release()
    {
        if (p) {
            cudaFree(p);
            lensed::note_buffers(-1);
        }
        p = nullptr;
    }
    int alloc(size_t count)
    {
        release();
        n = 0;
        if (lensed::alloc_failure_injected())
            return mfail(LENSED_E_NOMEM, "cudaMalloc: refused by the injected allocation failure");
        cudaError_t e = cudaMalloc(&p, std::max<size_t>(count, 1) * sizeof(T));
        if (e != cudaSuccess) {
            p = nullptr;
            return mfail(LENSED_E_NOMEM, "cudaMalloc: %s", cudaGetErrorString(e));
        }
        lensed::note_buffers(1);
        n = count;
        return LENSED_OK;
    }
};

// ---------------------------------------------------------------------------
// Proposals for the nested-sampling driver, drawn uniformly inside an
// ellipsoid and pre-screened by the network.
//
// Counter-based generator: Philox4x32-10 (Salmon, Moraes, Dror & Shaw, "Parallel
// random numbers: as easy as 1, 2, 3", SC'11), written from its published
// definition: ten rounds of two 32x32->64-bit products with the multipliers
// 0xD2511F53 and 0xCD9E8D57, the key bumped by the Weyl constants 0x9E3779B9
// and 0xBB67AE85 between rounds.  Candidate i of a stream draws the counters
// (i, j, 0, 0), j = 0, 1, ..., under the key (seed low, seed high), so every
// candidate is reproducible on its own.
struct Philox4 {
    uint32_t v[4];
};

__device__ __forceinline__ Philox4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t k0,
                                                 uint32_t k1)
{
    uint32_t x0 = c0, x1 = c1, x2 = 0u, x3 = 0u;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint64_t p0 = (uint64_t)0xD2511F53u * x0;
        const uint64_t p1 = (uint64_t)0xCD9E8D57u * x2;
        const uint32_t n0 = (uint32_t)(p1 >> 32) ^ x1 ^ k0;
        const uint32_t n2 = (uint32_t)(p0 >> 32) ^ x3 ^ k1;
        x1 = (uint32_t)p1;
        x3 = (uint32_t)p0;
        x0 = n0;
        x2 = n2;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return {{x0, x1, x2, x3}};
}

// 24-bit uniform in (0, 1)
__device__ __forceinline__ float u01f(uint32_t x)
{
    return ((float)(x >> 8) + 0.5f) * (1.f / 16777216.f);
}

constexpr int kMaxScreenDim = 32;

// Candidate `i` of stream `seed`: v = c + L z, z uniform in the unit ball
// (Gaussian direction by Box-Muller, radius U^(1/d)), in coordinates whose
// periodic axes are shifted by `shift` (0 on the others); returns whether v
// lies inside the open unit cube, and u = v + shift wrapped into [0, 1), the
// point in the sampler's coordinates (shifting and wrapping a periodic axis
// preserves the uniform measure).  FP32: a proposal needs no more than float
// resolution, and the sampler uses the point exactly as drawn.
__device__ bool ellipsoid_point(int d, unsigned long long seed, unsigned long long i,
                                const float *__restrict__ c, const float *__restrict__ L,
                                const float *__restrict__ shift, float *u)
{
    const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    float z[kMaxScreenDim];
    // d normals (Box-Muller pairs) and one uniform for the radius, four
    // uniforms per Philox call
    const int n_u = 2 * ((d + 1) / 2) + 1;
    float uu[kMaxScreenDim + 4];
    for (int j = 0; 4 * j < n_u; ++j) {
        const Philox4 r = philox4x32_10((uint32_t)i, (uint32_t)(i >> 32) ^ ((uint32_t)j << 16), k0,
                                        k1);
#pragma unroll
        for (int e = 0; e < 4; ++e) uu[4 * j + e] = u01f(r.v[e]);
    }
    float n2 = 0.f;
    for (int j = 0; j < d; j += 2) {
        const float rr = sqrtf(-2.f * logf(uu[j]));
        float sn, cs;
        sincospif(2.f * uu[j + 1], &sn, &cs);
        z[j] = rr * cs;
        n2 += z[j] * z[j];
        if (j + 1 < d) {
            z[j + 1] = rr * sn;
            n2 += z[j + 1] * z[j + 1];
        }
    }
    const float rad = exp2f(log2f(uu[n_u - 1]) / (float)d) * rsqrtf(n2);
    bool inside = true;
    for (int j = 0; j < d; ++j) {
        float a = 0.f;
        for (int k = 0; k <= j; ++k) a = fmaf(L[j * d + k], z[k], a);
        a = fmaf(a, rad, c[j]);
        inside = inside && a > 0.f && a < 1.f;
        if (shift) {
            a += shift[j];
            if (a >= 1.f) a -= 1.f;
        }
        u[j] = a;
    }
    return inside;
}

// Network inputs of candidates [first, first + n): X[i] = A (u_i - xc), and
// whether u_i lies inside the unit cube.
__global__ void k_ell_draw(int d, int n, unsigned long long seed, unsigned long long first,
                           const float *__restrict__ c, const float *__restrict__ L,
                           const float *__restrict__ shift, const float *__restrict__ xc,
                           const float *__restrict__ A, float *__restrict__ X,
                           unsigned char *__restrict__ inside)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float u[kMaxScreenDim];
    inside[i] = ellipsoid_point(d, seed, first + i, c, L, shift, u) ? 1 : 0;
    for (int j = 0; j < d; ++j) u[j] -= xc[j];
    for (int j = 0; j < d; ++j) {
        float a = 0.f;
        for (int k = 0; k < d; ++k) a = fmaf(A[j * d + k], u[k], a);
        X[(size_t)i * d + j] = a;
    }
}

// Survivors: inside the cube and (screened) with network output below the
// cut.  Each takes a slot by an atomic counter (the host restores the
// candidate order from idx_out) and gets its point recomputed.
__global__ void k_ell_select(int d, int n, unsigned long long seed, unsigned long long first,
                             const float *__restrict__ c, const float *__restrict__ L,
                             const float *__restrict__ shift,
                             const unsigned char *__restrict__ inside,
                             const float *__restrict__ y, float y_cut, double *__restrict__ u_out,
                             int *__restrict__ idx_out, int *__restrict__ n_out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float u[kMaxScreenDim];
    bool keep;
    if (inside) {
        keep = inside[i] && y[i] < y_cut;  // NaN outputs are screened out
        if (keep) ellipsoid_point(d, seed, first + i, c, L, shift, u);
    } else {
        keep = ellipsoid_point(d, seed, first + i, c, L, shift, u);
    }
    if (!keep) return;
    const int slot = atomicAdd(n_out, 1);
    idx_out[slot] = i;
    for (int j = 0; j < d; ++j) u_out[(size_t)slot * d + j] = (double)u[j];
}

}  // namespace

struct lensed_mlp {
    int n_in, H, kin, maxB, Bp;  // Bp: max batch rounded up to 64
    size_t np;                   // parameter count
    size_t o_b1, o_W2, o_b2, o_W3, o_b3, o_w4, o_b4;
    long long step = 0;
    Buf<float> p, m, v, g;
    Buf<bf16> W1b, W2b, W3b, WT;
    Buf<bf16> Xb, XbT, H1, H2, H3, HT, dZa, dZbuf, dZT;
    Buf<float> Z1, Z2, Z3, dZf, y, dy, lossrow, gW1, tmpcol;
    Buf<float> ws;    // split-K partial weight gradients [kMaxSplit][H][max(H, kin)]
    Buf<float> part;  // column-sum parts [kColParts][H]
    Buf<int> err;  // set by a tensor-core wait that expired
    int spin = kSpinLimit;  // poll limit of the GEMM pipeline waits
    // proposal screening scratch (grown on demand)
    Buf<float> sX, sy;
    Buf<unsigned char> sin;
};

namespace {

int launch_gemm(int epi, const bf16 *A, int lda, const bf16 *B, int ldb, int M, int N, int K,
                float *Cf, int ldc, const float *bias, const float *Zin, float *Zout, bf16 *Hout,
                int *err, cudaStream_t st, int spin = kSpinLimit)
{
    dim3 grid((N + TN - 1) / TN, (M + TM - 1) / TM);
    if (epi == EPI_F32)
        k_gemm_tc<EPI_F32><<<grid, 128, kGemmSmem, st>>>(A, lda, B, ldb, M, N, K, Cf, ldc, bias,
                                                         Zin, Zout, Hout, err, spin, 0);
    else if (epi == EPI_BIAS_SILU)
        k_gemm_tc<EPI_BIAS_SILU><<<grid, 128, kGemmSmem, st>>>(A, lda, B, ldb, M, N, K, Cf, ldc,
                                                               bias, Zin, Zout, Hout, err, spin, 0);
    else
        k_gemm_tc<EPI_DSILU><<<grid, 128, kGemmSmem, st>>>(A, lda, B, ldb, M, N, K, Cf, ldc, bias,
                                                           Zin, Zout, Hout, err, spin, 0);
    return LENSED_OK;
}

// Weight gradient C[M][N] = A B^T with a long contraction (K = the batch):
// split into S <= kMaxSplit ranges of >= 4 K-slices, one block row per range
// (so M/TM x N/TN x S blocks keep the tensor cores of many SMs busy), the
// partial products summed in range order (deterministic).
constexpr int kMaxSplit = 32;

__global__ void k_splitk_sum(const float *__restrict__ ws, int S, int M, int N,
                             float *__restrict__ C, int ldc)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= M * N) return;
    const int r = i / N, c = i - (i / N) * N;
    float s = 0.f;
    for (int z = 0; z < S; ++z) s += ws[(size_t)z * M * N + i];
    C[(size_t)r * ldc + c] = s;
}

void launch_wgrad(const bf16 *A, int lda, const bf16 *B, int ldb, int M, int N, int K, float *C,
                  int ldc, float *ws, int *err, cudaStream_t st, int spin)
{
    const int slices = (K + TK - 1) / TK;
    const int S = std::max(1, std::min(kMaxSplit, slices / 4));
    const int kchunk = (slices + S - 1) / S * TK;
    const int Sz = (K + kchunk - 1) / kchunk;
    dim3 grid((N + TN - 1) / TN, (M + TM - 1) / TM, Sz);
    k_gemm_tc<EPI_F32><<<grid, 128, kGemmSmem, st>>>(A, lda, B, ldb, M, N, K, ws, N, nullptr,
                                                     nullptr, nullptr, nullptr, err, spin, kchunk);
    k_splitk_sum<<<(M * N + 255) / 256, 256, 0, st>>>(ws, Sz, M, N, C, ldc);
}

void transpose(const bf16 *in, int R, int C, bf16 *out, cudaStream_t st)
{
    dim3 grid((C + 31) / 32, (R + 31) / 32), block(32, 8);
    k_transpose<<<grid, block, 0, st>>>(in, R, C, out);
}

// forward of rows [0, B) (B <= maxB): fills Xb, Z*, H*, y
void forward(lensed_mlp *m, const float *X, int B, float *y, bool keep_z, cudaStream_t st)
{
    const int Bp = (B + 63) / 64 * 64, H = m->H;
    const long long nx = (long long)Bp * m->kin;
    k_pack<<<(unsigned)((nx + 255) / 256), 256, 0, st>>>(X, B, m->n_in, Bp, m->kin, m->Xb.p);
    launch_gemm(EPI_BIAS_SILU, m->Xb.p, m->kin, m->W1b.p, m->kin, Bp, H, m->kin, nullptr, H,
                m->p.p + m->o_b1, nullptr, keep_z ? m->Z1.p : nullptr, m->H1.p, m->err.p, st, m->spin);
    launch_gemm(EPI_BIAS_SILU, m->H1.p, H, m->W2b.p, H, Bp, H, H, nullptr, H, m->p.p + m->o_b2,
                nullptr, keep_z ? m->Z2.p : nullptr, m->H2.p, m->err.p, st, m->spin);
    launch_gemm(EPI_BIAS_SILU, m->H2.p, H, m->W3b.p, H, Bp, H, H, nullptr, H, m->p.p + m->o_b3,
                nullptr, keep_z ? m->Z3.p : nullptr, m->H3.p, m->err.p, st, m->spin);
    k_out<<<(B + 7) / 8, 256, 0, st>>>(m->H3.p, H, m->p.p + m->o_w4, m->p.p + m->o_b4, B, y);
}

// out[n] = sum_m w[m] in[m][n] over M rows (w NULL: 1), fixed order
template <typename T>
void colsum(lensed_mlp *m, const T *in, const float *w, int M, int N, float *out, cudaStream_t st)
{
    const int R = (M + kColParts - 1) / kColParts;
    const int S = (M + R - 1) / R;
    k_colsum_part<T><<<dim3((N + 31) / 32, S), dim3(32, 8), 0, st>>>(in, w, M, N, R, m->part.p);
    k_colsum_final<<<(N + 127) / 128, 128, 0, st>>>(m->part.p, S, N, out);
}

// loss and gradient of rows [0, B) into m->g and loss (device scalar)
void gradient(lensed_mlp *m, const float *X, const float *t, int B, float *loss, cudaStream_t st)
{
    const int Bp = (B + 63) / 64 * 64, H = m->H;
    forward(m, X, B, m->y.p, true, st);
    const long long nbh = (long long)Bp * H;
    float *g = m->g.p;
    // output layer and dZ3
    k_out_back<<<(unsigned)((nbh + 255) / 256), 256, 0, st>>>(m->y.p, t, B, Bp, H,
                                                               m->p.p + m->o_w4, m->Z3.p, m->dy.p,
                                                               m->lossrow.p, m->dZf.p, m->dZa.p);
    k_sum<<<1, 1024, 0, st>>>(m->lossrow.p, Bp, loss);
    colsum(m, m->H3.p, m->dy.p, Bp, H, g + m->o_w4, st);  // dw4 = sum_m dy[m] h3[m]
    k_sum<<<1, 1024, 0, st>>>(m->dy.p, Bp, g + m->o_b4);
    // layer 3: dW3 = dZ3^T H2, db3, dZ2 = (dZ3 W3) * silu'(Z2)
    transpose(m->dZa.p, Bp, H, m->dZT.p, st);
    transpose(m->H2.p, Bp, H, m->HT.p, st);
    launch_wgrad(m->dZT.p, Bp, m->HT.p, Bp, H, H, Bp, g + m->o_W3, H, m->ws.p, m->err.p, st,
                 m->spin);
    colsum(m, m->dZf.p, nullptr, Bp, H, g + m->o_b3, st);
    transpose(m->W3b.p, H, H, m->WT.p, st);
    launch_gemm(EPI_DSILU, m->dZa.p, H, m->WT.p, H, Bp, H, H, nullptr, H, nullptr, m->Z2.p,
                m->dZf.p, m->dZbuf.p, m->err.p, st, m->spin);
    // layer 2
    transpose(m->dZbuf.p, Bp, H, m->dZT.p, st);
    transpose(m->H1.p, Bp, H, m->HT.p, st);
    launch_wgrad(m->dZT.p, Bp, m->HT.p, Bp, H, H, Bp, g + m->o_W2, H, m->ws.p, m->err.p, st,
                 m->spin);
    colsum(m, m->dZf.p, nullptr, Bp, H, g + m->o_b2, st);
    transpose(m->W2b.p, H, H, m->WT.p, st);
    launch_gemm(EPI_DSILU, m->dZbuf.p, H, m->WT.p, H, Bp, H, H, nullptr, H, nullptr, m->Z1.p,
                m->dZf.p, m->dZa.p, m->err.p, st, m->spin);
    // layer 1: dW1 = dZ1^T X (padded to kin columns), db1
    transpose(m->dZa.p, Bp, H, m->dZT.p, st);
    transpose(m->Xb.p, Bp, m->kin, m->XbT.p, st);
    launch_wgrad(m->dZT.p, Bp, m->XbT.p, Bp, H, m->kin, Bp, m->gW1.p, m->kin, m->ws.p, m->err.p,
                 st, m->spin);
    k_copy_cols<<<(H * m->n_in + 255) / 256, 256, 0, st>>>(m->gW1.p, H, m->kin, m->n_in, g);
    colsum(m, m->dZf.p, nullptr, Bp, H, g + m->o_b1, st);
}

int refresh(lensed_mlp *m, cudaStream_t st)
{
    const int n = std::max(m->H * m->kin, m->H * m->H);
    k_refresh<<<(n + 255) / 256, 256, 0, st>>>(m->p.p, m->n_in, m->kin, m->H, m->W1b.p, m->W2b.p,
                                                m->W3b.p);
    MCUDA(cudaGetLastError());
    return LENSED_OK;
}

}  // namespace

extern "C" const char *lensed_mlp_last_error(void) { return g_mlp_error.c_str(); }

extern "C" int lensed_mlp_create(int n_in, int hidden, int max_batch, lensed_mlp **out)
{
    g_mlp_error.clear();
    if (!out) return mfail(LENSED_E_ARG, "out is NULL");
    if (n_in < 1 || n_in > 64) return mfail(LENSED_E_ARG, "n_in = %d (1..64)", n_in);
    if (hidden < 64 || hidden % 64) return mfail(LENSED_E_ARG, "hidden = %d (multiple of 64)", hidden);
    if (max_batch < 1) return mfail(LENSED_E_ARG, "max_batch = %d", max_batch);
    cudaFuncSetAttribute(k_gemm_tc<EPI_F32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)kGemmSmem);
    cudaFuncSetAttribute(k_gemm_tc<EPI_BIAS_SILU>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)kGemmSmem);
    cudaFuncSetAttribute(k_gemm_tc<EPI_DSILU>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)kGemmSmem);
    lensed_mlp *m = new lensed_mlp();
    m->n_in = n_in;
    m->H = hidden;
    m->kin = (n_in + 31) / 32 * 32;
    m->maxB = max_batch;
    m->Bp = (max_batch + 63) / 64 * 64;
    const size_t H = hidden;
    m->o_b1 = H * n_in;
    m->o_W2 = m->o_b1 + H;
    m->o_b2 = m->o_W2 + H * H;
    m->o_W3 = m->o_b2 + H;
    m->o_b3 = m->o_W3 + H * H;
    m->o_w4 = m->o_b3 + H;
    m->o_b4 = m->o_w4 + H;
    m->np = m->o_b4 + 1;
    const size_t bh = (size_t)m->Bp * H;
    int rc;
    if ((rc = m->p.alloc(m->np)) || (rc = m->m.alloc(m->np)) || (rc = m->v.alloc(m->np)) ||
        (rc = m->g.alloc(m->np)) || (rc = m->W1b.alloc(H * m->kin)) ||
        (rc = m->W2b.alloc(H * H)) || (rc = m->W3b.alloc(H * H)) || (rc = m->WT.alloc(H * H)) ||
        (rc = m->Xb.alloc((size_t)m->Bp * m->kin)) || (rc = m->XbT.alloc((size_t)m->Bp * m->kin)) ||
        (rc = m->H1.alloc(bh)) || (rc = m->H2.alloc(bh)) || (rc = m->H3.alloc(bh)) ||
        (rc = m->HT.alloc(bh)) || (rc = m->dZa.alloc(bh)) || (rc = m->dZbuf.alloc(bh)) ||
        (rc = m->dZT.alloc(bh)) || (rc = m->Z1.alloc(bh)) || (rc = m->Z2.alloc(bh)) ||
        (rc = m->Z3.alloc(bh)) || (rc = m->dZf.alloc(bh)) || (rc = m->y.alloc(m->Bp)) ||
        (rc = m->dy.alloc(m->Bp)) || (rc = m->lossrow.alloc(m->Bp)) ||
        (rc = m->gW1.alloc(H * m->kin)) || (rc = m->tmpcol.alloc(H)) || (rc = m->err.alloc(1)) ||
        (rc = m->ws.alloc((size_t)kMaxSplit * H * std::max<size_t>(H, m->kin))) ||
        (rc = m->part.alloc((size_t)kColParts * H))) {
        std::string msg = g_mlp_error;
        delete m;
        g_mlp_error = msg;
        return rc;
    }
    cudaMemset(m->p.p, 0, m->np * sizeof(float));
    cudaMemset(m->err.p, 0, sizeof(int));
    cudaMemset(m->m.p, 0, m->np * sizeof(float));
    cudaMemset(m->v.p, 0, m->np * sizeof(float));
    if ((rc = refresh(m, nullptr))) {
        delete m;
        return rc;
    }
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        delete m;
        return mfail(LENSED_E_CUDA, "create: %s", cudaGetErrorString(e));
    }
    *out = m;
    return LENSED_OK;
}

extern "C" void lensed_mlp_destroy(lensed_mlp *m)
{
    if (!m) return;
    cudaDeviceSynchronize();
    delete m;
}

extern "C" long long lensed_mlp_param_count(const lensed_mlp *m) { return m ? (long long)m->np : -1; }

extern "C" int lensed_mlp_debug_spin_limit(lensed_mlp *m, int polls)
{
    if (!m) return mfail(LENSED_E_ARG, "NULL argument");
    if (polls < 0) return mfail(LENSED_E_ARG, "polls = %d must be >= 0", polls);
    m->spin = polls > kSpinLimit ? kSpinLimit : polls;
    return LENSED_OK;
}

extern "C" int lensed_mlp_set_params(lensed_mlp *m, const float *host_params)
{
    if (!m || !host_params) return mfail(LENSED_E_ARG, "NULL argument");
    MCUDA(cudaDeviceSynchronize());
    MCUDA(cudaMemcpy(m->p.p, host_params, m->np * sizeof(float), cudaMemcpyHostToDevice));
    MCUDA(cudaMemset(m->m.p, 0, m->np * sizeof(float)));
    MCUDA(cudaMemset(m->v.p, 0, m->np * sizeof(float)));
    MCUDA(cudaMemset(m->err.p, 0, sizeof(int)));  // a fresh state: no expired wait
    m->step = 0;
    int rc = refresh(m, nullptr);
    if (rc) return rc;
    MCUDA(cudaDeviceSynchronize());
    return LENSED_OK;
}

extern "C" int lensed_mlp_get_params(const lensed_mlp *m, float *host_params)
{
    if (!m || !host_params) return mfail(LENSED_E_ARG, "NULL argument");
    MCUDA(cudaDeviceSynchronize());
    int err = 0;
    MCUDA(cudaMemcpy(&err, m->err.p, sizeof(int), cudaMemcpyDeviceToHost));
    if (err)
        return mfail(LENSED_E_TIMEOUT, "a tensor-core wait expired in an earlier call; "
                                       "its results are invalid");
    MCUDA(cudaMemcpy(host_params, m->p.p, m->np * sizeof(float), cudaMemcpyDeviceToHost));
    return LENSED_OK;
}

extern "C" int lensed_mlp_forward(lensed_mlp *m, const float *X, int B, float *y, void *stream)
{
    if (!m || !X || !y) return mfail(LENSED_E_ARG, "NULL argument");
    if (B < 0) return mfail(LENSED_E_ARG, "B = %d", B);
    cudaStream_t st = (cudaStream_t)stream;
    for (int b0 = 0; b0 < B; b0 += m->maxB) {
        const int nb = std::min(m->maxB, B - b0);
        forward(m, X + (size_t)b0 * m->n_in, nb, y + b0, false, st);
    }
    MCUDA(cudaGetLastError());
    return LENSED_OK;
}

extern "C" int lensed_mlp_gradient(lensed_mlp *m, const float *X, const float *t, int B,
                                   float *grad, float *loss, void *stream)
{
    if (!m || !X || !t || !grad || !loss) return mfail(LENSED_E_ARG, "NULL argument");
    if (B < 1 || B > m->maxB) return mfail(LENSED_E_ARG, "B = %d (1..%d)", B, m->maxB);
    cudaStream_t st = (cudaStream_t)stream;
    gradient(m, X, t, B, loss, st);
    MCUDA(cudaMemcpyAsync(grad, m->g.p, m->np * sizeof(float), cudaMemcpyDeviceToDevice, st));
    MCUDA(cudaGetLastError());
    return LENSED_OK;
}

extern "C" int lensed_mlp_train_step(lensed_mlp *m, const float *X, const float *t, int B,
                                     float lr, float *loss, void *stream)
{
    if (!m || !X || !t || !loss) return mfail(LENSED_E_ARG, "NULL argument");
    if (B < 1 || B > m->maxB) return mfail(LENSED_E_ARG, "B = %d (1..%d)", B, m->maxB);
    if (!(lr > 0.f)) return mfail(LENSED_E_ARG, "lr must be > 0");
    cudaStream_t st = (cudaStream_t)stream;
    gradient(m, X, t, B, loss, st);
    m->step += 1;
    const float c1 = 1.f - powf(0.9f, (float)m->step), c2 = 1.f - powf(0.999f, (float)m->step);
    k_adam<<<(unsigned)((m->np + 255) / 256), 256, 0, st>>>(m->p.p, m->g.p, m->m.p, m->v.p,
                                                            (int)m->np, lr, c1, c2);
    const int n = std::max(m->H * m->kin, m->H * m->H);
    k_refresh<<<(n + 255) / 256, 256, 0, st>>>(m->p.p, m->n_in, m->kin, m->H, m->W1b.p, m->W2b.p,
                                                m->W3b.p);
    MCUDA(cudaGetLastError());
    return LENSED_OK;
}

extern "C" int lensed_mlp_screen_ellipsoid(lensed_mlp *m, int d, int n, unsigned long long seed,
                                           unsigned long long first, const float *center,
                                           const float *chol, const float *shift,
                                           const float *x_center, const float *x_whiten,
                                           float y_cut, double *u_out, int *idx_out, int *n_out,
                                           void *stream)
{
    if (d < 1 || d > kMaxScreenDim) return mfail(LENSED_E_ARG, "d = %d (1..%d)", d, kMaxScreenDim);
    if (n < 0) return mfail(LENSED_E_ARG, "n = %d", n);
    if (!center || !chol || !u_out || !idx_out || !n_out) return mfail(LENSED_E_ARG, "NULL argument");
    if (m && (m->n_in != d || !x_center || !x_whiten))
        return mfail(LENSED_E_ARG, "the network takes %d inputs and needs x_center, x_whiten",
                     m->n_in);
    cudaStream_t st = (cudaStream_t)stream;
    MCUDA(cudaMemsetAsync(n_out, 0, sizeof(int), st));
    if (n == 0) return LENSED_OK;
    const int threads = 128, blocks = (n + threads - 1) / threads;
    if (!m) {
        k_ell_select<<<blocks, threads, 0, st>>>(d, n, seed, first, center, chol, shift, nullptr,
                                                 nullptr, 0.f, u_out, idx_out, n_out);
        MCUDA(cudaGetLastError());
        return LENSED_OK;
    }
    if (m->sy.n < (size_t)n) {
        MCUDA(cudaStreamSynchronize(st));
        int rc;
        if ((rc = m->sX.alloc((size_t)n * d)) || (rc = m->sy.alloc(n)) || (rc = m->sin.alloc(n)))
            return rc;
    }
    k_ell_draw<<<blocks, threads, 0, st>>>(d, n, seed, first, center, chol, shift, x_center,
                                           x_whiten, m->sX.p, m->sin.p);
    for (int b0 = 0; b0 < n; b0 += m->maxB) {
        const int nb = std::min(m->maxB, n - b0);
        forward(m, m->sX.p + (size_t)b0 * d, nb, m->sy.p + b0, false, st);
    }
    k_ell_select<<<blocks, threads, 0, st>>>(d, n, seed, first, center, chol, shift, m->sin.p,
                                             m->sy.p, y_cut, u_out, idx_out, n_out);
    MCUDA(cudaGetLastError());
    return LENSED_OK;
}
