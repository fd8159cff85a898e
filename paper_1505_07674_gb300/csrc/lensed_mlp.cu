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
              int *__restrict__ err, int spin)
{
    extern __shared__ __align__(128) unsigned char g_smem[];
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

// out[n] = sum_m in[m][n] (fixed order), fp32 in
__global__ void k_colsum(const float *__restrict__ in, int M, int N, float *__restrict__ out)
{
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    float s = 0.f;
    for (int m = 0; m < M; ++m) s += in[(size_t)m * N + n];
    out[n] = s;
}

// dw4[k] = sum_m h3[m][k] dy[m]
__global__ void k_dw4(const bf16 *__restrict__ H3, const float *__restrict__ dy, int Bp, int H,
                      float *__restrict__ dw4)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= H) return;
    float s = 0.f;
    for (int m = 0; m < Bp; ++m) s += __bfloat162float(H3[(size_t)m * H + k]) * dy[m];
    dw4[k] = s;
}

__global__ void k_sum(const float *__restrict__ in, int n, float *__restrict__ out)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    float s = 0.f;
    for (int i = 0; i < n; ++i) s += in[i];
    out[0] = s;
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
    Buf<int> err;  // set by a tensor-core wait that expired
    int spin = kSpinLimit;  // poll limit of the GEMM pipeline waits
};

namespace {

int launch_gemm(int epi, const bf16 *A, int lda, const bf16 *B, int ldb, int M, int N, int K,
                float *Cf, int ldc, const float *bias, const float *Zin, float *Zout, bf16 *Hout,
                int *err, cudaStream_t st, int spin = kSpinLimit)
{
    dim3 grid((N + TN - 1) / TN, (M + TM - 1) / TM);
    if (epi == EPI_F32)
        k_gemm_tc<EPI_F32><<<grid, 128, kGemmSmem, st>>>(A, lda, B, ldb, M, N, K, Cf, ldc, bias,
                                                         Zin, Zout, Hout, err, spin);
    else if (epi == EPI_BIAS_SILU)
        k_gemm_tc<EPI_BIAS_SILU><<<grid, 128, kGemmSmem, st>>>(A, lda, B, ldb, M, N, K, Cf, ldc,
                                                               bias, Zin, Zout, Hout, err, spin);
    else
        k_gemm_tc<EPI_DSILU><<<grid, 128, kGemmSmem, st>>>(A, lda, B, ldb, M, N, K, Cf, ldc, bias,
                                                           Zin, Zout, Hout, err, spin);
    return LENSED_OK;
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
    k_sum<<<1, 32, 0, st>>>(m->lossrow.p, Bp, loss);
    k_dw4<<<(H + 127) / 128, 128, 0, st>>>(m->H3.p, m->dy.p, Bp, H, g + m->o_w4);
    k_sum<<<1, 32, 0, st>>>(m->dy.p, Bp, g + m->o_b4);
    // layer 3: dW3 = dZ3^T H2, db3, dZ2 = (dZ3 W3) * silu'(Z2)
    transpose(m->dZa.p, Bp, H, m->dZT.p, st);
    transpose(m->H2.p, Bp, H, m->HT.p, st);
    launch_gemm(EPI_F32, m->dZT.p, Bp, m->HT.p, Bp, H, H, Bp, g + m->o_W3, H, nullptr, nullptr,
                nullptr, nullptr, m->err.p, st, m->spin);
    k_colsum<<<(H + 127) / 128, 128, 0, st>>>(m->dZf.p, Bp, H, g + m->o_b3);
    transpose(m->W3b.p, H, H, m->WT.p, st);
    launch_gemm(EPI_DSILU, m->dZa.p, H, m->WT.p, H, Bp, H, H, nullptr, H, nullptr, m->Z2.p,
                m->dZf.p, m->dZbuf.p, m->err.p, st, m->spin);
    // layer 2
    transpose(m->dZbuf.p, Bp, H, m->dZT.p, st);
    transpose(m->H1.p, Bp, H, m->HT.p, st);
    launch_gemm(EPI_F32, m->dZT.p, Bp, m->HT.p, Bp, H, H, Bp, g + m->o_W2, H, nullptr, nullptr,
                nullptr, nullptr, m->err.p, st, m->spin);
    k_colsum<<<(H + 127) / 128, 128, 0, st>>>(m->dZf.p, Bp, H, g + m->o_b2);
    transpose(m->W2b.p, H, H, m->WT.p, st);
    launch_gemm(EPI_DSILU, m->dZbuf.p, H, m->WT.p, H, Bp, H, H, nullptr, H, nullptr, m->Z1.p,
                m->dZf.p, m->dZa.p, m->err.p, st, m->spin);
    // layer 1: dW1 = dZ1^T X (padded to kin columns), db1
    transpose(m->dZa.p, Bp, H, m->dZT.p, st);
    transpose(m->Xb.p, Bp, m->kin, m->XbT.p, st);
    launch_gemm(EPI_F32, m->dZT.p, Bp, m->XbT.p, Bp, H, m->kin, Bp, m->gW1.p, m->kin, nullptr,
                nullptr, nullptr, nullptr, m->err.p, st, m->spin);
    k_copy_cols<<<(H * m->n_in + 255) / 256, 256, 0, st>>>(m->gW1.p, H, m->kin, m->n_in, g);
    k_colsum<<<(H + 127) / 128, 128, 0, st>>>(m->dZf.p, Bp, H, g + m->o_b1);
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
        (rc = m->gW1.alloc(H * m->kin)) || (rc = m->tmpcol.alloc(H)) || (rc = m->err.alloc(1))) {
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
