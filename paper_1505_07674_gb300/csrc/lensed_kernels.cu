// Device kernels of the ray-tracing likelihood (sm_103a).
//
//   k_prologue  a1: per (system, point): resolve the free/fixed parameters,
//               check the domain, precompute per-component constants
//               (Sersic b_n by Newton on the incomplete gamma function, I_0
//               from the magnitude, PA cosines, SIE prefactors) in FP64 and
//               store FP32 and FP64 copies.
//   k_trace     a2-a5: one thread per needed pixel; for every ray of the
//               quadrature rule: ray position (Eq. 14), deflection (Eq. 1),
//               brightness at image and traced position (Eq. 2), weighted
//               sum into the pixel luminosity (Eq. 3), all in registers.
//   k_psf       a6-a7: a 64 x 32 output tile per block staged in shared
//               memory with its clamped halo (Eq. 15), 8 outputs per thread
//               with the PSF row and the image row segment held in
//               registers; then the masked chi^2 of the tile (Eq. 17) as a
//               warp-shuffle tree in FP64, or the convolved image.
//   k_finalize  a7: loglike = -1/2 sum of the tile partials, fixed order.
#include <math.h>

#include <utility>

#include "lensed_internal.cuh"

namespace lensed {

// ---------------------------------------------------------------------------
// math helpers

// MUFU base-2 exponential and logarithm (PTX ex2.approx / lg2.approx, flush
// to zero): used for the Sersic and Gaussian profiles in FP32.
__device__ __forceinline__ float ex2f(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float lg2f(float x)
{
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

template <typename T>
struct Math;
template <>
struct Math<float> {
    static __device__ __forceinline__ float sqrt_(float x) { return sqrtf(x); }
    static __device__ __forceinline__ float atan_(float x) { return atanf(x); }
    static __device__ __forceinline__ float atanh_(float x) { return atanhf(x); }
    static __device__ __forceinline__ float exp2_(float x) { return ex2f(x); }
    static __device__ __forceinline__ float log2_(float x) { return lg2f(x); }
};
template <>
struct Math<double> {
    static __device__ __forceinline__ double sqrt_(double x) { return sqrt(x); }
    static __device__ __forceinline__ double atan_(double x) { return atan(x); }
    static __device__ __forceinline__ double atanh_(double x) { return atanh(x); }
    static __device__ __forceinline__ double exp2_(double x) { return exp2(x); }
    static __device__ __forceinline__ double log2_(double x) { return log2(x); }
};

// ---------------------------------------------------------------------------
// a1: parameter prologue

// Regularised lower incomplete gamma P(a, x) by its power series.
__device__ double lower_gamma_p(double a, double x)
{
    if (x <= 0.0) return 0.0;
    double term = 1.0, sum = 1.0;
    for (int k = 1; k < 5000; ++k) {
        term *= x / (a + k);
        sum += term;
        if (term < 1e-17 * sum) break;
    }
    return exp(a * log(x) - x - lgamma(a + 1.0)) * sum;
}

// Sersic b_n: root of P(2n, b) = 1/2.  Newton from the Ciotti & Bertin
// (1999) asymptotic expansion, safeguarded by the bracket [0, 2n].
__device__ double sersic_b(double n)
{
    const double a = 2.0 * n;
    double lo = 0.0, hi = a;
    double b = a - 1.0 / 3.0 + 4.0 / (405.0 * n) + 46.0 / (25515.0 * n * n) +
               131.0 / (1148175.0 * n * n * n);
    if (!(b > lo && b < hi)) b = 0.5 * (lo + hi);
    const double lga = lgamma(a);
    for (int it = 0; it < 200; ++it) {
        double f = lower_gamma_p(a, b) - 0.5;
        if (f == 0.0) break;
        if (f < 0.0) lo = b;
        else hi = b;
        double df = exp((a - 1.0) * log(b) - b - lga);
        double nb = b - f / df;
        if (!(nb > lo && nb < hi)) nb = 0.5 * (lo + hi);
        if (fabs(nb - b) <= 4e-16 * b) { b = nb; break; }
        b = nb;
    }
    return b;
}

__global__ void k_prologue(const SysDev *__restrict__ sys, int s0, int nS,
                           const int *__restrict__ comp_type, const int *__restrict__ comp_free,
                           const double *__restrict__ comp_value,
                           const double *__restrict__ params, int single_row, int P, int p0,
                           int nP,
                           int n_par_stride, int C_total, float *__restrict__ cf,
                           double *__restrict__ cd, unsigned char *__restrict__ valid)
{
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (tid >= (long long)nS * nP) return;
    const int s = s0 + (int)(tid / nP);
    const int p = p0 + (int)(tid % nP);
    const SysDev S = sys[s];
    const double *row = single_row ? params : params + ((size_t)s * P + p) * n_par_stride;
    bool ok = true;
    for (int c = 0; c < S.ncomp; ++c) {
        const int gc = S.comp_off + c;
        const int type = comp_type[gc];
        double v[LENSED_MAX_COMPONENT_PARAMS];
        for (int k = 0; k < LENSED_MAX_COMPONENT_PARAMS; ++k) {
            const int fi = comp_free[gc * LENSED_MAX_COMPONENT_PARAMS + k];
            v[k] = fi >= 0 ? row[fi] : comp_value[gc * LENSED_MAX_COMPONENT_PARAMS + k];
        }
        double o[kNC];
        for (int k = 0; k < kNC; ++k) o[k] = 0.0;
        int np = 0;
        switch (type) {
        case LENSED_SIE: np = 6; break;
        case LENSED_SHEAR: np = 4; break;
        case LENSED_POINTMASS: np = 3; break;
        case LENSED_SERSIC: np = 7; break;
        default: np = 6; break;
        }
        for (int k = 0; k < np; ++k) ok = ok && isfinite(v[k]);
        o[0] = v[0];
        o[1] = v[1];
        if (type == LENSED_SIE) {
            const double b = v[2], q = v[3], sc = v[5];
            ok = ok && q > 0.0 && q <= 1.0 && b >= 0.0 && sc >= 0.0;
            double sn, cs;
            sincospi(v[4] / 180.0, &sn, &cs);
            const double e = sqrt((1.0 - q) * (1.0 + q));
            const bool series = e < kSeriesE;
            o[2] = cs;
            o[3] = sn;
            o[4] = q * q;
            o[5] = sc * sc;
            o[6] = sc;
            o[7] = q * q * sc;
            o[8] = e;
            o[9] = series ? b * sqrt(q) : b * sqrt(q) / e;
            o[10] = series ? 1.0 : 0.0;
            o[11] = e * e;
            o[12] = e < kMixedRoundE ? 1.0 : 0.0;
            o[13] = kMixedCoreFactor * sc;
        } else if (type == LENSED_SHEAR) {
            double sn, cs;
            sincospi(v[3] / 90.0, &sn, &cs);  // 2 phi
            o[2] = v[2] * cs;
            o[3] = v[2] * sn;
        } else if (type == LENSED_POINTMASS) {
            ok = ok && v[2] >= 0.0;
            o[2] = v[2] * v[2];
        } else {
            // light: Sersic (x y r mag n q pa), de Vaucouleurs (x y r mag q pa),
            // Gaussian (x y sigma mag q pa)
            const double r = v[2];
            const double F = pow(10.0, -0.4 * (v[3] - S.zeropoint));
            double n = 4.0, q, pa;
            if (type == LENSED_SERSIC) { n = v[4]; q = v[5]; pa = v[6]; }
            else { q = v[4]; pa = v[5]; }
            ok = ok && r > 0.0 && n > 0.0 && q > 0.0 && q <= 1.0;
            double sn, cs;
            sincospi(pa / 180.0, &sn, &cs);
            o[2] = cs;
            o[3] = sn;
            o[4] = q;
            o[5] = 1.0 / q;
            if (ok && type == LENSED_GAUSS) {
                o[6] = 1.0;
                o[7] = 1.4426950408889634 / (2.0 * r * r);  // log2(e) / (2 sigma^2)
                o[8] = F / (2.0 * M_PI * r * r) * S.hd * S.hd;
                o[9] = kKindGauss;
            } else if (ok) {
                const double bn = sersic_b(n);
                // I_0 = F b^(2n) / (2 pi n r^2 Gamma(2n)), in logs
                const double lI0 = log(F) + 2.0 * n * log(bn) - log(2.0 * M_PI * n * r * r) -
                                   lgamma(2.0 * n);
                o[6] = 0.5 / n;
                o[7] = log2(bn) + log2(1.4426950408889634) - log2(r) / n;
                o[8] = exp(lI0) * S.hd * S.hd;
                o[9] = kKindPower;
            }
        }
        const size_t base = ((size_t)p * C_total + gc) * kNC;
        for (int k = 0; k < kNC; ++k) {
            cd[base + k] = o[k];
            cf[base + k] = (float)o[k];
        }
    }
    valid[(size_t)s * P + p] = ok ? 1 : 0;
}

void launch_prologue(const SysDev *sys, int s0, int nS, const int *comp_type,
                     const int *comp_free, const double *comp_value, const double *params,
                     bool single_row, int P, int p0, int nP, int n_par_stride, int C_total,
                     float *cf, double *cd, unsigned char *valid, cudaStream_t st)
{
    const long long n = (long long)nS * nP;
    const int threads = 128;
    const unsigned blocks = (unsigned)((n + threads - 1) / threads);
    k_prologue<<<blocks, threads, 0, st>>>(sys, s0, nS, comp_type, comp_free, comp_value, params,
                                           single_row ? 1 : 0, P, p0, nP, n_par_stride, C_total,
                                           cf, cd, valid);
}

// ---------------------------------------------------------------------------
// a3: deflection; a4: brightness

// SIE with core (geometric-mean convention) in precision T.  c: packed
// constants x0 y0 cos sin q^2 s^2 s q^2s e pref series e^2.
template <typename T>
__device__ __forceinline__ void sie_deflect(T x, T y, const T *c, T &ax, T &ay)
{
    const T dx = x - c[0], dy = y - c[1];
    const T u = dx * c[2] + dy * c[3];
    const T v = dy * c[2] - dx * c[3];
    const T psi = Math<T>::sqrt_(c[4] * (c[5] + u * u) + v * v);
    const T zu = u / (psi + c[6]);
    const T zv = v / (psi + c[7]);
    T au, av;
    if (c[10] != T(0)) {
        // atan(e z)/e and atanh(e z)/e to O(e^4)
        const T e2 = c[11];
        const T zu2 = zu * zu, zv2 = zv * zv;
        au = c[9] * zu * (T(1) - e2 * zu2 * (T(1) / T(3)) + e2 * e2 * zu2 * zu2 * (T(1) / T(5)));
        av = c[9] * zv * (T(1) + e2 * zv2 * (T(1) / T(3)) + e2 * e2 * zv2 * zv2 * (T(1) / T(5)));
    } else {
        au = c[9] * Math<T>::atan_(c[8] * zu);
        av = c[9] * Math<T>::atanh_(c[8] * zv);
    }
    ax += au * c[2] - av * c[3];
    ay += au * c[3] + av * c[2];
}

// Light profile in precision T.  c: x0 y0 cos sin q 1/q p2 lc|k A kind.
template <typename T>
__device__ __forceinline__ T light(T x, T y, const T *c)
{
    const T dx = x - c[0], dy = y - c[1];
    const T u = dx * c[2] + dy * c[3];
    const T v = dy * c[2] - dx * c[3];
    const T R2 = c[4] * u * u + c[5] * v * v;
    T t;
    if (c[9] == T(kKindGauss)) t = c[7] * R2;
    else t = Math<T>::exp2_(c[6] * Math<T>::log2_(R2) + c[7]);
    return c[8] * Math<T>::exp2_(-t);
}

// Total image-plane brightness at one ray (Eqs. 1-2).  MODE selects the
// precision; in MIXED the SIE switches to FP64 near q = 1 and near its core,
// with the FP64 ray position rebuilt from the pixel and node indices.
struct RayCtx {
    int ncomp;
    const int *type;
    const int *plane;
    const float *cf;
    const double *cd;
    double xd, yd;  // FP64 ray position (MIXED branch only; filled lazily)
};

template <int MODE>
__device__ __forceinline__ float brightness_f32(float x, float y, const RayCtx &R, int j, int i,
                                                double ud, double vd, double cxd, double cyd,
                                                double hd)
{
    float I = 0.f, ax = 0.f, ay = 0.f;
    for (int c = 0; c < R.ncomp; ++c) {
        const int pl = R.plane[c];
        const float *cc = R.cf + c * kNC;
        if (pl == LENSED_PLANE_FOREGROUND) {
            I += light<float>(x, y, cc);
        } else if (pl == LENSED_PLANE_LENS) {
            const int t = R.type[c];
            if (t == LENSED_SIE) {
                if (MODE == LENSED_PREC_MIXED) {
                    bool use64 = cc[12] != 0.f;
                    if (!use64) {
                        const float dx = x - cc[0], dy = y - cc[1];
                        const float u = dx * cc[2] + dy * cc[3];
                        const float v = dy * cc[2] - dx * cc[3];
                        const float psi = sqrtf(cc[4] * (cc[5] + u * u) + v * v);
                        use64 = psi < cc[13];
                    }
                    if (use64) {
                        const double xd = ((double)j - cxd) * hd + ud;
                        const double yd = ((double)i - cyd) * hd + vd;
                        double dax = 0.0, day = 0.0;
                        sie_deflect<double>(xd, yd, R.cd + c * kNC, dax, day);
                        ax += (float)dax;
                        ay += (float)day;
                        continue;
                    }
                }
                sie_deflect<float>(x, y, cc, ax, ay);
            } else if (t == LENSED_SHEAR) {
                const float dx = x - cc[0], dy = y - cc[1];
                ax += cc[2] * dx + cc[3] * dy;
                ay += cc[3] * dx - cc[2] * dy;
            } else {  // point mass
                const float dx = x - cc[0], dy = y - cc[1];
                const float r2 = dx * dx + dy * dy;
                const float f = r2 > 0.f ? cc[2] / r2 : 0.f;
                ax += f * dx;
                ay += f * dy;
            }
        }
    }
    const float sx = x - ax, sy = y - ay;
    for (int c = 0; c < R.ncomp; ++c)
        if (R.plane[c] == LENSED_PLANE_SOURCE) I += light<float>(sx, sy, R.cf + c * kNC);
    return I;
}

__device__ __forceinline__ double brightness_f64(double x, double y, const RayCtx &R)
{
    double I = 0.0, ax = 0.0, ay = 0.0;
    for (int c = 0; c < R.ncomp; ++c) {
        const int pl = R.plane[c];
        const double *cc = R.cd + c * kNC;
        if (pl == LENSED_PLANE_FOREGROUND) {
            I += light<double>(x, y, cc);
        } else if (pl == LENSED_PLANE_LENS) {
            const int t = R.type[c];
            if (t == LENSED_SIE) {
                sie_deflect<double>(x, y, cc, ax, ay);
            } else if (t == LENSED_SHEAR) {
                const double dx = x - cc[0], dy = y - cc[1];
                ax += cc[2] * dx + cc[3] * dy;
                ay += cc[3] * dx - cc[2] * dy;
            } else {
                const double dx = x - cc[0], dy = y - cc[1];
                const double r2 = dx * dx + dy * dy;
                const double f = r2 > 0.0 ? cc[2] / r2 : 0.0;
                ax += f * dx;
                ay += f * dy;
            }
        }
    }
    const double sx = x - ax, sy = y - ay;
    for (int c = 0; c < R.ncomp; ++c)
        if (R.plane[c] == LENSED_PLANE_SOURCE) I += light<double>(sx, sy, R.cd + c * kNC);
    return I;
}

// ---------------------------------------------------------------------------
// a2-a5: ray tracing and pixel integration

template <int MODE, int PPT>
__global__ void __launch_bounds__(256)
    k_trace(const SysDev *__restrict__ sys, const int *__restrict__ comp_type,
            const int *__restrict__ comp_plane, const float *__restrict__ cf,
            const double *__restrict__ cd, const unsigned char *__restrict__ valid, int P,
            int C_total, const TraceBlock *__restrict__ blocks, const int *__restrict__ need,
            const float *__restrict__ node_u, const float *__restrict__ node_w,
            const double *__restrict__ node_ud, const double *__restrict__ node_wd, int p0,
            void *__restrict__ Lbuf, long long L_stride)
{
    __shared__ __align__(16) float s_cf[LENSED_MAX_COMPONENTS * kNC];
    __shared__ __align__(16) double s_cd[(MODE == LENSED_PREC_FP32) ? 1 : LENSED_MAX_COMPONENTS * kNC];
    __shared__ int s_type[LENSED_MAX_COMPONENTS], s_plane[LENSED_MAX_COMPONENTS];
    __shared__ float s_u[LENSED_MAX_RULE_ORDER], s_w[LENSED_MAX_RULE_ORDER];
    __shared__ double s_ud[LENSED_MAX_RULE_ORDER], s_wd[LENSED_MAX_RULE_ORDER];

    const TraceBlock tb = blocks[blockIdx.x];
    const int p = p0 + blockIdx.y;
    if (!valid[(size_t)tb.sys * P + p]) return;
    const SysDev &S = sys[tb.sys];
    const int ncomp = S.ncomp, nn = S.nn;
    const size_t cbase = ((size_t)p * C_total + S.comp_off) * kNC;
    for (int k = threadIdx.x; k < ncomp * kNC; k += blockDim.x) {
        s_cf[k] = cf[cbase + k];
        if (MODE != LENSED_PREC_FP32) s_cd[k] = cd[cbase + k];
    }
    for (int k = threadIdx.x; k < ncomp; k += blockDim.x) {
        s_type[k] = comp_type[S.comp_off + k];
        s_plane[k] = comp_plane[S.comp_off + k];
    }
    for (int k = threadIdx.x; k < nn; k += blockDim.x) {
        s_u[k] = node_u[S.node_off + k];
        s_w[k] = node_w[S.node_off + k];
        s_ud[k] = node_ud[S.node_off + k];
        s_wd[k] = node_wd[S.node_off + k];
    }
    __syncthreads();

    RayCtx R;
    R.ncomp = ncomp;
    R.type = s_type;
    R.plane = s_plane;
    R.cf = s_cf;
    R.cd = s_cd;
    const int nx = S.nx;
    const size_t lbase = (size_t)(p - p0) * L_stride + S.pix_off;

#pragma unroll
    for (int k = 0; k < PPT; ++k) {
        const int idx = tb.start + threadIdx.x + k * blockDim.x;
        if (idx >= tb.end) break;
        const int pix = need ? need[S.need_off + idx] : idx;
        const int i = pix / nx, j = pix - (pix / nx) * nx;
        if (MODE == LENSED_PREC_FP64) {
            const double xc = ((double)j - (double)S.cx) * S.hd;
            const double yc = ((double)i - (double)S.cy) * S.hd;
            double acc = 0.0;
            for (int b = 0; b < nn; ++b) {
                const double y = yc + s_ud[b];
                double row = 0.0;
                for (int a = 0; a < nn; ++a) row += s_wd[a] * brightness_f64(xc + s_ud[a], y, R);
                acc += s_wd[b] * row;
            }
            ((double *)Lbuf)[lbase + pix] = acc;
        } else {
            const float xc = ((float)j - S.cx) * S.h;
            const float yc = ((float)i - S.cy) * S.h;
            float acc = 0.f;
            for (int b = 0; b < nn; ++b) {
                const float y = yc + s_u[b];
                float row = 0.f;
                for (int a = 0; a < nn; ++a)
                    row += s_w[a] * brightness_f32<MODE>(xc + s_u[a], y, R, j, i, s_ud[a],
                                                         s_ud[b], (double)S.cx, (double)S.cy,
                                                         S.hd);
                acc += s_w[b] * row;
            }
            ((float *)Lbuf)[lbase + pix] = acc;
        }
    }
}

template <int MODE, int PPT>
static void trace_launch_t(int threads, const SysDev *sys, const int *comp_type,
                           const int *comp_plane, const float *cf, const double *cd,
                           const unsigned char *valid, int P, int C_total,
                           const TraceBlock *blocks, int n_blocks, const int *need,
                           NodeTables nodes, int p0, int nP, void *Lbuf, long long L_stride,
                           cudaStream_t st)
{
    dim3 grid((unsigned)n_blocks, (unsigned)nP);
    k_trace<MODE, PPT><<<grid, threads, 0, st>>>(sys, comp_type, comp_plane, cf, cd, valid, P,
                                                 C_total, blocks, need, nodes.u, nodes.w,
                                                 nodes.ud, nodes.wd, p0, Lbuf, L_stride);
}

void launch_trace(int precision, LaunchCfg cfg, const SysDev *sys, const int *comp_type,
                  const int *comp_plane, const float *cf, const double *cd,
                  const unsigned char *valid, int P, int C_total, const TraceBlock *blocks,
                  int n_blocks, const int *need, NodeTables nodes, int p0, int nP, void *Lbuf,
                  long long L_stride, cudaStream_t st)
{
    if (n_blocks <= 0 || nP <= 0) return;
#define LENSED_TRACE(M, K)                                                                    \
    trace_launch_t<M, K>(cfg.trace_threads, sys, comp_type, comp_plane, cf, cd, valid, P,    \
                         C_total, blocks, n_blocks, need, nodes, p0, nP, Lbuf, L_stride, st)
    if (precision == LENSED_PREC_FP64) {
        LENSED_TRACE(LENSED_PREC_FP64, 1);
    } else if (precision == LENSED_PREC_MIXED) {
        if (cfg.pix_per_thread == 2) LENSED_TRACE(LENSED_PREC_MIXED, 2);
        else LENSED_TRACE(LENSED_PREC_MIXED, 1);
    } else {
        if (cfg.pix_per_thread == 2) LENSED_TRACE(LENSED_PREC_FP32, 2);
        else LENSED_TRACE(LENSED_PREC_FP32, 1);
    }
#undef LENSED_TRACE
}

// ---------------------------------------------------------------------------
// a6-a7: PSF convolution and masked chi^2

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

static __host__ __device__ __forceinline__ int psf_row_stride(int q)
{
    // row of the staged tile: kTileW + 2q values, rounded up to a multiple of 4
    return (kTileW + 2 * q + 3) & ~3;
}

template <typename T, int Q>
__global__ void __launch_bounds__(kPsfThreads)
    k_psf(const SysDev *__restrict__ sys, const T *__restrict__ psf,
          const T *__restrict__ data, const T *__restrict__ weight,
          const unsigned char *__restrict__ valid, int P, const PsfBlock *__restrict__ blocks,
          int p0, const T *__restrict__ Lbuf, long long L_stride, double *__restrict__ partial,
          int T_total, float *__restrict__ out)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *s_L = reinterpret_cast<T *>(smem_raw);
    constexpr int W = 2 * Q + 1;
    const PsfBlock pb = blocks[blockIdx.x];
    const int p = p0 + blockIdx.y;
    const SysDev &S = sys[pb.sys];
    const bool ok = valid[(size_t)pb.sys * P + p] != 0;
    const int Ph = S.psf_p;
    const int rows = kTileH + 2 * Ph;
    const int stride = psf_row_stride(Q);
    T *s_F = s_L + (size_t)rows * stride;
    const int nx = S.nx, ny = S.ny;

    if (!ok) {
        // Outside the domain: the partial is unused; the rendered image is NaN.
        if (out) {
            for (int k = threadIdx.x; k < kTileW * kTileH; k += blockDim.x) {
                const int i = pb.i0 + k / kTileW, j = pb.j0 + k % kTileW;
                if (i < ny && j < nx) out[(size_t)i * nx + j] = __int_as_float(0x7fc00000);
            }
        }
        return;
    }

    // stage the flipped, normalised PSF and the clamped tile + halo
    for (int k = threadIdx.x; k < (2 * Ph + 1) * W; k += blockDim.x) s_F[k] = psf[S.psf_off + k];
    const T *L = Lbuf + (size_t)(p - p0) * L_stride + S.pix_off;
    const int cols = kTileW + 2 * Q;
    for (int k = threadIdx.x; k < rows * cols; k += blockDim.x) {
        const int r = k / cols, c = k - (k / cols) * cols;
        const int gi = min(max(pb.i0 - Ph + r, 0), ny - 1);
        const int gj = min(max(pb.j0 - Q + c, 0), nx - 1);
        s_L[r * stride + c] = L[(size_t)gi * nx + gj];
    }
    __syncthreads();

    const int tc = threadIdx.x % (kTileW / kOutPerThread);
    const int tr = threadIdx.x / (kTileW / kOutPerThread);
    T acc[kOutPerThread];
#pragma unroll
    for (int o = 0; o < kOutPerThread; ++o) acc[o] = T(0);
    for (int kk = 0; kk <= 2 * Ph; ++kk) {
        T f[W];
#pragma unroll
        for (int l = 0; l < W; ++l) f[l] = s_F[kk * W + l];
        const T *srow = s_L + (tr + kk) * stride + tc * kOutPerThread;
        T lv[kOutPerThread + 2 * Q];
#pragma unroll
        for (int m = 0; m < kOutPerThread + 2 * Q; ++m) lv[m] = srow[m];
#pragma unroll
        for (int o = 0; o < kOutPerThread; ++o)
#pragma unroll
            for (int l = 0; l < W; ++l) acc[o] += f[l] * lv[o + l];
    }

    const int i = pb.i0 + tr;
    const int jb = pb.j0 + tc * kOutPerThread;
    if (partial) {
        double chi = 0.0;
        if (i < ny) {
#pragma unroll
            for (int o = 0; o < kOutPerThread; ++o) {
                const int j = jb + o;
                if (j < nx) {
                    const size_t pix = S.pix_off + (size_t)i * nx + j;
                    const T w = weight[pix];
                    if (w > T(0)) {
                        const T r = data[pix] - acc[o];
                        chi += (double)w * ((double)r * (double)r);
                    }
                }
            }
        }
        // warp-shuffle tree, then across the 8 warps in fixed order
        __shared__ double s_red[kPsfThreads / 32];
        chi = warp_sum(chi);
        if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = chi;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int w = 0; w < kPsfThreads / 32; ++w) t += s_red[w];
            partial[(size_t)p * T_total + pb.tile] = t;
        }
    } else if (out && i < ny) {
#pragma unroll
        for (int o = 0; o < kOutPerThread; ++o) {
            const int j = jb + o;
            if (j < nx) out[(size_t)i * nx + j] = (float)acc[o];
        }
    }
}

template <typename T, int Q>
static void psf_launch_t(int p_max, const SysDev *sys, const T *psf, const T *data,
                         const T *weight, const unsigned char *valid, int P,
                         const PsfBlock *blocks, int n_blocks, int p0, int nP, const T *Lbuf,
                         long long L_stride, double *partial, int T_total, float *out,
                         cudaStream_t st)
{
    const size_t smem = ((size_t)(kTileH + 2 * p_max) * psf_row_stride(Q) +
                         (size_t)(2 * p_max + 1) * (2 * Q + 1)) * sizeof(T);
    dim3 grid((unsigned)n_blocks, (unsigned)nP);
    k_psf<T, Q><<<grid, kPsfThreads, smem, st>>>(sys, psf, data, weight, valid, P, blocks, p0,
                                                  Lbuf, L_stride, partial, T_total, out);
}

// Largest dynamic shared memory a k_psf instance can ask for (Q = P = 15, FP64).
static constexpr int kPsfSmemMax =
    ((kTileH + 2 * LENSED_MAX_PSF_HALF) * ((kTileW + 2 * LENSED_MAX_PSF_HALF + 3) & ~3) +
     (2 * LENSED_MAX_PSF_HALF + 1) * (2 * LENSED_MAX_PSF_HALF + 1)) * (int)sizeof(double);

template <typename T, int Q>
static void psf_attr_t()
{
    cudaFuncSetAttribute(k_psf<T, Q>, cudaFuncAttributeMaxDynamicSharedMemorySize, kPsfSmemMax);
}

template <typename T, int... Qs>
static void psf_attr_all(std::integer_sequence<int, Qs...>)
{
    (psf_attr_t<T, Qs>(), ...);
}

void init_kernel_attributes()
{
    psf_attr_all<float>(std::make_integer_sequence<int, LENSED_MAX_PSF_HALF + 1>{});
    psf_attr_all<double>(std::make_integer_sequence<int, LENSED_MAX_PSF_HALF + 1>{});
}

template <typename T>
static void psf_dispatch(int q, int p_max, const SysDev *sys, const T *psf, const T *data,
                         const T *weight, const unsigned char *valid, int P,
                         const PsfBlock *blocks, int n_blocks, int p0, int nP, const T *Lbuf,
                         long long L_stride, double *partial, int T_total, float *out,
                         cudaStream_t st)
{
#define LENSED_PSF_CASE(QQ)                                                                  \
    case QQ:                                                                                 \
        psf_launch_t<T, QQ>(p_max, sys, psf, data, weight, valid, P, blocks, n_blocks, p0,  \
                            nP, Lbuf, L_stride, partial, T_total, out, st);                  \
        break;
    switch (q) {
        LENSED_PSF_CASE(0)
        LENSED_PSF_CASE(1)
        LENSED_PSF_CASE(2)
        LENSED_PSF_CASE(3)
        LENSED_PSF_CASE(4)
        LENSED_PSF_CASE(5)
        LENSED_PSF_CASE(6)
        LENSED_PSF_CASE(7)
        LENSED_PSF_CASE(8)
        LENSED_PSF_CASE(9)
        LENSED_PSF_CASE(10)
        LENSED_PSF_CASE(11)
        LENSED_PSF_CASE(12)
        LENSED_PSF_CASE(13)
        LENSED_PSF_CASE(14)
        LENSED_PSF_CASE(15)
    default: break;
    }
#undef LENSED_PSF_CASE
}

void launch_psf(int precision, int q, int p_max, const SysDev *sys, const float *psf_f,
                const double *psf_d, const float *data, const float *weight,
                const double *data_d, const double *weight_d,
                const unsigned char *valid, int P, const PsfBlock *blocks, int n_blocks, int p0,
                int nP, const void *Lbuf, long long L_stride, double *partial, int T_total,
                float *out, cudaStream_t st)
{
    if (n_blocks <= 0 || nP <= 0) return;
    if (precision == LENSED_PREC_FP64)
        psf_dispatch<double>(q, p_max, sys, psf_d, data_d, weight_d, valid, P, blocks, n_blocks, p0,
                             nP, (const double *)Lbuf, L_stride, partial, T_total, out, st);
    else
        psf_dispatch<float>(q, p_max, sys, psf_f, data, weight, valid, P, blocks, n_blocks, p0,
                            nP, (const float *)Lbuf, L_stride, partial, T_total, out, st);
}

// ---------------------------------------------------------------------------
// a7: final reduction

__global__ void k_finalize(const SysDev *__restrict__ sys, const unsigned char *__restrict__ valid,
                           int P, const double *__restrict__ partial, int T_total,
                           double *__restrict__ out, int s0, int p0, int nS, int nP)
{
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (tid >= (long long)nS * nP) return;
    const int s = s0 + (int)(tid / nP);
    const int p = p0 + (int)(tid % nP);
    const SysDev &S = sys[s];
    double v;
    if (!valid[(size_t)s * P + p]) {
        v = -INFINITY;
    } else {
        double t = 0.0;
        const double *row = partial + (size_t)p * T_total + S.tile_off;
        for (int k = 0; k < S.n_tiles; ++k) t += row[k];
        v = -0.5 * t;
    }
    out[(size_t)s * P + p] = v;
}

void launch_finalize(const SysDev *sys, const unsigned char *valid, int P,
                     const double *partial, int T_total, double *out, int s0, int p0, int nS,
                     int nP, cudaStream_t st)
{
    const long long n = (long long)nS * nP;
    const int threads = 128;
    k_finalize<<<(unsigned)((n + threads - 1) / threads), threads, 0, st>>>(
        sys, valid, P, partial, T_total, out, s0, p0, nS, nP);
}

__global__ void k_copy_image(int fp64, const void *__restrict__ Lbuf, long long off, int npix,
                             const unsigned char *__restrict__ valid, float *__restrict__ out)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= npix) return;
    if (!valid[0]) {
        out[k] = __int_as_float(0x7fc00000);
        return;
    }
    out[k] = fp64 ? (float)((const double *)Lbuf)[off + k] : ((const float *)Lbuf)[off + k];
}

void launch_copy_image(int precision, const void *Lbuf, long long off, int npix,
                       const unsigned char *valid, float *out, cudaStream_t st)
{
    k_copy_image<<<(npix + 255) / 256, 256, 0, st>>>(precision == LENSED_PREC_FP64, Lbuf, off,
                                                      npix, valid, out);
}

}  // namespace lensed
