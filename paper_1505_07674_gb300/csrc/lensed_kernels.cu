// Device kernels of the ray-tracing likelihood (sm_103a).
//
//   k_prologue_comp / k_prologue_valid
//               a1: per (point, component): resolve the free/fixed
//               parameters, check the domain, precompute the constants
//               (Sersic b_n from a Chebyshev table in log n with a Newton
//               fallback on the incomplete gamma function, I_0 from the
//               magnitude, PA cosines, SIE prefactors) in FP64 with FP32
//               copies; per (system, point): validity, and the image-plane
//               priors (a source moved to theta - alpha(theta)).
//   k_trace_rows, k_trace_rows_pq
//               a2-a5: one thread per needed pixel; for every ray of the
//               quadrature rule: ray position (Eq. 14), deflection (Eq. 1),
//               brightness at image and traced position (Eq. 2), weighted
//               sum into the pixel luminosity (Eq. 3), in registers, starting
//               from the once-per-model integral of the fixed lights.  The
//               rays of a node row are traced in pairs with packed FP32
//               instructions (lensed_vec2.cuh).  _pq: the same work as a
//               persistent grid taking (trace block, point) items from a
//               counter.  MIXED_FF re-traces the rays near a source centre
//               in float-float, inside the block (a block-wide queue) or in
//               a second pass:
//   k_refine_ff, k_retrace_ff, k_apply_ff
//               the flagged pixels recomputed with their near rays queued,
//               the queued rays re-traced, and added in ray order.
//   k_trace_fix64, k_trace_f64
//               MIXED: the pixels the FP64 SIE rule reaches; FP64 mode.
//   k_psf, k_psf_sep
//               a6-a7: a 64 x 32 output tile per block staged in shared
//               memory with its clamped halo (Eq. 15), 8 outputs per thread
//               with the PSF row and the image row segment held in
//               registers (or, for a PSF of rank <= 3, a row pass and a
//               column pass per separable term); then the masked chi^2 of the
//               tile (Eq. 17) as a warp-shuffle tree in FP64, or the image.
//   k_finalize  a7: loglike = -1/2 sum of the tile partials, fixed order.
//   k_error_image
//               the Gauss-Kronrod error estimate |L_K - L_G| of a render.
#include <math.h>

#include <algorithm>
#include <type_traits>
#include <utility>

#include "lensed_internal.cuh"
#include "lensed_sie_trig.cuh"

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

// ---------------------------------------------------------------------------
// a1: parameter prologue

// Regularised lower incomplete gamma P(a, x) by its power series
//   P(a, x) = x^a e^-x / Gamma(a+1) * sum_k x^k / ((a+1)...(a+k)),
// summed as one fraction N / D (D the running product of (a+j), N the
// matching numerator) so the loop has no division; lg_a1 = lgamma(a + 1).
__device__ double lower_gamma_p(double a, double x, double lg_a1)
{
    if (x <= 0.0) return 0.0;
    double N = 1.0, D = 1.0, xk = 1.0;
    for (int k = 1; k < 400; ++k) {
        const double f = a + k;
        xk *= x;
        N = N * f + xk;
        D *= f;
        if (xk < 1e-17 * N) break;
        if (D > 1e250) {  // rescale before the product overflows
            N *= 1e-250;
            D *= 1e-250;
            xk *= 1e-250;
        }
    }
    return exp(a * log(x) - x - lg_a1) * (N / D);
}

// Sersic b_n: root of P(2n, b) = 1/2.  Newton from the Ciotti & Bertin
// (1999) asymptotic expansion, safeguarded by the bracket [0, 2n].
__device__ double sersic_b(double n)
{
    const double a = 2.0 * n;
    double lo = 0.0, hi = a;
    double b = a - 1.0 / 3.0 + 4.0 / (405.0 * n) + 46.0 / (25515.0 * n * n) +
               131.0 / (1148175.0 * n * n * n) - 2194697.0 / (30690717750.0 * n * n * n * n);
    if (!(b > lo && b < hi)) b = 0.5 * (lo + hi);
    const double lga = lgamma(a), lga1 = lga + log(a);
    for (int it = 0; it < 100; ++it) {
        double f = lower_gamma_p(a, b, lga1) - 0.5;
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

// b_n from the Chebyshev table when n lies in its range, else by Newton.
__device__ double sersic_b_lookup(double n, const double *__restrict__ table)
{
    if (table && n >= kBnMin && n <= kBnMax) {
        const double l0 = log(kBnMin), dl = (log(kBnMax) - l0) / kBnSeg;
        const double ln = log(n);
        const int k = min(max((int)((ln - l0) / dl), 0), kBnSeg - 1);
        const double lo = l0 + k * dl;
        const double t = (2.0 * (ln - lo) - dl) / dl;  // [-1, 1]
        const double *c = table + k * (kBnDeg + 1);
        // Clenshaw
        double b1 = 0.0, b2 = 0.0;
        for (int j = kBnDeg; j >= 1; --j) {
            const double b0 = 2.0 * t * b1 - b2 + c[j];
            b2 = b1;
            b1 = b0;
        }
        return t * b1 - b2 + c[0];
    }
    return sersic_b(n);
}

// One thread per (point, component): resolve the component's parameters,
// check its domain and write its packed constants and a validity byte.
__global__ void k_prologue_comp(const SysDev *__restrict__ sys, const int *__restrict__ comp_sys,
                                int c0, int nC, const int *__restrict__ comp_type,
                                const int *__restrict__ comp_free,
                                const double *__restrict__ comp_value,
                                const double *__restrict__ params, int single_row, int P, int p0,
                                int nP, int n_par_stride, int C_total,
                                const double *__restrict__ bn_table, float *__restrict__ cf,
                                double *__restrict__ cd, unsigned char *__restrict__ cvalid)
{
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (tid >= (long long)nC * nP) return;
    const int gc = c0 + (int)(tid % nC);
    const int p = p0 + (int)(tid / nC);
    const int s = comp_sys[gc];
    const double zeropoint = sys[s].zeropoint;
    const double hd = sys[s].hd;
    const double *row = single_row ? params : params + ((size_t)s * P + p) * n_par_stride;
    const int type = comp_type[gc];
    double v[LENSED_MAX_COMPONENT_PARAMS];
#pragma unroll
    for (int k = 0; k < LENSED_MAX_COMPONENT_PARAMS; ++k) {
        const int fi = comp_free[gc * LENSED_MAX_COMPONENT_PARAMS + k];
        v[k] = fi >= 0 ? row[fi] : comp_value[gc * LENSED_MAX_COMPONENT_PARAMS + k];
    }
    double o[kNC];
#pragma unroll
    for (int k = 0; k < kNC; ++k) o[k] = 0.0;
    // slots whose FP32 copy gets a residual partner: lo[k] = partner of k
    int lo[kNC];
#pragma unroll
    for (int k = 0; k < kNC; ++k) lo[k] = -1;
    const int np = type == LENSED_SIE ? 6 : type == LENSED_SHEAR ? 4
                 : type == LENSED_POINTMASS ? 3 : type == LENSED_SERSIC ? 7
                 : type == LENSED_SKY ? 1 : 6;
    bool ok = true;
    for (int k = 0; k < np; ++k) ok = ok && isfinite(v[k]);
    o[0] = v[0];
    o[1] = v[1];
    if (type == LENSED_SIE) {
        // 0 x0, 1 y0, 2 cos, 3 sin, 4 cos_lo, 5 sin_lo, 6 q^2, 7 q^2_lo,
        // 8 s^2, 9 s, 10 q^2 s, 11 e, 12 e_lo, 13 pref, 14 pref_lo,
        // 15 series flag, 16 e^2, 17 FP64 flag (MIXED, e < 0.05),
        // 18 (2 s / q)^2: pixels whose square comes inside this radius of
        // the lens centre take the FP64 branch in MIXED;
        // 19 x0_lo, 20 y0_lo, 21 s^2_lo, 22 s_lo, 23 q^2 s_lo (the float-float
        // re-trace reads every constant as a pair)
        const double b = v[2], q = v[3], sc = v[5];
        ok = ok && q > 0.0 && q <= 1.0 && b >= 0.0 && sc >= 0.0;
        double sn, cs;
        sincospi(v[4] / 180.0, &sn, &cs);
        const double e = sqrt((1.0 - q) * (1.0 + q));
        const bool series = e < kSeriesE;
        o[2] = cs;
        o[3] = sn;
        o[6] = q * q;
        o[8] = sc * sc;
        o[9] = sc;
        o[10] = q * q * sc;
        o[11] = e;
        o[13] = series ? b * sqrt(q) : b * sqrt(q) / e;
        o[15] = series ? 1.0 : 0.0;
        o[16] = e * e;
        o[17] = e < kMixedRoundE ? 1.0 : 0.0;
        const double rc = ok ? kMixedCoreFactor * sc / q : 0.0;
        o[18] = rc * rc;
        lo[2] = 4;
        lo[3] = 5;
        lo[6] = 7;
        lo[11] = 12;
        lo[13] = 14;
        lo[0] = 19;
        lo[1] = 20;
        lo[8] = 21;
        lo[9] = 22;
        lo[10] = 23;
    } else if (type == LENSED_SHEAR) {
        // 0 x0, 1 y0, 2 gamma_1, 3 gamma_2; 4-7 their residuals
        double sn, cs;
        sincospi(v[3] / 90.0, &sn, &cs);  // 2 phi
        o[2] = v[2] * cs;
        o[3] = v[2] * sn;
        lo[0] = 4;
        lo[1] = 5;
        lo[2] = 6;
        lo[3] = 7;
    } else if (type == LENSED_POINTMASS) {
        // 0 x0, 1 y0, 2 theta_E^2; 3-5 their residuals
        ok = ok && v[2] >= 0.0;
        o[2] = v[2] * v[2];
        lo[0] = 3;
        lo[1] = 4;
        lo[2] = 5;
    } else if (type == LENSED_SKY) {
        // flat sky (Sec. 5): 13 A = S h^2, 14 A_lo, 15 kind; no position
        o[0] = 0.0;
        o[1] = 0.0;
        o[13] = v[0] * hd * hd;
        o[15] = kKindFlat;
        lo[13] = 14;
    } else {
        // light: Sersic (x y r mag n q pa), de Vaucouleurs (x y r mag q pa),
        // Gaussian (x y sigma mag q pa).
        // 0 x0, 1 y0, 2 cos, 3 sin, 4 cos_lo, 5 sin_lo, 6 q/r^2, 7 1/(q r^2),
        // 8 q/r^2 lo, 9 1/(q r^2) lo, 10 p2, 11 B, 12 B_lo, 13 A, 14 A_lo,
        // 15 kind, 16 x0_lo, 17 y0_lo.  rho^2 = (q u^2 + v^2/q)/r^2; Sersic t = B rho^(2 p2) with
        // B = b_n log2(e), p2 = 1/(2n); Gaussian (r = sqrt(2) sigma) t =
        // B rho^2 with B = log2(e); I = A 2^-t with A = I_0 h^2.
        const double r = v[2];
        const double F = pow(10.0, -0.4 * (v[3] - zeropoint));
        double n = 4.0, q, pa;
        if (type == LENSED_SERSIC) { n = v[4]; q = v[5]; pa = v[6]; }
        else { q = v[4]; pa = v[5]; }
        ok = ok && r > 0.0 && n > 0.0 && q > 0.0 && q <= 1.0;
        double sn, cs;
        sincospi(pa / 180.0, &sn, &cs);
        o[2] = cs;
        o[3] = sn;
        lo[2] = 4;
        lo[3] = 5;
        lo[6] = 8;
        lo[7] = 9;
        lo[11] = 12;
        lo[13] = 14;
        lo[0] = 16;
        lo[1] = 17;
        if (ok && type == LENSED_GAUSS) {
            const double r2 = 2.0 * r * r;
            o[6] = q / r2;
            o[7] = 1.0 / (q * r2);
            o[10] = 1.0;
            o[11] = 1.4426950408889634;  // log2(e)
            o[13] = F / (M_PI * r2) * hd * hd;
            o[15] = kKindGauss;
        } else if (ok) {
            const double bn = sersic_b_lookup(n, bn_table);
            // I_0 = F b^(2n) / (2 pi n r^2 Gamma(2n)), in logs
            const double lI0 = log(F) + 2.0 * n * log(bn) - log(2.0 * M_PI * n * r * r) -
                               lgamma(2.0 * n);
            o[6] = q / (r * r);
            o[7] = 1.0 / (q * r * r);
            o[10] = 0.5 / n;
            o[11] = bn * 1.4426950408889634;
            o[13] = exp(lI0) * hd * hd;
            o[15] = kKindPower;
        }
    }
    const size_t base = ((size_t)p * C_total + gc) * kNC;
    float f[kNC];
#pragma unroll
    for (int k = 0; k < kNC; ++k) f[k] = (float)o[k];
#pragma unroll
    for (int k = 0; k < kNC; ++k)
        if (lo[k] >= 0) f[lo[k]] = (float)(o[k] - (double)f[k]);
#pragma unroll
    for (int k = 0; k < kNC; ++k) {
        cd[base + k] = o[k];
        cf[base + k] = f[k];
    }
    cvalid[(size_t)p * C_total + gc] = ok ? 1 : 0;
}

// ---------------------------------------------------------------------------
// a3: deflection; a4: brightness

// SIE with core (geometric-mean convention) in FP64 (constants as packed by
// the prologue; residual slots are zero in the FP64 copy).  A ray exactly at
// the centre of a coreless SIE gets no deflection.
__device__ __forceinline__ void sie_deflect_f64(double x, double y, const double *c, double &ax,
                                                double &ay)
{
    const double dx = x - c[0], dy = y - c[1];
    const double u = dx * c[2] + dy * c[3];
    const double v = dy * c[2] - dx * c[3];
    const double psi = sqrt(c[6] * (c[8] + u * u) + v * v);
    const double du = psi + c[9], dv = psi + c[10];
    if (!(du > 0.0)) return;
    const double zu = u / du;
    const double zv = v / dv;
    double au, av;
    if (c[15] != 0.0) {
        // atan(e z)/e and atanh(e z)/e to O(e^4)
        const double e2 = c[16], zu2 = zu * zu, zv2 = zv * zv;
        au = c[13] * zu * (1.0 - e2 * zu2 / 3.0 + e2 * e2 * zu2 * zu2 / 5.0);
        av = c[13] * zv * (1.0 + e2 * zv2 / 3.0 + e2 * e2 * zv2 * zv2 / 5.0);
    } else {
        au = c[13] * atan(c[11] * zu);
        av = c[13] * atanh(c[11] * zv);
    }
    ax += au * c[2] - av * c[3];
    ay += au * c[3] + av * c[2];
}

// Light profile in FP64.
__device__ __forceinline__ double light_f64(double x, double y, const double *c)
{
    if (c[15] == (double)kKindFlat) return c[13];
    const double dx = x - c[0], dy = y - c[1];
    const double u = dx * c[2] + dy * c[3];
    const double v = dy * c[2] - dx * c[3];
    const double rho2 = c[6] * u * u + c[7] * v * v;
    const double t = (c[15] == (double)kKindGauss) ? c[11] * rho2
                                                    : c[11] * exp2(c[10] * log2(rho2));
    return c[13] * exp2(-t);
}

// FP32 constants of one component held in registers for a row of rays.
struct SieF {
    float x0, y0, cs, sn, csl, snl, q2, q2l, s2, s, q2s, e, el, pref, prefl, series, e2;
};
struct LightF {
    float x0, y0, cs, sn, csl, snl, qr, iqr, qrl, iqrl, p2, B, Bl, A, Al, kind;
};

__device__ __forceinline__ SieF load_sie(const float *c)
{
    const float4 a = reinterpret_cast<const float4 *>(c)[0];
    const float4 b = reinterpret_cast<const float4 *>(c)[1];
    const float4 d = reinterpret_cast<const float4 *>(c)[2];
    const float4 f = reinterpret_cast<const float4 *>(c)[3];
    SieF k;
    k.x0 = a.x; k.y0 = a.y; k.cs = a.z; k.sn = a.w;
    k.csl = b.x; k.snl = b.y; k.q2 = b.z; k.q2l = b.w;
    k.s2 = d.x; k.s = d.y; k.q2s = d.z; k.e = d.w;
    k.el = f.x; k.pref = f.y; k.prefl = f.z; k.series = f.w;
    k.e2 = c[16];
    return k;
}

__device__ __forceinline__ LightF load_light(const float *c)
{
    const float4 a = reinterpret_cast<const float4 *>(c)[0];
    const float4 b = reinterpret_cast<const float4 *>(c)[1];
    const float4 d = reinterpret_cast<const float4 *>(c)[2];
    const float4 f = reinterpret_cast<const float4 *>(c)[3];
    LightF k;
    k.x0 = a.x; k.y0 = a.y; k.cs = a.z; k.sn = a.w;
    k.csl = b.x; k.snl = b.y; k.qr = b.z; k.iqr = b.w;
    k.qrl = d.x; k.iqrl = d.y; k.p2 = d.z; k.B = d.w;
    k.Bl = f.x; k.A = f.y; k.Al = f.z; k.kind = f.w;
    return k;
}

// SIE in FP32 with compensated constants: every product with a constant
// that carries a residual partner is a float-pair multiply-add, so the
// float rounding of the constants does not bias the deflection field.
// Quotients and the square root use the fast forms (a few ulp, random in
// sign from ray to ray); atan and atanh are the minimax forms of
// lensed_sie_trig.cuh, fed the numerator and denominator of their argument.
__device__ __forceinline__ void sie_f32(const SieF &k, float x, float y, float &ax, float &ay)
{
    const float dx = x - k.x0, dy = y - k.y0;
    const float u = fmaf(dx, k.cs, fmaf(dy, k.sn, fmaf(dx, k.csl, dy * k.snl)));
    const float v = fmaf(dy, k.cs, fmaf(-dx, k.sn, fmaf(dy, k.csl, -dx * k.snl)));
    const float w = fmaf(u, u, k.s2);
    const float psi2 = fmaf(k.q2, w, fmaf(k.q2l, w, v * v));
    const float psi = psi2 > 0.f ? psi2 * rsqrtf(psi2) : 0.f;
    const float du = psi + k.s, dv = psi + k.q2s;
    float A1, A2;
    if (k.series != 0.f) {
        const float zu = du > 0.f ? __fdividef(u, du) : 0.f;
        const float zv = du > 0.f ? __fdividef(v, dv) : 0.f;
        const float zu2 = zu * zu, zv2 = zv * zv;
        A1 = zu * (1.f - k.e2 * zu2 * (1.f / 3.f) + k.e2 * k.e2 * zu2 * zu2 * 0.2f);
        A2 = zv * (1.f + k.e2 * zv2 * (1.f / 3.f) + k.e2 * k.e2 * zv2 * zv2 * 0.2f);
    } else {
        A1 = atan_ratio(fmaf(k.e, u, k.el * u), du);
        A2 = atanh_ratio(fmaf(k.e, v, k.el * v), dv);
    }
    const float au = fmaf(k.pref, A1, k.prefl * A1);
    const float av = fmaf(k.pref, A2, k.prefl * A2);
    ax += fmaf(au, k.cs, fmaf(-av, k.sn, fmaf(au, k.csl, -av * k.snl)));
    ay += fmaf(au, k.sn, fmaf(av, k.cs, fmaf(au, k.snl, av * k.csl)));
}

// Light profile in FP32 with compensated constants; MUFU lg2 / ex2.
__device__ __forceinline__ float light_f32(const LightF &k, float x, float y)
{
    const float dx = x - k.x0, dy = y - k.y0;
    const float u = fmaf(dx, k.cs, fmaf(dy, k.sn, fmaf(dx, k.csl, dy * k.snl)));
    const float v = fmaf(dy, k.cs, fmaf(-dx, k.sn, fmaf(dy, k.csl, -dx * k.snl)));
    const float uu = u * u, vv = v * v;
    const float rho2 = fmaf(k.qr, uu, fmaf(k.iqr, vv, fmaf(k.qrl, uu, k.iqrl * vv)));
    const float f = (k.kind == (float)kKindGauss) ? rho2 : ex2f(k.p2 * lg2f(rho2));
    const float t = fmaf(k.B, f, k.Bl * f);
    const float g = ex2f(-t);
    return fmaf(k.A, g, k.Al * g);
}

// Any light profile, including the flat sky (kind kKindFlat: I = A).
__device__ __forceinline__ float light_any_f32(const LightF &k, float x, float y)
{
    return k.kind == (float)kKindFlat ? k.A : light_f32(k, x, y);
}

// The parts of a rotation into a component's frame that depend on the row
// coordinate alone, dy = y - y0 (shared by the G rays of a node row):
// du = dy sin(PA), dv = dy cos(PA), each compensated like the per-ray terms.
struct RowTerms {
    float du, dv;
};
__device__ __forceinline__ RowTerms row_terms(float y, float y0, float cs, float sn, float csl,
                                              float snl)
{
    const float dy = y - y0;
    return {fmaf(dy, sn, dy * snl), fmaf(dy, cs, dy * csl)};
}

// sie_f32 for the rays of a node row whose terms are R (the row's products
// computed once), one ray (V = float) or a pair (V = float2): the same
// formulas, every operation rounded once (lensed_vec2.cuh), the products with
// -sin taken as products with the negated constant (exact).
template <class V>
__device__ __forceinline__ void sie_row_v(const SieF &k, const RowTerms &R, V x, V &ax, V &ay)
{
    const V dx = vsub(x, vsplat<V>(k.x0));
    const V u = vfma(dx, vsplat<V>(k.cs), vfma(dx, vsplat<V>(k.csl), vsplat<V>(R.du)));
    const V v = vfma(dx, vsplat<V>(-k.sn), vfma(dx, vsplat<V>(-k.snl), vsplat<V>(R.dv)));
    const V w = vfma(u, u, vsplat<V>(k.s2));
    const V psi2 = vfma(vsplat<V>(k.q2), w, vfma(vsplat<V>(k.q2l), w, vmul(v, v)));
    const V psi = vmul(psi2, vmap(psi2, [](float a) { return a > 0.f ? rsqrtf(a) : 0.f; }));
    const V du = vadd(psi, vsplat<V>(k.s)), dv = vadd(psi, vsplat<V>(k.q2s));
    V A1, A2;
    if (k.series != 0.f) {
        // q -> 1: atan(e z)/e and atanh(e z)/e by their series in e z
        const float e2 = k.e2, e4 = __fmul_rn(e2, e2);
        A1 = vmap(u, du, [=](float uu, float d) {
            const float z = d > 0.f ? __fdividef(uu, d) : 0.f, z2 = __fmul_rn(z, z);
            return __fmul_rn(z, __fadd_rn(__fsub_rn(1.f, __fmul_rn(__fmul_rn(e2, z2), 1.f / 3.f)),
                                          __fmul_rn(__fmul_rn(__fmul_rn(e4, z2), z2), 0.2f)));
        });
        A2 = vmap(v, dv, du, du, [=](float vv, float d, float dd, float) {
            const float z = dd > 0.f ? __fdividef(vv, d) : 0.f, z2 = __fmul_rn(z, z);
            return __fmul_rn(z, __fadd_rn(__fadd_rn(1.f, __fmul_rn(__fmul_rn(e2, z2), 1.f / 3.f)),
                                          __fmul_rn(__fmul_rn(__fmul_rn(e4, z2), z2), 0.2f)));
        });
    } else {
        A1 = atan_ratio(vfma(vsplat<V>(k.e), u, vmul(vsplat<V>(k.el), u)), du);
        A2 = atanh_ratio(vfma(vsplat<V>(k.e), v, vmul(vsplat<V>(k.el), v)), dv);
    }
    const V au = vfma(vsplat<V>(k.pref), A1, vmul(vsplat<V>(k.prefl), A1));
    const V av = vfma(vsplat<V>(k.pref), A2, vmul(vsplat<V>(k.prefl), A2));
    ax = vadd(ax, vfma(au, vsplat<V>(k.cs),
                       vfma(av, vsplat<V>(-k.sn), vfma(au, vsplat<V>(k.csl), vmul(av, vsplat<V>(-k.snl))))));
    ay = vadd(ay, vfma(au, vsplat<V>(k.sn),
                       vfma(av, vsplat<V>(k.cs), vfma(au, vsplat<V>(k.snl), vmul(av, vsplat<V>(k.csl))))));
}

// A light profile at frame coordinates (u, v) (major axis along u), one ray
// or a pair; with rho2 != nullptr also (R / r)^2 of each ray.
template <class V>
__device__ __forceinline__ V light_uv_v(const LightF &k, V u, V v, V *rho2_out)
{
    const V uu = vmul(u, u), vv = vmul(v, v);
    const V rho2 = vfma(vsplat<V>(k.qr), uu,
                        vfma(vsplat<V>(k.iqr), vv, vfma(vsplat<V>(k.qrl), uu, vmul(vsplat<V>(k.iqrl), vv))));
    if (rho2_out) *rho2_out = rho2;
    V f = rho2;
    if (k.kind != (float)kKindGauss)
        f = vmap(vmul(vsplat<V>(k.p2), vmap(rho2, [](float a) { return lg2f(a); })),
                 [](float a) { return ex2f(a); });
    const V t = vfma(vsplat<V>(k.B), f, vmul(vsplat<V>(k.Bl), f));
    const V g = vmap(t, [](float a) { return ex2f(-a); });
    return vfma(vsplat<V>(k.A), g, vmul(vsplat<V>(k.Al), g));
}

// light_f32 for the rays of a node row whose terms are R
template <class V>
__device__ __forceinline__ V light_row_v(const LightF &k, const RowTerms &R, V x)
{
    const V dx = vsub(x, vsplat<V>(k.x0));
    const V u = vfma(dx, vsplat<V>(k.cs), vfma(dx, vsplat<V>(k.csl), vsplat<V>(R.du)));
    const V v = vfma(dx, vsplat<V>(-k.sn), vfma(dx, vsplat<V>(-k.snl), vsplat<V>(R.dv)));
    return light_uv_v(k, u, v, (V *)nullptr);
}

// light_f32 (and (R / r)^2 with rho2 != nullptr) at source-plane positions
// (x, y), one ray or a pair
template <class V>
__device__ __forceinline__ V light_at_v(const LightF &k, V x, V y, V *rho2)
{
    const V dx = vsub(x, vsplat<V>(k.x0)), dy = vsub(y, vsplat<V>(k.y0));
    const V u = vfma(dx, vsplat<V>(k.cs),
                     vfma(dy, vsplat<V>(k.sn), vfma(dx, vsplat<V>(k.csl), vmul(dy, vsplat<V>(k.snl)))));
    const V v = vfma(dy, vsplat<V>(k.cs),
                     vfma(dx, vsplat<V>(-k.sn), vfma(dy, vsplat<V>(k.csl), vmul(dx, vsplat<V>(-k.snl)))));
    return light_uv_v(k, u, v, rho2);
}

// FP64 SIE of one ray in a MIXED evaluation.  Out of line, so that none of
// its double-precision arithmetic is scheduled on the FP32 path; the ray
// position is rebuilt in FP64 from the pixel index and the FP64 node offsets.
__device__ __noinline__ void sie_ray_f64(float jc, float ic, double hd, double ua, double vb,
                                         const double *c, float &ax, float &ay)
{
    double dax = 0.0, day = 0.0;
    sie_deflect_f64((double)jc * hd + ua, (double)ic * hd + vb, c, dax, day);
    ax += (float)dax;
    ay += (float)day;
}

// Deflection of one mass component in FP64, added to (ax, ay).
__device__ __forceinline__ void deflect_f64(int t, double x, double y, const double *cc,
                                            double &ax, double &ay)
{
    if (t == LENSED_SIE) {
        sie_deflect_f64(x, y, cc, ax, ay);
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

// Total image-plane brightness at one ray in FP64 (Eqs. 1-2).
struct RayCtx {
    int ncomp;
    const int *type;
    const int *plane;
    const double *cd;
};

__device__ __forceinline__ double brightness_f64(double x, double y, const RayCtx &R)
{
    double I = 0.0, ax = 0.0, ay = 0.0;
    for (int c = 0; c < R.ncomp; ++c) {
        const int pl = R.plane[c];
        const double *cc = R.cd + c * kNC;
        if (pl == LENSED_PLANE_FOREGROUND) {
            I += light_f64(x, y, cc);
        } else if (pl == LENSED_PLANE_LENS) {
            deflect_f64(R.type[c], x, y, cc, ax, ay);
        }
    }
    const double sx = x - ax, sy = y - ay;
    for (int c = 0; c < R.ncomp; ++c)
        if (R.plane[c] == LENSED_PLANE_SOURCE) I += light_f64(sx, sy, R.cd + c * kNC);
    return I;
}

// Validity of a (system, point): every component in its domain.  Then the
// image-plane priors (Sec. 5): a source whose position parameters are an
// image-plane position theta is moved to theta - alpha(theta) (Eq. 1), the
// deflection of the same point's lens in FP64.
__global__ void k_prologue_valid(const SysDev *__restrict__ sys, int s0, int nS, int P, int p0,
                                 int nP, int C_total, const int *__restrict__ comp_type,
                                 const unsigned char *__restrict__ cvalid, float *__restrict__ cf,
                                 double *__restrict__ cd, unsigned char *__restrict__ valid)
{
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (tid >= (long long)nS * nP) return;
    const int s = s0 + (int)(tid / nP);
    const int p = p0 + (int)(tid % nP);
    const SysDev &S = sys[s];
    unsigned char ok = 1;
    for (int c = 0; c < S.ncomp; ++c) ok &= cvalid[(size_t)p * C_total + S.comp_off + c];
    if (ok && S.imgpos_mask) {
        const size_t base = ((size_t)p * C_total + S.comp_off) * kNC;
        for (int c = 0; c < S.ncomp; ++c) {
            if (!((S.imgpos_mask >> c) & 1)) continue;
            double *cc = cd + base + (size_t)c * kNC;
            const double tx = cc[0], ty = cc[1];
            double ax = 0.0, ay = 0.0;
            for (int l = 0; l < S.ncomp; ++l) {
                const int t = comp_type[S.comp_off + l];
                if (t <= LENSED_POINTMASS) deflect_f64(t, tx, ty, cd + base + (size_t)l * kNC, ax, ay);
            }
            const double yx = tx - ax, yy = ty - ay;
            if (!isfinite(yx) || !isfinite(yy)) ok = 0;
            cc[0] = yx;
            cc[1] = yy;
            float *fc = cf + base + (size_t)c * kNC;
            fc[0] = (float)yx;
            fc[1] = (float)yy;
            fc[16] = (float)(yx - (double)fc[0]);
            fc[17] = (float)(yy - (double)fc[1]);
        }
    }
    valid[(size_t)s * P + p] = ok;
}

void launch_prologue(const SysDev *sys, const int *comp_sys, int s0, int nS, int c0, int nC,
                     const int *comp_type, const int *comp_free, const double *comp_value,
                     const double *params, bool single_row, int P, int p0, int nP,
                     int n_par_stride, int C_total, const double *bn_table, float *cf,
                     double *cd, unsigned char *cvalid, unsigned char *valid, cudaStream_t st)
{
    const long long n = (long long)nC * nP;
    const int threads = 64;
    k_prologue_comp<<<(unsigned)((n + threads - 1) / threads), threads, 0, st>>>(
        sys, comp_sys, c0, nC, comp_type, comp_free, comp_value, params, single_row ? 1 : 0, P,
        p0, nP, n_par_stride, C_total, bn_table, cf, cd, cvalid);
    const long long n2 = (long long)nS * nP;
    k_prologue_valid<<<(unsigned)((n2 + 127) / 128), 128, 0, st>>>(
        sys, s0, nS, P, p0, nP, C_total, comp_type, cvalid, cf, cd, valid);
}


// ---------------------------------------------------------------------------
// a2-a5: ray tracing and pixel integration

// Shared-memory staging common to the trace kernels: the point's packed
// constants, component types and planes, node offsets and 2-D weights.
struct TraceSmem {
    float cf[LENSED_MAX_COMPONENTS * kNC];
    double cd[LENSED_MAX_COMPONENTS * kNC];
    float uh[LENSED_MAX_RULE_ORDER], ul[LENSED_MAX_RULE_ORDER];            // ud as float pairs
    int type[LENSED_MAX_COMPONENTS], plane[LENSED_MAX_COMPONENTS];
    float u[LENSED_MAX_RULE_ORDER];
    double ud[LENSED_MAX_RULE_ORDER];
    float w[LENSED_MAX_RULE_ORDER * LENSED_MAX_RULE_ORDER];
    double wd[LENSED_MAX_RULE_ORDER * LENSED_MAX_RULE_ORDER];
};

__device__ __forceinline__ void stage_point(TraceSmem &sm, const SysDev &S, const int *comp_type,
                                            const int *comp_plane, const float *cf,
                                            const double *cd, size_t cbase, bool need_f64,
                                            bool w_f64, const NodeTables &nodes)
{
    const int ncomp = S.ncomp, nn = S.nn;
    for (int k = threadIdx.x; k < ncomp * kNC; k += blockDim.x) {
        sm.cf[k] = cf[cbase + k];
        if (need_f64) sm.cd[k] = cd[cbase + k];
    }
    for (int k = threadIdx.x; k < ncomp; k += blockDim.x) {
        sm.type[k] = comp_type[S.comp_off + k];
        sm.plane[k] = comp_plane[S.comp_off + k];
    }
    for (int k = threadIdx.x; k < nn; k += blockDim.x) {
        sm.u[k] = nodes.u[S.node_off + k];
        const double v = nodes.ud[S.node_off + k];
        sm.ud[k] = v;
        sm.uh[k] = (float)v;
        sm.ul[k] = (float)(v - (double)(float)v);
    }
    for (int k = threadIdx.x; k < nn * nn; k += blockDim.x) {
        if (w_f64) sm.wd[k] = nodes.wd[S.w2_off + k];
        else sm.w[k] = nodes.w[S.w2_off + k];
    }
}

// ---- float-float lens equation for the rays MIXED re-traces near the centre
// of a source profile.  There the brightness is steep on the scale of the
// float grid of the traced position (~1e-7 arcsec near the Einstein radius),
// so the MIXED_FF rule gives every ray that the FP32 pass sees inside half an
// effective radius of a Sersic-type source (R < r/2) a source-plane position
// in float-float arithmetic (a value carried as an unevaluated sum hi + lo of
// two floats; Dekker 1971, Knuth's two-sum): the ray position, the
// deflection of every lens component and y = x - alpha.  The light is then
// evaluated in FP32 at that position.  FP64 would do the same at 1/64 of the
// FP32 rate on this GPU.
struct ff {
    float hi, lo;
};

__device__ __forceinline__ ff ff_quick(float a, float b)  // |a| >= |b|
{
    const float s = a + b;
    return {s, b - (s - a)};
}
__device__ __forceinline__ ff ff_two_sum(float a, float b)
{
    const float s = a + b, bb = s - a;
    return {s, (a - (s - bb)) + (b - bb)};
}
__device__ __forceinline__ ff ff_add(ff x, ff y)
{
    const ff s = ff_two_sum(x.hi, y.hi);
    return ff_quick(s.hi, s.lo + (x.lo + y.lo));
}
__device__ __forceinline__ ff ff_neg(ff x) { return {-x.hi, -x.lo}; }
__device__ __forceinline__ ff ff_sub(ff x, ff y) { return ff_add(x, ff_neg(y)); }
__device__ __forceinline__ ff ff_mul(ff x, ff y)
{
    const float p = x.hi * y.hi;
    const float e = fmaf(x.hi, y.hi, -p);
    return ff_quick(p, fmaf(x.hi, y.lo, fmaf(x.lo, y.hi, e)));
}
__device__ __forceinline__ ff ff_mulf(ff x, float f)
{
    const float p = x.hi * f;
    const float e = fmaf(x.hi, f, -p);
    return ff_quick(p, fmaf(x.lo, f, e));
}
__device__ __forceinline__ ff ff_addf(ff x, float f) { return ff_add(x, ff{f, 0.f}); }
// MUFU approximate reciprocal and reciprocal square root (rcp.approx /
// rsqrt.approx, ~22 correct bits): the float-float operations below start
// from them and recover the remaining digits from exact remainders.
__device__ __forceinline__ float rcp_approx(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float rsqrt_approx(float x)
{
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// x / y for y != 0: two quotient digits, the second from the exact
// remainder x - y q1 (relative error ~2^-44, far below what the re-trace
// needs: positions to ~1e-10 arcsec)
__device__ __forceinline__ ff ff_div(ff x, ff y)
{
    const float r = rcp_approx(y.hi);
    const float q1 = x.hi * r;
    const ff rem = ff_sub(x, ff_mulf(y, q1));
    const float q2 = rem.hi * r;
    return ff_quick(q1, q2);
}
// sqrt(x) for x >= 0: approximate root, then one Newton correction from the
// exact residual x - s^2 (quadratic: ~2^-44)
__device__ __forceinline__ ff ff_sqrt(ff x)
{
    if (!(x.hi > 0.f)) return {0.f, 0.f};
    const float rs = rsqrt_approx(x.hi);
    const float s = x.hi * rs;
    const float p = s * s;
    const ff sq{p, fmaf(s, s, -p)};
    const ff d = ff_sub(x, sq);
    return ff_quick(s, d.hi * (0.5f * rs));
}

// tan(k/16), k = 0..26, and tanh(k/16), k = 0..127, as float pairs (computed
// by the runtime in long double): reduction points for atan and atanh.
__constant__ float kTan16[27][2];
__constant__ float kTanh16[128][2];

// atan(t) = k/16 + atan(w), w = (t - tan(k/16)) / (1 + t tan(k/16)), k the
// multiple of 1/16 nearest to an estimate of atan(t) (t / (1 + 0.28 t^2),
// or pi/2 minus that of 1/t beyond 1; error < 0.005), so |w| <= tan(1/32 +
// 0.005) and the series w - w^3/3 + w^5/5 - w^7/7 + w^9/9 leaves < 1e-15;
// its tail after w is applied in float.  Odd in t.
__device__ __forceinline__ ff ff_atan(ff t)
{
    const bool neg = t.hi < 0.f;
    if (neg) t = ff_neg(t);
    const float a = t.hi;
    const float est = a <= 1.f ? a * rcp_approx(fmaf(0.28f, a * a, 1.f))
                               : 1.5707964f - a * rcp_approx(fmaf(a, a, 0.28f));
    const int k = min(max(__float2int_rn(16.f * est), 0), 26);
    const ff c{kTan16[k][0], kTan16[k][1]};
    const ff w = ff_div(ff_sub(t, c), ff_addf(ff_mul(t, c), 1.f));
    const float s = w.hi * w.hi;
    const float tail = w.hi * s * fmaf(s, fmaf(s, fmaf(s, 1.f / 9.f, -1.f / 7.f), 0.2f), -1.f / 3.f);
    ff r = ff_addf(ff_add(ff{k * 0.0625f, 0.f}, w), tail);
    return neg ? ff_neg(r) : r;
}

// atanh(z), |z| < 1: the same reduction with tanh(k/16) and
// w = (z - tanh(k/16)) / (1 - z tanh(k/16)), k from the estimate
// (ln 2 / 2)(lg2(1 + z) - lg2(1 - z)); series w + w^3/3 + ... + w^9/9.
__device__ __forceinline__ ff ff_atanh(ff z)
{
    const bool neg = z.hi < 0.f;
    if (neg) z = ff_neg(z);
    const float a = fminf(z.hi, 0.99999994f);
    const float est = 0.34657359f * (lg2f(1.f + a) - lg2f(1.f - a));
    const int k = min(max(__float2int_rn(16.f * est), 0), 127);
    const ff c{kTanh16[k][0], kTanh16[k][1]};
    const ff w = ff_div(ff_sub(z, c), ff_add(ff{1.f, 0.f}, ff_neg(ff_mul(z, c))));
    const float s = w.hi * w.hi;
    const float tail = w.hi * s * fmaf(s, fmaf(s, fmaf(s, 1.f / 9.f, 1.f / 7.f), 0.2f), 1.f / 3.f);
    ff r = ff_addf(ff_add(ff{k * 0.0625f, 0.f}, w), tail);
    return neg ? ff_neg(r) : r;
}

// A packed constant as a float pair: its FP32 value and the residual the
// prologue stored in slot `lo` of the same component.
__device__ __forceinline__ ff ff_pair(const float *c, int hi, int lo) { return {c[hi], c[lo]}; }

// FP32 light profile at a given offset (dx, dy) from its centre.
__device__ __forceinline__ float light_f32_at(const LightF &k, float dx, float dy)
{
    const float u = fmaf(dx, k.cs, fmaf(dy, k.sn, fmaf(dx, k.csl, dy * k.snl)));
    const float v = fmaf(dy, k.cs, fmaf(-dx, k.sn, fmaf(dy, k.csl, -dx * k.snl)));
    const float uu = u * u, vv = v * v;
    const float rho2 = fmaf(k.qr, uu, fmaf(k.iqr, vv, fmaf(k.qrl, uu, k.iqrl * vv)));
    const float f = (k.kind == (float)kKindGauss) ? rho2 : ex2f(k.p2 * lg2f(rho2));
    const float t = fmaf(k.B, f, k.Bl * f);
    const float g = ex2f(-t);
    return fmaf(k.A, g, k.Al * g);
}

// Where the float-float re-trace reads a point's constants: the packed FP32
// blocks of its components, their types and planes (shared memory in the
// trace block, global memory in the second pass).
struct FfConsts {
    const float *cf;
    const int *type, *plane;
};

// A node offset (FP64) as a float pair.
__device__ __forceinline__ ff node_pair(double v)
{
    const float hi = (float)v;
    return {hi, (float)(v - (double)hi)};
}

// Source-plane brightness of a ray of pixel (jc, ic) with node offsets ua
// (along x) and vb (along y) as float pairs, with the lens equation in
// float-float (all lens components) and the light in FP32.  Every constant
// comes as a float pair from the component's packed FP32 block (value and
// residual slots, see k_prologue_comp).
__device__ __noinline__ float source_brightness_ff_at(FfConsts K, int ncomp, float jc, float ic,
                                                      float h, float h_lo, ff ua, ff vb)
{
    // ray position: (j - cx) h + t_a h, with h and the node offset as float pairs
    ff x = ff_add(ff_add(ff{jc * h, fmaf(jc, h, -(jc * h))}, ff{jc * h_lo, 0.f}), ua);
    ff y = ff_add(ff_add(ff{ic * h, fmaf(ic, h, -(ic * h))}, ff{ic * h_lo, 0.f}), vb);
    ff ax{0.f, 0.f}, ay{0.f, 0.f};
    for (int c = 0; c < ncomp; ++c) {
        if (K.plane[c] != LENSED_PLANE_LENS) continue;
        const float *k = K.cf + c * kNC;
        const int t = K.type[c];
        if (t == LENSED_SIE) {
            const ff dx = ff_sub(x, ff_pair(k, 0, 19)), dy = ff_sub(y, ff_pair(k, 1, 20));
            const ff cs = ff_pair(k, 2, 4), sn = ff_pair(k, 3, 5);
            const ff u = ff_add(ff_mul(dx, cs), ff_mul(dy, sn));
            const ff v = ff_sub(ff_mul(dy, cs), ff_mul(dx, sn));
            const ff psi = ff_sqrt(ff_add(ff_mul(ff_pair(k, 6, 7),
                                                 ff_add(ff_pair(k, 8, 21), ff_mul(u, u))),
                                          ff_mul(v, v)));
            const ff du = ff_add(psi, ff_pair(k, 9, 22));
            const ff dv = ff_add(psi, ff_pair(k, 10, 23));
            if (!(du.hi > 0.f)) continue;  // exact centre of a coreless SIE
            ff A1, A2;
            if (k[15] != 0.f) {
                const ff zu = ff_div(u, du), zv = ff_div(v, dv);
                const float e2 = k[16];
                const float su = e2 * zu.hi * zu.hi, sv = e2 * zv.hi * zv.hi;
                A1 = ff_addf(zu, zu.hi * su * fmaf(su, 0.2f, -1.f / 3.f));
                A2 = ff_addf(zv, zv.hi * sv * fmaf(sv, 0.2f, 1.f / 3.f));
            } else {
                const ff e = ff_pair(k, 11, 12);
                A1 = ff_atan(ff_div(ff_mul(e, u), du));
                A2 = ff_atanh(ff_div(ff_mul(e, v), dv));
            }
            const ff pref = ff_pair(k, 13, 14);
            const ff au = ff_mul(pref, A1), av = ff_mul(pref, A2);
            ax = ff_add(ax, ff_sub(ff_mul(au, cs), ff_mul(av, sn)));
            ay = ff_add(ay, ff_add(ff_mul(au, sn), ff_mul(av, cs)));
        } else if (t == LENSED_SHEAR) {
            const ff dx = ff_sub(x, ff_pair(k, 0, 4)), dy = ff_sub(y, ff_pair(k, 1, 5));
            const ff g1 = ff_pair(k, 2, 6), g2 = ff_pair(k, 3, 7);
            ax = ff_add(ax, ff_add(ff_mul(g1, dx), ff_mul(g2, dy)));
            ay = ff_add(ay, ff_sub(ff_mul(g2, dx), ff_mul(g1, dy)));
        } else {
            const ff dx = ff_sub(x, ff_pair(k, 0, 3)), dy = ff_sub(y, ff_pair(k, 1, 4));
            const ff r2 = ff_add(ff_mul(dx, dx), ff_mul(dy, dy));
            if (!(r2.hi > 0.f)) continue;
            const ff f = ff_div(ff_pair(k, 2, 5), r2);
            ax = ff_add(ax, ff_mul(f, dx));
            ay = ff_add(ay, ff_mul(f, dy));
        }
    }
    const ff sx = ff_sub(x, ax), sy = ff_sub(y, ay);
    float I = 0.f;
    for (int c = 0; c < ncomp; ++c) {
        if (K.plane[c] != LENSED_PLANE_SOURCE) continue;
        const float *k = K.cf + c * kNC;
        const LightF L = load_light(k);
        if (L.kind == (float)kKindFlat) {
            I += L.A;
            continue;
        }
        const ff ox = ff_sub(sx, ff_pair(k, 0, 16)), oy = ff_sub(sy, ff_pair(k, 1, 17));
        I += light_f32_at(L, ox.hi + ox.lo, oy.hi + oy.lo);
    }
    return I;
}

// The same for ray (a, b) of the rule, with the point staged in shared memory.
__device__ __forceinline__ float source_brightness_ff(const TraceSmem &sm, int ncomp, float jc,
                                                      float ic, float h, float h_lo, int a, int b)
{
    return source_brightness_ff_at(FfConsts{sm.cf, sm.type, sm.plane}, ncomp, jc, ic, h, h_lo,
                                   ff{sm.uh[a], sm.ul[a]}, ff{sm.uh[b], sm.ul[b]});
}

// FP32 light of a source, also reporting (R / r)^2 of the ray.
__device__ __forceinline__ float light_f32_rho(const LightF &k, float x, float y, float &rho2)
{
    const float dx = x - k.x0, dy = y - k.y0;
    const float u = fmaf(dx, k.cs, fmaf(dy, k.sn, fmaf(dx, k.csl, dy * k.snl)));
    const float v = fmaf(dy, k.cs, fmaf(-dx, k.sn, fmaf(dy, k.csl, -dx * k.snl)));
    const float uu = u * u, vv = v * v;
    rho2 = fmaf(k.qr, uu, fmaf(k.iqr, vv, fmaf(k.qrl, uu, k.iqrl * vv)));
    const float f = (k.kind == (float)kKindGauss) ? rho2 : ex2f(k.p2 * lg2f(rho2));
    const float t = fmaf(k.B, f, k.Bl * f);
    const float g = ex2f(-t);
    return fmaf(k.A, g, k.Al * g);
}

// MIXED_FF re-traces rays with (R / r)^2 below this.  Measured against the
// oracle (225 prior points of the 200x200 workload, 256 of the 64x64 one),
// R < r/2 leaves the largest log-likelihood errors as low as R < r does
// (7.2e-4 and 4.7e-4 against 9.3e-4 and 3.7e-4: the worst points are set by
// other float terms) at a quarter of the re-traced rays; below it they grow
// (R < 0.32 r: 1.1e-3, R < 0.2 r: 3.1e-3 on the 200x200 sample).
constexpr float kCuspRho2 = 0.25f;
constexpr int kQCap = 2048;       // deferred float-float rays per trace block

// a2-a5 in FP32 (also the first pass of MIXED): one thread per pixel; for
// every row of the rule's node grid, G rays are traced together component by
// component, so each component's constants are read into registers once per
// G rays and the G independent rays give the scheduler instruction-level
// parallelism.  EXACT: the rule has exactly G nodes per row (no guards).
// GQ (MIXED_FF, EXACT): the float-float re-traces go to the launch's global
// queue, appended warp by warp, for k_retrace_ff and k_apply_ff.
// What a pixel's ray loop does with rays near the centre of a Sersic-type
// source (MIXED_FF): nothing (other modes), record the smallest (R/r)^2 of
// all rays in pmin, defer the rays' source light to the queue (their bits in
// mask; the rest of the light summed now), or re-trace them in place.
constexpr int kNearIgnore = 0, kNearFlag = 1, kNearDefer = 2, kNearInPlace = 3;

// Where a pixel's ray loop reads its point's constants: the trace block's
// staged copy in shared memory, or global memory (a pixel of any point).
struct SmemConsts {
    const TraceSmem &sm;
    __device__ const float *cf(int c) const { return sm.cf + c * kNC; }
    __device__ int plane(int c) const { return sm.plane[c]; }
    __device__ int type(int c) const { return sm.type[c]; }
    __device__ float u(int a) const { return sm.u[a]; }
    __device__ float w(int r) const { return sm.w[r]; }
    __device__ float ff(int ncomp, float jc, float ic, float h, float h_lo, int a, int b) const
    {
        return source_brightness_ff(sm, ncomp, jc, ic, h, h_lo, a, b);
    }
};
struct GlobalConsts {
    const float *cfp;
    const int *typ, *pln;
    const float *uu, *ww;
    const double *ud;
    __device__ const float *cf(int c) const { return cfp + c * kNC; }
    __device__ int plane(int c) const { return pln[c]; }
    __device__ int type(int c) const { return typ[c]; }
    __device__ float u(int a) const { return uu[a]; }
    __device__ float w(int r) const { return ww[r]; }
    __device__ float ff(int ncomp, float jc, float ic, float h, float h_lo, int a, int b) const
    {
        return source_brightness_ff_at(FfConsts{cfp, typ, pln}, ncomp, jc, ic, h, h_lo,
                                       node_pair(ud[a]), node_pair(ud[b]));
    }
};

// a2-a5 for one pixel (centre (jc, ic) in pixels from the image centre): for
// every row of the rule's node grid, G rays traced together component by
// component (each component's constants read once per G rays), two at a
// time in packed FP32 instructions, each ray's brightness added to acc with
// its weight in ray order.  EXACT: the rule has exactly G nodes per row.
template <int MODE, int G, bool EXACT, int NEAR, class KC>
__device__ __forceinline__ float pixel_rays(const KC &kc, const SysDev &S, int ncomp, int nn,
                                            float jc, float ic, float acc,
                                            unsigned long long &mask, float &pmin)
{
    // pixel centre (j - cx) h with h as a float pair: one rounding, no
    // coherent scale error
    const float xc = fmaf(jc, S.h, jc * S.h_lo);
    const float yc = fmaf(ic, S.h, ic * S.h_lo);
    for (int b = 0; b < nn; ++b) {
        const float y = yc + kc.u(b);
        for (int a0 = 0; a0 < nn; a0 += G) {
            // the G rays of the chunk, traced in pairs (packed FP32) and, for
            // odd G, one more alone; every value is the same bits either way
            Rays<G> xk, ax, ay, I;
#pragma unroll
            for (int k = 0; k < G; ++k) {
                const int a = EXACT ? k : min(a0 + k, nn - 1);
                xk.set(k, xc + kc.u(a));
            }
            ax.fill(0.f);
            ay.fill(0.f);
            I.fill(0.f);
            for (int c = 0; c < ncomp; ++c) {
                const int pl = kc.plane(c);
                const float *cc = kc.cf(c);
                if (pl == LENSED_PLANE_FOREGROUND) {
                    const LightF L = load_light(cc);
                    if (L.kind == (float)kKindFlat) {
                        for_rays<G>([&](auto &i) {
                            using V = std::remove_reference_t<decltype(i)>;
                            i = vadd(i, vsplat<V>(L.A));
                        }, I);
                    } else {
                        const RowTerms R = row_terms(y, L.y0, L.cs, L.sn, L.csl, L.snl);
                        for_rays<G>([&](auto &x, auto &i) { i = vadd(i, light_row_v(L, R, x)); },
                                    xk, I);
                    }
                } else if (pl == LENSED_PLANE_LENS) {
                    const int t = kc.type(c);
                    if (t == LENSED_SIE) {
                        const SieF K = load_sie(cc);
                        const RowTerms R = row_terms(y, K.y0, K.cs, K.sn, K.csl, K.snl);
                        for_rays<G>([&](auto &x, auto &dx, auto &dy) { sie_row_v(K, R, x, dx, dy); },
                                    xk, ax, ay);
                    } else if (t == LENSED_SHEAR) {
                        const float x0 = cc[0], y0 = cc[1], g1 = cc[2], g2 = cc[3];
                        const float dy = y - y0, g2dy = g2 * dy, g1dy = -g1 * dy;
                        for_rays<G>([&](auto &x, auto &dx_, auto &dy_) {
                            using V = std::remove_reference_t<decltype(x)>;
                            const V dx = vsub(x, vsplat<V>(x0));
                            dx_ = vadd(dx_, vfma(vsplat<V>(g1), dx, vsplat<V>(g2dy)));
                            dy_ = vadd(dy_, vfma(vsplat<V>(g2), dx, vsplat<V>(g1dy)));
                        }, xk, ax, ay);
                    } else {  // point mass
                        const float x0 = cc[0], y0 = cc[1], te2 = cc[2];
                        const float dy = y - y0, dy2 = dy * dy;
                        for_rays<G>([&](auto &x, auto &dx_, auto &dy_) {
                            using V = std::remove_reference_t<decltype(x)>;
                            const V dx = vsub(x, vsplat<V>(x0));
                            const V r2 = vfma(dx, dx, vsplat<V>(dy2));
                            const V f = vmap(r2, [=](float r) { return r > 0.f ? __fdividef(te2, r) : 0.f; });
                            dx_ = vfma(f, dx, dx_);
                            dy_ = vfma(f, vsplat<V>(dy), dy_);
                        }, xk, ax, ay);
                    }
                }
            }
            // rmin: (R/r)^2 of the ray at the nearest Sersic-type source,
            // capped at the re-trace threshold (a float minimum per source,
            // the comparison once per ray)
            Rays<G> Ifg = I, rmin;
            rmin.fill(kCuspRho2);
            for (int c = 0; c < ncomp; ++c) {
                if (kc.plane(c) != LENSED_PLANE_SOURCE) continue;
                const LightF L = load_light(kc.cf(c));
                if (L.kind == (float)kKindFlat) {
                    for_rays<G>([&](auto &i) {
                        using V = std::remove_reference_t<decltype(i)>;
                        i = vadd(i, vsplat<V>(L.A));
                    }, I);
                } else if (NEAR != kNearIgnore && L.kind == (float)kKindPower) {
                    for_rays<G>([&](auto &x, auto &dx, auto &dy, auto &i, auto &rm) {
                        using V = std::remove_reference_t<decltype(x)>;
                        V r2;
                        i = vadd(i, light_at_v(L, vsub(x, dx), vsub(vsplat<V>(y), dy), &r2));
                        if (NEAR == kNearFlag) pmin = fminf(pmin, vminlane(r2));
                        else rm = vmap(rm, r2, [](float p, float q) { return fminf(p, q); });
                    }, xk, ax, ay, I, rmin);
                } else {
                    for_rays<G>([&](auto &x, auto &dx, auto &dy, auto &i) {
                        using V = std::remove_reference_t<decltype(x)>;
                        i = vadd(i, light_at_v(L, vsub(x, dx), vsub(vsplat<V>(y), dy), (V *)nullptr));
                    }, xk, ax, ay, I);
                }
            }
            if (NEAR == kNearDefer) {
                // the source part comes from the queue; keep the rest (the
                // row's flags gathered first, one shift into the mask per row)
                unsigned row = 0u;
#pragma unroll
                for (int k = 0; k < G; ++k) {
                    const bool nk = rmin.get(k) < kCuspRho2;
                    row |= nk ? 1u << k : 0u;
                    I.set(k, nk ? Ifg.get(k) : I.get(k));
                }
                mask |= (unsigned long long)row << (b * nn);
            } else if (NEAR == kNearInPlace) {
#pragma unroll
                for (int k = 0; k < G; ++k) {
                    if (!(rmin.get(k) < kCuspRho2) || !(EXACT || a0 + k < nn)) continue;
                    I.set(k, Ifg.get(k) + kc.ff(ncomp, jc, ic, S.h, S.h_lo, a0 + k, b));
                }
            }
#pragma unroll
            for (int k = 0; k < G; ++k)
                if (EXACT || a0 + k < nn) acc = fmaf(kc.w(b * nn + a0 + k), I.get(k), acc);
        }
    }
    return acc;
}

// The work of one trace block tb at point p (every thread of the CTA calls
// it; it returns to the caller, which may take another item).  stage = false:
// the shared constants already hold tb's system at point p.
template <int MODE, int G, bool EXACT, bool GQ>
__device__ __forceinline__ void trace_item(const SysDev *__restrict__ sys,
                                           const int *__restrict__ comp_type,
                                           const int *__restrict__ comp_plane,
                                           const float *__restrict__ cf,
                                           const double *__restrict__ cd,
                                           const unsigned char *__restrict__ valid, int P,
                                           int C_total, const int *__restrict__ need,
                                           const NodeTables &nodes, int p0,
                                           float *__restrict__ Lbuf, long long L_stride,
                                           const FfQueue &fq, const TraceBlock tb, const int p,
                                           const bool stage = true)
{
    __shared__ __align__(16) TraceSmem sm;
    if (!valid[(size_t)tb.sys * P + p]) return;
    const SysDev &S = sys[tb.sys];
    const size_t cbase = ((size_t)p * C_total + S.comp_off) * kNC;
    // MIXED_FF with at most 8 nodes per row defers its float-float re-traces
    // (64-bit ray mask per pixel): to a block-wide queue processed by all
    // lanes after the main loop, or (GQ) to the launch's global queue; the
    // others re-trace in place
    constexpr bool kFfDefer = (MODE == LENSED_PREC_MIXED_FF) && EXACT;
    constexpr bool kQueue = kFfDefer && !GQ;
    constexpr bool kWarpQ = kFfDefer && GQ;
    __shared__ int q_n;
    __shared__ unsigned short q_t[kQueue ? kQCap : 1];
    __shared__ unsigned char q_r[kQueue ? kQCap : 1];
    __shared__ float q_v[kQueue ? kQCap : 1];
    if (stage) stage_point(sm, S, comp_type, comp_plane, cf, cd, cbase, false, false, nodes);
    if (kQueue && threadIdx.x == 0) q_n = 0;
    __syncthreads();

    const int idx = tb.start + threadIdx.x;
    const bool active = idx < tb.end;
    // (a warp appending to the global queue needs all its lanes)
    if (!kQueue && !kWarpQ && !active) return;
    const int ncomp = S.ncomp;
    const int nn = EXACT ? G : S.nn;
    const int nx = S.nx;
    const int pix = active ? (need ? need[S.need_off + idx] : idx) : 0;
    const int i = pix / nx, j = pix - (pix / nx) * nx;
    const float jc = (float)j - S.cx, ic = (float)i - S.cy;

    float acc = (nodes.pre_f && S.pre_off >= 0 && active) ? nodes.pre_f[S.pre_off + pix] : 0.f;
    unsigned long long mask = 0ull;  // rays deferred to the queue
    float pmin = kCuspRho2;          // smallest (R/r)^2 of the pixel's rays
    constexpr int kNear = MODE != LENSED_PREC_MIXED_FF ? kNearIgnore
                        : !EXACT                     ? kNearInPlace
                        : GQ                         ? kNearFlag
                                                     : kNearDefer;
    if (active)
        acc = pixel_rays<MODE, G, EXACT, kNear>(SmemConsts{sm}, S, ncomp, nn, jc, ic, acc, mask,
                                                pmin);
    if (kWarpQ) {
        // a pixel with a ray inside half an effective radius of a source
        // centre goes to the pixel queue (one atomic per warp): k_refine_ff
        // recomputes it with those rays deferred.  Every other pixel's sum is
        // final here (the same arithmetic as the deferring loop, which leaves
        // a pixel without such rays unchanged).
        const unsigned full = 0xffffffffu, lane = threadIdx.x & 31u;
        const bool flag = active && pmin < kCuspRho2;
        const unsigned ball = __ballot_sync(full, flag);
        const size_t lin = (size_t)(p - p0) * L_stride + S.pix_off + pix;
        if (ball) {
            unsigned long long base = 0ull;
            if (lane == 0u) base = atomicAdd(fq.cnt + 1, (unsigned long long)__popc(ball));
            base = __shfl_sync(full, base, 0);
            const unsigned long long e = base + (unsigned long long)__popc(ball & ((1u << lane) - 1u));
            if (flag && e < (unsigned long long)fq.pcap)
                fq.pix[e] = FfEntry{(unsigned)lin, (unsigned)tb.sys};
        }
        if (active) Lbuf[lin] = acc;
        return;
    }
    if (kQueue) {
        // each pixel's deferred rays take consecutive slots in ray order
        const int n_t = __popcll(mask);
        const int base = n_t ? atomicAdd(&q_n, n_t) : 0;
        const bool fits = base + n_t <= kQCap;
        if (fits) {
            unsigned long long m = mask;
            for (int e = 0; m; ++e) {
                const int r = __ffsll((long long)m) - 1;
                m &= m - 1ull;
                q_t[base + e] = (unsigned short)threadIdx.x;
                q_r[base + e] = (unsigned char)r;
            }
        }
        __syncthreads();
        const int nq = min(q_n, kQCap);
        for (int e = threadIdx.x; e < nq; e += blockDim.x) {
            const int t = q_t[e], r = q_r[e];
            const int pt = need ? need[S.need_off + tb.start + t] : tb.start + t;
            const int it = pt / nx, jt = pt - (pt / nx) * nx;
            q_v[e] = source_brightness_ff(sm, ncomp, (float)jt - S.cx, (float)it - S.cy, S.h,
                                          S.h_lo, r % nn, r / nn);
        }
        __syncthreads();
        if (active && n_t) {
            unsigned long long m = mask;
            for (int e = 0; m; ++e) {
                const int r = __ffsll((long long)m) - 1;
                m &= m - 1ull;
                const float v = fits ? q_v[base + e]
                                     : source_brightness_ff(sm, ncomp, jc, ic, S.h, S.h_lo,
                                                            r % nn, r / nn);
                acc = fmaf(sm.w[r], v, acc);
            }
        }
    }
    if (active) Lbuf[(size_t)(p - p0) * L_stride + S.pix_off + pix] = acc;
}

template <int MODE, int G, bool EXACT, bool GQ>
__global__ void __launch_bounds__(256)
    k_trace_rows(const SysDev *__restrict__ sys, const int *__restrict__ comp_type,
                 const int *__restrict__ comp_plane, const float *__restrict__ cf,
                 const double *__restrict__ cd, const unsigned char *__restrict__ valid, int P,
                 int C_total, const TraceBlock *__restrict__ blocks, const int *__restrict__ need,
                 NodeTables nodes, int p0, float *__restrict__ Lbuf, long long L_stride,
                 FfQueue fq)
{
    trace_item<MODE, G, EXACT, GQ>(sys, comp_type, comp_plane, cf, cd, valid, P, C_total, need,
                                   nodes, p0, Lbuf, L_stride, fq, blocks[blockIdx.x],
                                   p0 + (int)blockIdx.y);
}

// The same work as a persistent, work-queued launch: a grid sized to the
// resident CTAs of the GPU takes (trace block, point) items, point-major,
// kPqGrab at a time from the counter *work (zeroed before the launch) until
// n_items are done, staging a point's constants only when the system or the
// point changes.
constexpr int kPqGrab = 4;
template <int MODE, int G, bool EXACT, bool GQ>
__global__ void __launch_bounds__(256)
    k_trace_rows_pq(const SysDev *__restrict__ sys, const int *__restrict__ comp_type,
                    const int *__restrict__ comp_plane, const float *__restrict__ cf,
                    const double *__restrict__ cd, const unsigned char *__restrict__ valid, int P,
                    int C_total, const TraceBlock *__restrict__ blocks,
                    const int *__restrict__ need, NodeTables nodes, int p0,
                    float *__restrict__ Lbuf, long long L_stride, FfQueue fq, int n_blocks,
                    long long n_items, unsigned long long *__restrict__ work)
{
    __shared__ long long s_item;
    int cur_sys = -1, cur_p = -1;
    for (;;) {
        if (threadIdx.x == 0) s_item = (long long)atomicAdd(work, (unsigned long long)kPqGrab);
        __syncthreads();
        const long long first = s_item;
        __syncthreads();  // read by all before thread 0 takes the next ones
        if (first >= n_items) return;
        const long long last = min(first + kPqGrab, n_items);
        for (long long item = first; item < last; ++item) {
            const int q = (int)(item / n_blocks);
            const TraceBlock tb = blocks[item - (long long)q * n_blocks];
            const int p = p0 + q;
            trace_item<MODE, G, EXACT, GQ>(sys, comp_type, comp_plane, cf, cd, valid, P, C_total,
                                           need, nodes, p0, Lbuf, L_stride, fq, tb, p,
                                           tb.sys != cur_sys || p != cur_p);
            cur_sys = tb.sys;
            cur_p = p;
            __syncthreads();  // the item is done with the shared arrays
        }
    }
}

constexpr int kFfThreads = 128;  // threads per CTA of the second-pass kernels

// MIXED_FF second pass, part 1: the pixels the trace kernel flagged.  One
// thread per pixel record (records of any system and point share a warp; the
// constants come from global memory) recomputes the pixel's sum with the rays
// near a source centre deferred -- the same loop and arithmetic as the
// in-block form -- and the warp reserves consecutive slots of the ray queue
// for its lanes' deferred rays (each pixel's in ray order), or, when they do
// not fit, marks its slots inside the queue empty and re-traces the rays
// itself, in ray order.
template <int G>
__global__ void __launch_bounds__(kFfThreads)
    k_refine_ff(const SysDev *__restrict__ sys, const int *__restrict__ comp_type,
                const int *__restrict__ comp_plane, const float *__restrict__ cf, int C_total,
                NodeTables nodes, int p0, unsigned L_stride, float *__restrict__ Lbuf, FfQueue fq)
{
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const long long n = min((long long)fq.cnt[1], fq.pcap);
    const long long wpb = blockDim.x / 32;
    for (long long e0 = (blockIdx.x * wpb + threadIdx.x / 32) * 32; e0 < n;
         e0 += (long long)gridDim.x * wpb * 32) {
        const long long e = e0 + lane;
        const bool active = e < n;
        unsigned lin = 0u, s = 0u;
        int pix = 0, p = p0;
        if (active) {
            const FfEntry R = fq.pix[e];
            lin = R.lin;
            s = R.sr;
            const unsigned q = lin / L_stride;
            pix = (int)(lin - q * L_stride) - sys[s].pix_off;
            p = p0 + (int)q;
        }
        const SysDev &S = sys[s];
        const int j = pix - (pix / S.nx) * S.nx, i = pix / S.nx;
        const float jc = (float)j - S.cx, ic = (float)i - S.cy;
        const GlobalConsts K{cf + ((size_t)p * C_total + S.comp_off) * kNC,
                             comp_type + S.comp_off, comp_plane + S.comp_off,
                             nodes.u + S.node_off, nodes.w + S.w2_off, nodes.ud + S.node_off};
        unsigned long long mask = 0ull;
        float acc = 0.f, pmin = kCuspRho2;
        if (active) {
            acc = (nodes.pre_f && S.pre_off >= 0) ? nodes.pre_f[S.pre_off + pix] : 0.f;
            acc = pixel_rays<LENSED_PREC_MIXED_FF, G, true, kNearDefer>(K, S, S.ncomp, G, jc, ic,
                                                                       acc, mask, pmin);
        }
        const int n_t = __popcll(mask);
        if (__any_sync(full, n_t != 0)) {
            int incl = n_t;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int v = __shfl_up_sync(full, incl, o);
                if (lane >= o) incl += v;
            }
            const int total = __shfl_sync(full, incl, 31);
            unsigned long long base = 0ull;
            if (lane == 31) base = atomicAdd(fq.cnt, (unsigned long long)total);
            base = __shfl_sync(full, base, 31);
            const unsigned long long cap = (unsigned long long)fq.ecap;
            unsigned long long q = base + (unsigned long long)(incl - n_t);
            if (base + (unsigned long long)total <= cap) {
                if (active) fq.prun[e] = make_uint2((unsigned)q, (unsigned)n_t);
                const unsigned sys8 = s << 8;
                for (unsigned long long m = mask; m; m &= m - 1ull, ++q)
                    fq.ent[q] = FfEntry{lin, sys8 | (unsigned)(__ffsll((long long)m) - 1)};
            } else {
                if (active) fq.prun[e] = make_uint2(0u, 0u);
                for (int k = 0; k < n_t; ++k, ++q)
                    if (q < cap) fq.ent[q] = FfEntry{kFfNone, 0u};
                for (unsigned long long m = mask; m; m &= m - 1ull) {
                    const int r = __ffsll((long long)m) - 1;
                    acc = fmaf(K.w(r), K.ff(S.ncomp, jc, ic, S.h, S.h_lo, r % G, r / G), acc);
                }
            }
        } else if (active) {
            fq.prun[e] = make_uint2(0u, 0u);
        }
        if (active) Lbuf[lin] = acc;
    }
}

// MIXED_FF second pass over a trace launch's global queue: one thread per
// entry (the rays of many warps and points fill whole warps here) reads its
// point's constants from global memory and writes the ray's source-plane
// brightness; k_apply_ff then adds each pixel's rays to its first-pass sum in
// ray order -- the same arithmetic in the same order as the in-block path.

// SMs of the current device, read once per model (sizes the second pass's
// persistent grid outside any stream capture)
static int g_sm_count = 0;

__global__ void __launch_bounds__(kFfThreads)
    k_retrace_ff(const SysDev *__restrict__ sys, const int *__restrict__ comp_type,
                 const int *__restrict__ comp_plane, const float *__restrict__ cf, int C_total,
                 NodeTables nodes, int p0, unsigned L_stride, FfQueue fq)
{
    const long long n = min((long long)*fq.cnt, fq.ecap);
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
         e += (long long)gridDim.x * blockDim.x) {
        const FfEntry E = fq.ent[e];
        if (E.lin == kFfNone) continue;
        const SysDev &S = sys[E.sr >> 8];
        const int r = (int)(E.sr & 255u), nn = S.nn;
        const unsigned q = E.lin / L_stride;
        const int pix = (int)(E.lin - q * L_stride) - S.pix_off;
        const int i = pix / S.nx, j = pix - i * S.nx;
        const int a = r % nn, b = r / nn;
        const FfConsts K{cf + ((size_t)(p0 + (int)q) * C_total + S.comp_off) * kNC,
                         comp_type + S.comp_off, comp_plane + S.comp_off};
        fq.val[e] = source_brightness_ff_at(K, S.ncomp, (float)j - S.cx, (float)i - S.cy, S.h,
                                            S.h_lo, node_pair(nodes.ud[S.node_off + a]),
                                            node_pair(nodes.ud[S.node_off + b]));
    }
}

// Each refined pixel's re-traced rays are added, in ray order, to the sum
// k_refine_ff stored: one thread per pixel record, its rays a contiguous
// slice of the queue.
__global__ void k_apply_ff(const SysDev *__restrict__ sys, NodeTables nodes,
                           float *__restrict__ Lbuf, FfQueue fq)
{
    const long long n = min((long long)fq.cnt[1], fq.pcap);
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
         e += (long long)gridDim.x * blockDim.x) {
        const uint2 run = fq.prun[e];
        if (run.y == 0u) continue;
        const FfEntry R = fq.pix[e];
        const int w2 = sys[R.sr].w2_off;
        float acc = Lbuf[R.lin];
        for (unsigned k = 0; k < run.y; ++k)
            acc = fmaf(nodes.w[w2 + (int)(fq.ent[run.x + k].sr & 255u)], fq.val[run.x + k], acc);
        Lbuf[R.lin] = acc;
    }
}

// a2-a5 in FP64 (validation mode): plain per-ray loop.
__global__ void __launch_bounds__(256)
    k_trace_f64(const SysDev *__restrict__ sys, const int *__restrict__ comp_type,
                const int *__restrict__ comp_plane, const float *__restrict__ cf,
                const double *__restrict__ cd, const unsigned char *__restrict__ valid, int P,
                int C_total, const TraceBlock *__restrict__ blocks, const int *__restrict__ need,
                NodeTables nodes, int p0, double *__restrict__ Lbuf, long long L_stride)
{
    __shared__ __align__(16) TraceSmem sm;
    const TraceBlock tb = blocks[blockIdx.x];
    const int p = p0 + blockIdx.y;
    if (!valid[(size_t)tb.sys * P + p]) return;
    const SysDev &S = sys[tb.sys];
    const size_t cbase = ((size_t)p * C_total + S.comp_off) * kNC;
    stage_point(sm, S, comp_type, comp_plane, cf, cd, cbase, true, true, nodes);
    __syncthreads();
    const int idx = tb.start + threadIdx.x;
    if (idx >= tb.end) return;
    RayCtx R{S.ncomp, sm.type, sm.plane, sm.cd};
    const int nn = S.nn, nx = S.nx;
    const int pix = need ? need[S.need_off + idx] : idx;
    const int i = pix / nx, j = pix - (pix / nx) * nx;
    const double xc = ((double)j - (double)S.cx) * S.hd;
    const double yc = ((double)i - (double)S.cy) * S.hd;
    double acc = (nodes.pre_d && S.pre_off >= 0) ? nodes.pre_d[S.pre_off + pix] : 0.0;
    for (int b = 0; b < nn; ++b) {
        const double y = yc + sm.ud[b];
        for (int a = 0; a < nn; ++a) acc += sm.wd[b * nn + a] * brightness_f64(xc + sm.ud[a], y, R);
    }
    Lbuf[(size_t)(p - p0) * L_stride + S.pix_off + pix] = acc;
}

// work == nullptr: one CTA per (trace block, point); else a persistent grid
// of as many CTAs as fit on the GPU at once, fed by the counter *work
template <int MODE, int G, bool EXACT, bool GQ>
static void trace_rows_t(int threads, const SysDev *sys, const int *comp_type,
                         const int *comp_plane, const float *cf, const double *cd,
                         const unsigned char *valid, int P, int C_total, const TraceBlock *blocks,
                         int n_blocks, const int *need, NodeTables nodes, int p0, int nP,
                         void *Lbuf, long long L_stride, cudaStream_t st, FfQueue fq,
                         unsigned long long *work)
{
    if (!work) {
        dim3 grid((unsigned)n_blocks, (unsigned)nP);
        k_trace_rows<MODE, G, EXACT, GQ><<<grid, threads, 0, st>>>(
            sys, comp_type, comp_plane, cf, cd, valid, P, C_total, blocks, need, nodes, p0,
            (float *)Lbuf, L_stride, fq);
        return;
    }
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_trace_rows_pq<MODE, G, EXACT, GQ>,
                                                  threads, 0);
    const long long n_items = (long long)n_blocks * nP;
    const long long want = (long long)std::max(g_sm_count, 1) * std::max(per_sm, 1);
    const unsigned grid = (unsigned)std::max(1LL, std::min(want, n_items));
    cudaMemsetAsync(work, 0, sizeof(unsigned long long), st);
    k_trace_rows_pq<MODE, G, EXACT, GQ><<<grid, threads, 0, st>>>(
        sys, comp_type, comp_plane, cf, cd, valid, P, C_total, blocks, need, nodes, p0,
        (float *)Lbuf, L_stride, fq, n_blocks, n_items, work);
}

// GQ: the launch has a global float-float queue (MIXED_FF, at most 8 nodes per row)
template <int MODE, bool GQ>
static void trace_rows_dispatch(int nn, int threads, const SysDev *sys, const int *comp_type,
                                const int *comp_plane, const float *cf, const double *cd,
                                const unsigned char *valid, int P, int C_total,
                                const TraceBlock *blocks, int n_blocks, const int *need,
                                NodeTables nodes, int p0, int nP, void *Lbuf, long long L_stride,
                                cudaStream_t st, FfQueue fq, unsigned long long *work)
{
#define LENSED_ROWS(GG, EX, Q)                                                                  \
    trace_rows_t<MODE, GG, EX, Q>(threads, sys, comp_type, comp_plane, cf, cd, valid, P, C_total, \
                                  blocks, n_blocks, need, nodes, p0, nP, Lbuf, L_stride, st, fq, \
                                  work)
    switch (nn) {
    case 1: LENSED_ROWS(1, true, GQ); break;
    case 2: LENSED_ROWS(2, true, GQ); break;
    case 3: LENSED_ROWS(3, true, GQ); break;
    case 4: LENSED_ROWS(4, true, GQ); break;
    case 5: LENSED_ROWS(5, true, GQ); break;
    case 6: LENSED_ROWS(6, true, GQ); break;
    case 7: LENSED_ROWS(7, true, GQ); break;
    case 8: LENSED_ROWS(8, true, GQ); break;
    default: LENSED_ROWS(4, false, false); break;
    }
#undef LENSED_ROWS
}

void launch_trace(int precision, LaunchCfg cfg, int nn, const SysDev *sys, const int *comp_type,
                  const int *comp_plane, const float *cf, const double *cd,
                  const unsigned char *valid, int P, int C_total, const TraceBlock *blocks,
                  int n_blocks, const int *need, NodeTables nodes, int p0, int nP, void *Lbuf,
                  long long L_stride, cudaStream_t st, FfQueue q, unsigned long long *work)
{
    if (n_blocks <= 0 || nP <= 0) return;
    if (!cfg.persistent) work = nullptr;
    if (precision == LENSED_PREC_FP64) {
        dim3 grid((unsigned)n_blocks, (unsigned)nP);
        k_trace_f64<<<grid, cfg.trace_threads, 0, st>>>(sys, comp_type, comp_plane, cf, cd,
                                                         valid, P, C_total, blocks, need, nodes,
                                                         p0, (double *)Lbuf, L_stride);
    } else if (precision == LENSED_PREC_MIXED_FF) {
        // the global queue needs the deferral mask, i.e. at most 8 nodes per
        // row, and 32-bit pixel indices into this launch's scratch
        const bool split = cfg.ff_split && q.cnt && q.ent && q.val && q.pix && q.prun && nn >= 1 &&
                           nn <= 8 &&
                           (long long)nP * L_stride < (long long)kFfNone;
        if (split) {
            cudaMemsetAsync(q.cnt, 0, 2 * sizeof(unsigned long long), st);
            trace_rows_dispatch<LENSED_PREC_MIXED_FF, true>(
                nn, cfg.trace_threads, sys, comp_type, comp_plane, cf, cd, valid, P, C_total,
                blocks, n_blocks, need, nodes, p0, nP, Lbuf, L_stride, st, q, work);
            const unsigned grid = (unsigned)std::max(1, g_sm_count) * 8;
#define LENSED_REFINE(GG)                                                                     \
    k_refine_ff<GG><<<grid, kFfThreads, 0, st>>>(sys, comp_type, comp_plane, cf, C_total, nodes, \
                                                 p0, (unsigned)L_stride, (float *)Lbuf, q)
            switch (nn) {
            case 1: LENSED_REFINE(1); break;
            case 2: LENSED_REFINE(2); break;
            case 3: LENSED_REFINE(3); break;
            case 4: LENSED_REFINE(4); break;
            case 5: LENSED_REFINE(5); break;
            case 6: LENSED_REFINE(6); break;
            case 7: LENSED_REFINE(7); break;
            default: LENSED_REFINE(8); break;
            }
#undef LENSED_REFINE
            k_retrace_ff<<<grid, kFfThreads, 0, st>>>(sys, comp_type, comp_plane, cf, C_total,
                                                     nodes, p0, (unsigned)L_stride, q);
            k_apply_ff<<<grid, kFfThreads, 0, st>>>(sys, nodes, (float *)Lbuf, q);
        } else {
            trace_rows_dispatch<LENSED_PREC_MIXED_FF, false>(
                nn, cfg.trace_threads, sys, comp_type, comp_plane, cf, cd, valid, P, C_total,
                blocks, n_blocks, need, nodes, p0, nP, Lbuf, L_stride, st, FfQueue{}, work);
        }
    } else {
        trace_rows_dispatch<LENSED_PREC_FP32, false>(nn, cfg.trace_threads, sys, comp_type,
                                                     comp_plane, cf, cd, valid, P, C_total, blocks,
                                                     n_blocks, need, nodes, p0, nP, Lbuf, L_stride,
                                                     st, FfQueue{}, work);
    }
}

// MIXED second pass.  One block per (system, point).  The MIXED rule puts
// the SIE in FP64 for every ray of a point whose SIE is nearly round
// (e < 0.05), and otherwise for the rays within 2 s / q of an SIE centre.
// The pixels holding such rays -- every listed pixel in the first case, the
// pixels whose square reaches the disc in the second -- are recomputed (that
// SIE in FP64, every other component in FP32) and overwrite the first pass.
// Work is spread one thread per (pixel, ray); each pixel then sums its rays in
// the fixed node order.

// Brightness of ray (a, b) of pixel (i, j) under the MIXED rule.
__device__ float ray_mixed(const TraceSmem &sm, const SysDev &S, int i, int j, int a, int b,
                          bool ff)
{
    const int ncomp = S.ncomp;
    const float jc = (float)j - S.cx, ic = (float)i - S.cy;
    const float x = fmaf(jc, S.h, jc * S.h_lo) + sm.u[a];
    const float y = fmaf(ic, S.h, ic * S.h_lo) + sm.u[b];
    float I = 0.f, ax = 0.f, ay = 0.f;
    for (int c = 0; c < ncomp; ++c) {
        const int pl = sm.plane[c];
        const float *cc = sm.cf + c * kNC;
        if (pl == LENSED_PLANE_FOREGROUND) {
            I += light_any_f32(load_light(cc), x, y);
        } else if (pl == LENSED_PLANE_LENS) {
            const int t = sm.type[c];
            if (t == LENSED_SIE) {
                const double *cd = sm.cd + c * kNC;
                bool use64 = cd[17] != 0.0;
                if (!use64) {
                    const double dx = (double)jc * S.hd + sm.ud[a] - cd[0];
                    const double dy = (double)ic * S.hd + sm.ud[b] - cd[1];
                    use64 = dx * dx + dy * dy < cd[18];
                }
                if (use64) sie_ray_f64(jc, ic, S.hd, sm.ud[a], sm.ud[b], cd, ax, ay);
                else sie_f32(load_sie(cc), x, y, ax, ay);
            } else if (t == LENSED_SHEAR) {
                const float dx = x - cc[0], dy = y - cc[1];
                ax += fmaf(cc[2], dx, cc[3] * dy);
                ay += fmaf(cc[3], dx, -cc[2] * dy);
            } else {
                const float dx = x - cc[0], dy = y - cc[1];
                const float r2 = fmaf(dx, dx, dy * dy);
                const float f = r2 > 0.f ? __fdividef(cc[2], r2) : 0.f;
                ax = fmaf(f, dx, ax);
                ay = fmaf(f, dy, ay);
            }
        }
    }
    const float Ifg = I;
    bool near = false;
    for (int c = 0; c < ncomp; ++c) {
        if (sm.plane[c] != LENSED_PLANE_SOURCE) continue;
        const LightF L = load_light(sm.cf + c * kNC);
        if (ff && L.kind == (float)kKindPower) {
            float r2;
            I += light_f32_rho(L, x - ax, y - ay, r2);
            near = near || r2 < kCuspRho2;
        } else {
            I += light_any_f32(L, x - ax, y - ay);
        }
    }
    if (near) I = Ifg + source_brightness_ff(sm, ncomp, jc, ic, S.h, S.h_lo, a, b);
    return I;
}

// Does pixel (i, j)'s square reach within sqrt(r2) of (x0, y0)?
__device__ __forceinline__ bool pixel_near(const SysDev &S, int i, int j, double x0, double y0,
                                           double r2)
{
    const double xc = ((double)j - (double)S.cx) * S.hd, yc = ((double)i - (double)S.cy) * S.hd;
    const double dx = fmax(fabs(xc - x0) - 0.5 * S.hd, 0.0);
    const double dy = fmax(fabs(yc - y0) - 0.5 * S.hd, 0.0);
    return dx * dx + dy * dy < r2;
}

constexpr int kFixRays = 1024;  // ray contributions staged per batch

// Recompute the pixels of s_pix[0..n) (batches of kFixRays / (nn*nn)).
__device__ void fix_pixels(const TraceSmem &sm, const SysDev &S, const int *s_pix, int n,
                           float *s_ray, float *L, const float *pre, bool ff)
{
    const int nn = S.nn, nr = nn * nn, nx = S.nx;
    const int per = kFixRays / nr;
    for (int b0 = 0; b0 < n; b0 += per) {
        const int m = min(per, n - b0);
        for (int t = threadIdx.x; t < m * nr; t += blockDim.x) {
            const int pix = s_pix[b0 + t / nr], r = t % nr;
            const int i = pix / nx, j = pix - (pix / nx) * nx;
            s_ray[t] = ray_mixed(sm, S, i, j, r % nn, r / nn, ff);
        }
        __syncthreads();
        for (int k = threadIdx.x; k < m; k += blockDim.x) {
            float acc = pre ? pre[s_pix[b0 + k]] : 0.f;
            for (int r = 0; r < nr; ++r) acc = fmaf(sm.w[r], s_ray[k * nr + r], acc);
            L[s_pix[b0 + k]] = acc;
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(128)
    k_trace_fix64(const SysDev *__restrict__ sys, int s0, const int *__restrict__ comp_type,
                  const int *__restrict__ comp_plane, const float *__restrict__ cf,
                  const double *__restrict__ cd, const unsigned char *__restrict__ valid, int P,
                  int C_total, const int *__restrict__ need, NodeTables nodes, int p0,
                  float *__restrict__ Lbuf, long long L_stride)
{
    __shared__ __align__(16) TraceSmem sm;
    __shared__ float s_ray[kFixRays];
    __shared__ int s_pix[kFixRays];
    __shared__ int s_n;
    const int s = s0 + blockIdx.x;
    const int p = p0 + blockIdx.y;
    if (!valid[(size_t)s * P + p]) return;
    const SysDev &S = sys[s];
    const size_t cbase = ((size_t)p * C_total + S.comp_off) * kNC;
    stage_point(sm, S, comp_type, comp_plane, cf, cd, cbase, true, false, nodes);
    __syncthreads();
    const int ncomp = S.ncomp, nx = S.nx, ny = S.ny;
    float *L = Lbuf + (size_t)(p - p0) * L_stride + S.pix_off;
    const float *pre = (nodes.pre_f && S.pre_off >= 0) ? nodes.pre_f + S.pre_off : nullptr;
    bool whole = false;
    for (int c = 0; c < ncomp; ++c)
        if (sm.type[c] == LENSED_SIE && sm.cd[c * kNC + 17] != 0.0) whole = true;
    if (whole) {
        // every listed pixel, in slices of kFixRays
        const int n = need ? S.n_need : S.npix;
        for (int q0 = 0; q0 < n; q0 += kFixRays) {
            const int m = min(kFixRays, n - q0);
            for (int k = threadIdx.x; k < m; k += blockDim.x)
                s_pix[k] = need ? need[S.need_off + q0 + k] : q0 + k;
            __syncthreads();
            fix_pixels(sm, S, s_pix, m, s_ray, L, pre, nodes.ff != 0);
        }
        return;
    }
    // core discs, one SIE after the other; a pixel already covered by an
    // earlier SIE's disc is skipped so every pixel is written once
    for (int c = 0; c < ncomp; ++c) {
        if (sm.type[c] != LENSED_SIE) continue;
        const double *cc = sm.cd + c * kNC;
        const double r = sqrt(cc[18]);
        if (!(r > 0.0)) continue;
        const int j0 = max(0, (int)floor((cc[0] - r) / S.hd + S.cx - 1.0));
        const int j1 = min(nx - 1, (int)ceil((cc[0] + r) / S.hd + S.cx + 1.0));
        const int i0 = max(0, (int)floor((cc[1] - r) / S.hd + S.cy - 1.0));
        const int i1 = min(ny - 1, (int)ceil((cc[1] + r) / S.hd + S.cy + 1.0));
        if (j1 < j0 || i1 < i0) continue;
        const int bw = j1 - j0 + 1, nbox = bw * (i1 - i0 + 1);
        for (int q0 = 0; q0 < nbox; q0 += kFixRays) {
            if (threadIdx.x == 0) s_n = 0;
            __syncthreads();
            for (int idx = q0 + threadIdx.x; idx < min(nbox, q0 + kFixRays); idx += blockDim.x) {
                const int i = i0 + idx / bw, j = j0 + idx % bw;
                if (!pixel_near(S, i, j, cc[0], cc[1], cc[18])) continue;
                bool earlier = false;
                for (int c2 = 0; c2 < c; ++c2) {
                    const double *c2c = sm.cd + c2 * kNC;
                    if (sm.type[c2] == LENSED_SIE && pixel_near(S, i, j, c2c[0], c2c[1], c2c[18]))
                        earlier = true;
                }
                if (!earlier) s_pix[atomicAdd(&s_n, 1)] = i * nx + j;
            }
            __syncthreads();
            const int n = s_n;
            __syncthreads();
            fix_pixels(sm, S, s_pix, n, s_ray, L, pre, nodes.ff != 0);
        }
    }
}

void launch_fix64(LaunchCfg cfg, const SysDev *sys, int s0, int nS, const int *comp_type,
                  const int *comp_plane, const float *cf, const double *cd,
                  const unsigned char *valid, int P, int C_total, const int *need,
                  NodeTables nodes, int p0, int nP, void *Lbuf, long long L_stride,
                  cudaStream_t st)
{
    (void)cfg;
    if (nS <= 0 || nP <= 0) return;
    dim3 grid((unsigned)nS, (unsigned)nP);
    k_trace_fix64<<<grid, 128, 0, st>>>(sys, s0, comp_type, comp_plane, cf, cd, valid, P, C_total,
                                         need, nodes, p0, (float *)Lbuf, L_stride);
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

// The separable kernel's strides.  Staged tile: psf_row_stride with an odd
// number of 16-byte quads, so the two rows one 8-lane phase of its row pass
// reads fall on different banks.  Row-pass output: 72 floats, 18 quads (2
// mod 8), so the 4 rows x 2 interleaved quads of a column-pass phase do too.
static __host__ __device__ __forceinline__ int psf_sep_row_stride(int q)
{
    return psf_row_stride(q) | 4;
}
constexpr int kHStride = kTileW + 8;

// Row stride of the staged PSF: 2q+1 taps rounded up to a multiple of 4 so
// each row starts 16-byte aligned.
static __host__ __device__ __forceinline__ int psf_tap_stride(int q) { return (2 * q + 1 + 3) & ~3; }

// Asynchronous global -> shared copy of one element (cp.async, cached in
// L1: neighbouring tiles read the same halo), and the wait for all of a
// thread's copies.
__device__ __forceinline__ void cp_async_elem(float *dst, const float *src)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_elem(double *dst, const double *src)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all()
{
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;" ::: "memory");
}

// Stage rows x cols of an image into shared memory (row stride `stride`),
// from image row i0 and column j0 on, indices clamped to the image (Eq. 15's
// edge padding): one warp per row, consecutive lanes on consecutive columns
// (coalesced), no integer division.  The copies are asynchronous, so every
// load of the tile is in flight at once; the caller's barrier follows.
template <typename T>
__device__ __forceinline__ void stage_tile(T *s, int stride, const T *__restrict__ L, int nx,
                                           int ny, int i0, int j0, int rows, int cols)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int r = warp; r < rows; r += (int)(blockDim.x >> 5)) {
        const T *src = L + (size_t)min(max(i0 + r, 0), ny - 1) * nx;
        T *dst = s + r * stride;
        for (int c = lane; c < cols; c += 32) cp_async_elem(dst + c, src + min(max(j0 + c, 0), nx - 1));
    }
    cp_async_wait_all();
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
    constexpr int WS = (W + 3) & ~3;  // padded tap row
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

    // stage the flipped, normalised PSF (rows padded to WS) and the clamped
    // tile + halo
    for (int k = threadIdx.x; k < (2 * Ph + 1) * WS; k += blockDim.x) {
        const int r = k / WS, c = k - (k / WS) * WS;
        s_F[k] = c < W ? psf[S.psf_off + r * W + c] : T(0);
    }
    const T *L = Lbuf + (size_t)(p - p0) * L_stride + S.pix_off;
    stage_tile(s_L, stride, L, nx, ny, pb.i0 - Ph, pb.j0 - Q, rows, kTileW + 2 * Q);
    __syncthreads();

    // each warp owns a 16 x 16 block of outputs (the tile is 2 x 4 warps);
    // each lane 8 consecutive outputs of one row
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tr = (warp >> 2) * 16 + (lane >> 1);
    const int tcol = (warp & 3) * 16 + (lane & 1) * kOutPerThread;
    const int i = pb.i0 + tr;
    const int jb = pb.j0 + tcol;
    // chi^2 mode: a warp none of whose outputs carries weight skips the
    // convolution (its partial is zero)
    const bool live = !partial || ((pb.live_warps >> warp) & 1u);
    T acc[kOutPerThread];
#pragma unroll
    for (int o = 0; o < kOutPerThread; ++o) acc[o] = T(0);
    for (int kk = 0; live && kk <= 2 * Ph; ++kk) {
        T f[WS];
#pragma unroll
        for (int l = 0; l < WS; ++l) f[l] = s_F[kk * WS + l];
        const T *srow = s_L + (tr + kk) * stride + tcol;
        T lv[kOutPerThread + 2 * Q];
#pragma unroll
        for (int m = 0; m < kOutPerThread + 2 * Q; ++m) lv[m] = srow[m];
        // each PSF row is summed on its own and then added to the output: the
        // float rounding of the sum grows like sqrt(rows) + sqrt(taps per
        // row) instead of sqrt(all taps), which on a 21 x 21 PSF cuts its
        // share of the log-likelihood error ~5x for 5 % more additions
#pragma unroll
        for (int o = 0; o < kOutPerThread; ++o) {
            T part = T(0);
#pragma unroll
            for (int l = 0; l < W; ++l) part += f[l] * lv[o + l];
            acc[o] += part;
        }
    }

    if (partial) {
        double chi = 0.0;
        if (live && i < ny) {
#pragma unroll
            for (int o = 0; o < kOutPerThread; ++o) {
                const int j = jb + o;
                if (j < nx) {
                    const size_t pix = S.pix_off + (size_t)i * nx + j;
                    const T w = weight[pix];
                    if (w > T(0)) {
                        // one product per pixel in the working precision,
                        // accumulated in FP64
                        const T r = data[pix] - acc[o];
                        chi += (double)(w * r * r);
                    }
                }
            }
        }
        // warp-shuffle tree, then across the 8 warps in fixed order
        __shared__ double s_red[kPsfThreads / 32];
        chi = warp_sum(chi);
        if (lane == 0) s_red[warp] = chi;
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

// a6-a7 with a PSF of low numerical rank, F = sum_k c_k r_k^T (FP32 modes):
// the staged tile + halo is convolved along rows with each r_k (pass 1, into
// shared memory), then along columns with c_k (pass 2), which is the same
// two-dimensional sum of Eq. 15 on the clamped tile, in (2q+1)(32+2p)/32 +
// (2p+1) multiply-adds per term and output instead of (2p+1)(2q+1).  The
// output mapping, the warp skip and the chi^2 reduction are those of k_psf.
template <int Q>
__global__ void __launch_bounds__(kPsfThreads, 4)
    k_psf_sep(const SysDev *__restrict__ sys, const float *__restrict__ psf,
              const float *__restrict__ data, const float *__restrict__ weight,
              const unsigned char *__restrict__ valid, int P, const PsfBlock *__restrict__ blocks,
              int p0, const float *__restrict__ Lbuf, long long L_stride,
              double *__restrict__ partial, int T_total, float *__restrict__ out)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int W = 2 * Q + 1;
    constexpr int WS = (W + 3) & ~3;
    const PsfBlock pb = blocks[blockIdx.x];
    const int p = p0 + blockIdx.y;
    const SysDev &S = sys[pb.sys];
    const bool ok = valid[(size_t)pb.sys * P + p] != 0;
    const int Ph = S.psf_p, R = S.psf_rank;
    const int rows = kTileH + 2 * Ph;
    const int stride = psf_sep_row_stride(Q);
    const int nx = S.nx, ny = S.ny;
    float *s_L = reinterpret_cast<float *>(smem_raw);
    float *s_H = s_L + (size_t)rows * stride;        // [R][rows][kHStride]
    float *s_c = s_H + (size_t)R * rows * kHStride;  // [R][2p+1]
    float *s_r = s_c + R * (2 * Ph + 1);             // [R][WS]

    if (!ok) {
        if (out) {
            for (int k = threadIdx.x; k < kTileW * kTileH; k += blockDim.x) {
                const int i = pb.i0 + k / kTileW, j = pb.j0 + k % kTileW;
                if (i < ny && j < nx) out[(size_t)i * nx + j] = __int_as_float(0x7fc00000);
            }
        }
        return;
    }
    const float *fac = psf + S.psf_sep_off;
    const int nf = 2 * Ph + 1 + W;
    for (int k = threadIdx.x; k < R * (2 * Ph + 1); k += blockDim.x)
        s_c[k] = fac[(k / (2 * Ph + 1)) * nf + k % (2 * Ph + 1)];
    for (int k = threadIdx.x; k < R * WS; k += blockDim.x) {
        const int t = k / WS, l = k - (k / WS) * WS;
        s_r[k] = l < W ? fac[t * nf + 2 * Ph + 1 + l] : 0.f;
    }
    const float *L = Lbuf + (size_t)(p - p0) * L_stride + S.pix_off;
    stage_tile(s_L, stride, L, nx, ny, pb.i0 - Ph, pb.j0 - Q, rows, kTileW + 2 * Q);
    __syncthreads();

    // pass 1: rows, kOutPerThread outputs per item.  A warp takes 4 rows x 8
    // segments; each 8-lane phase 2 adjacent rows x 4 segments.
    constexpr int kSeg = kTileW / kOutPerThread;
    static_assert(kSeg == 8 && kPsfThreads == 256, "row-pass mapping");
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int phase = lane >> 3;
    const int seg = 4 * (phase >> 1) + (lane & 3);
    const int rgrp = warp * 4 + 2 * (phase & 1) + ((lane >> 2) & 1);
    for (int t = 0; t < R; ++t)
    for (int r = rgrp; r < rows; r += kPsfThreads / kSeg) {
        if (partial) {
            // chi^2 mode: staged row r feeds output rows r - 2p .. r; skip it
            // when none of them carries a weighted pixel
            const int lo = max(0, r - 2 * Ph), n = min(kTileH - 1, r) - lo + 1;
            const unsigned win = n >= 32 ? ~0u : (1u << n) - 1u;
            if (n <= 0 || ((pb.live_rows >> lo) & win) == 0u) continue;
        }
        const int j0 = seg * kOutPerThread;
        const float *srow = s_L + r * stride + j0;
        float lv[kOutPerThread + 2 * Q];
#pragma unroll
        for (int m = 0; m < kOutPerThread + 2 * Q; ++m) lv[m] = srow[m];
        float acc[kOutPerThread];
#pragma unroll
        for (int o = 0; o < kOutPerThread; ++o) acc[o] = 0.f;
#pragma unroll
        for (int l = 0; l < W; ++l) {
            const float f = s_r[t * WS + l];
#pragma unroll
            for (int o = 0; o < kOutPerThread; ++o) acc[o] = fmaf(f, lv[o + l], acc[o]);
        }
        float4 *h = reinterpret_cast<float4 *>(s_H + ((size_t)t * rows + r) * kHStride + j0);
        h[0] = make_float4(acc[0], acc[1], acc[2], acc[3]);
        h[1] = make_float4(acc[4], acc[5], acc[6], acc[7]);
    }
    __syncthreads();

    // pass 2: columns.  Warp w owns the 16 x 16 outputs of k_psf's warp w;
    // a lane 8 outputs of one row, in two quads 8 columns apart (columns
    // jb + 0..3 and jb + 8..11)
    const int tr = (warp >> 2) * 16 + (lane >> 1);
    const int tq = (warp & 3) * 16 + (lane & 1) * 4;
    const int i = pb.i0 + tr;
    const int jb = pb.j0 + tq;
    const bool live = !partial || ((pb.live_warps >> warp) & 1u);
    // chi^2 mode: the epilogue's data and weights, loaded before the sums
    float dv[kOutPerThread], wv[kOutPerThread];
#pragma unroll
    for (int o = 0; o < kOutPerThread; ++o) {
        const int j = jb + (o & 3) + 8 * (o >> 2);
        const bool in = partial && live && i < ny && j < nx;
        const size_t pix = S.pix_off + (size_t)i * nx + j;
        wv[o] = in ? weight[pix] : 0.f;
        dv[o] = in ? data[pix] : 0.f;
    }
    float acc[kOutPerThread];
#pragma unroll
    for (int o = 0; o < kOutPerThread; ++o) acc[o] = 0.f;
    for (int t = 0; live && t < R; ++t) {
        for (int m = 0; m <= 2 * Ph; ++m) {
            const float c = s_c[t * (2 * Ph + 1) + m];
            const float *hr = s_H + ((size_t)t * rows + tr + m) * kHStride + tq;
            const float4 a = *reinterpret_cast<const float4 *>(hr);
            const float4 b = *reinterpret_cast<const float4 *>(hr + 8);
            acc[0] = fmaf(c, a.x, acc[0]);
            acc[1] = fmaf(c, a.y, acc[1]);
            acc[2] = fmaf(c, a.z, acc[2]);
            acc[3] = fmaf(c, a.w, acc[3]);
            acc[4] = fmaf(c, b.x, acc[4]);
            acc[5] = fmaf(c, b.y, acc[5]);
            acc[6] = fmaf(c, b.z, acc[6]);
            acc[7] = fmaf(c, b.w, acc[7]);
        }
    }

    if (partial) {
        double chi = 0.0;
#pragma unroll
        for (int o = 0; o < kOutPerThread; ++o) {
            if (wv[o] > 0.f) {
                const float r = dv[o] - acc[o];
                chi += (double)(wv[o] * r * r);
            }
        }
        __shared__ double s_red[kPsfThreads / 32];
        chi = warp_sum(chi);
        if (lane == 0) s_red[warp] = chi;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int w = 0; w < kPsfThreads / 32; ++w) t += s_red[w];
            partial[(size_t)p * T_total + pb.tile] = t;
        }
    } else if (out && i < ny) {
#pragma unroll
        for (int o = 0; o < kOutPerThread; ++o) {
            const int j = jb + (o & 3) + 8 * (o >> 2);
            if (j < nx) out[(size_t)i * nx + j] = acc[o];
        }
    }
}

// Largest dynamic shared memory of a k_psf_sep instance (P = Q = 15, rank 3).
static constexpr int kPsfSepSmemMax =
    ((kTileH + 2 * LENSED_MAX_PSF_HALF) * (((kTileW + 2 * LENSED_MAX_PSF_HALF + 3) & ~3) | 4) +
     3 * (kTileH + 2 * LENSED_MAX_PSF_HALF) * kHStride + 3 * (2 * LENSED_MAX_PSF_HALF + 1) +
     3 * ((2 * LENSED_MAX_PSF_HALF + 1 + 3) & ~3)) *
    (int)sizeof(float);

// Largest dynamic shared memory a k_psf instance can ask for (Q = P = 15, FP64).
static constexpr int kPsfSmemMax =
    ((kTileH + 2 * LENSED_MAX_PSF_HALF) * ((kTileW + 2 * LENSED_MAX_PSF_HALF + 3) & ~3) +
     (2 * LENSED_MAX_PSF_HALF + 1) * ((2 * LENSED_MAX_PSF_HALF + 1 + 3) & ~3)) *
    (int)sizeof(double);

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

template <int... Qs>
static void psf_sep_attr_all(std::integer_sequence<int, Qs...>)
{
    (cudaFuncSetAttribute(k_psf_sep<Qs>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                          kPsfSepSmemMax),
     ...);
}

// Reduction tables of the float-float atan / atanh (long double on the host).
static void init_ff_tables()
{
    float t[27][2], th[128][2];
    for (int k = 0; k < 27; ++k) {
        const long double v = tanl(k / 16.0L);
        t[k][0] = (float)v;
        t[k][1] = (float)(v - (long double)t[k][0]);
    }
    for (int k = 0; k < 128; ++k) {
        const long double v = tanhl(k / 16.0L);
        th[k][0] = (float)v;
        th[k][1] = (float)(v - (long double)th[k][0]);
    }
    cudaMemcpyToSymbol(kTan16, t, sizeof(t));
    cudaMemcpyToSymbol(kTanh16, th, sizeof(th));
}

void init_kernel_attributes()
{
    int dev = 0;
    if (cudaGetDevice(&dev) == cudaSuccess)
        cudaDeviceGetAttribute(&g_sm_count, cudaDevAttrMultiProcessorCount, dev);
    init_ff_tables();
    psf_attr_all<float>(std::make_integer_sequence<int, LENSED_MAX_PSF_HALF + 1>{});
    psf_attr_all<double>(std::make_integer_sequence<int, LENSED_MAX_PSF_HALF + 1>{});
    psf_sep_attr_all(std::make_integer_sequence<int, LENSED_MAX_PSF_HALF + 1>{});
}

// Separable launches: the group's largest p and rank size the shared memory.
template <int Q>
static void psf_sep_launch_t(int p_max, int r_max, const SysDev *sys, const float *psf,
                             const float *data, const float *weight, const unsigned char *valid,
                             int P, const PsfBlock *blocks, int n_blocks, int p0, int nP,
                             const float *Lbuf, long long L_stride, double *partial, int T_total,
                             float *out, cudaStream_t st)
{
    const int rows = kTileH + 2 * p_max;
    const size_t smem = ((size_t)rows * psf_sep_row_stride(Q) + (size_t)r_max * rows * kHStride +
                         (size_t)r_max * (2 * p_max + 1) + (size_t)r_max * psf_tap_stride(Q)) *
                        sizeof(float);
    dim3 grid((unsigned)n_blocks, (unsigned)nP);
    k_psf_sep<Q><<<grid, kPsfThreads, smem, st>>>(sys, psf, data, weight, valid, P, blocks, p0,
                                                   Lbuf, L_stride, partial, T_total, out);
}

template <int... Qs>
static void psf_sep_dispatch(std::integer_sequence<int, Qs...>, int q, int p_max, int r_max,
                             const SysDev *sys, const float *psf, const float *data,
                             const float *weight, const unsigned char *valid, int P,
                             const PsfBlock *blocks, int n_blocks, int p0, int nP,
                             const float *Lbuf, long long L_stride, double *partial,
                             int T_total, float *out, cudaStream_t st)
{
    ((q == Qs ? psf_sep_launch_t<Qs>(p_max, r_max, sys, psf, data, weight, valid, P, blocks,
                                     n_blocks, p0, nP, Lbuf, L_stride, partial, T_total, out, st)
              : void()),
     ...);
}

template <typename T, int Q>
static void psf_launch_t(int p_max, const SysDev *sys, const T *psf, const T *data,
                         const T *weight, const unsigned char *valid, int P,
                         const PsfBlock *blocks, int n_blocks, int p0, int nP, const T *Lbuf,
                         long long L_stride, double *partial, int T_total, float *out,
                         cudaStream_t st)
{
    const size_t smem = ((size_t)(kTileH + 2 * p_max) * psf_row_stride(Q) +
                         (size_t)(2 * p_max + 1) * psf_tap_stride(Q)) * sizeof(T);
    dim3 grid((unsigned)n_blocks, (unsigned)nP);
    k_psf<T, Q><<<grid, kPsfThreads, smem, st>>>(sys, psf, data, weight, valid, P, blocks, p0,
                                                  Lbuf, L_stride, partial, T_total, out);
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

void launch_psf(int precision, int q, int sep, int p_max, const SysDev *sys, const float *psf_f,
                const double *psf_d, const float *data, const float *weight,
                const double *data_d, const double *weight_d,
                const unsigned char *valid, int P, const PsfBlock *blocks, int n_blocks, int p0,
                int nP, const void *Lbuf, long long L_stride, double *partial, int T_total,
                float *out, cudaStream_t st)
{
    if (n_blocks <= 0 || nP <= 0) return;
    if (sep > 0 && precision != LENSED_PREC_FP64)
        psf_sep_dispatch(std::make_integer_sequence<int, LENSED_MAX_PSF_HALF + 1>{}, q, p_max,
                         sep, sys, psf_f, data, weight, valid, P, blocks, n_blocks, p0, nP,
                         (const float *)Lbuf, L_stride, partial, T_total, out, st);
    else if (precision == LENSED_PREC_FP64)
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
        v = -0.5 * (S.wscale * t);  // the partials use the relative weights
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

__global__ void k_error_image(int fp64, const void *__restrict__ LK, const void *__restrict__ LG,
                              long long off, int npix, const unsigned char *__restrict__ valid,
                              float *__restrict__ out)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= npix) return;
    if (!valid[0]) {
        out[k] = __int_as_float(0x7fc00000);
        return;
    }
    out[k] = fp64 ? (float)fabs(((const double *)LK)[off + k] - ((const double *)LG)[off + k])
                  : fabsf(((const float *)LK)[off + k] - ((const float *)LG)[off + k]);
}

void launch_error_image(int precision, const void *LK, const void *LG, long long off, int npix,
                        const unsigned char *valid, float *out, cudaStream_t st)
{
    k_error_image<<<(npix + 255) / 256, 256, 0, st>>>(precision == LENSED_PREC_FP64, LK, LG, off,
                                                       npix, valid, out);
}

}  // namespace lensed
