// Host runtime of the ray-tracing likelihood: the C ABI of include/lensed.h.
//
// lensed_create_model validates the systems, prepares the per-pixel data,
// weights and the normalised PSF (Sec. 3.1-3.3; low-rank PSFs also as
// separable factors), the quadrature tables (Eq. 14; Gauss-Legendre and
// Gauss-Kronrod nodes computed here) and the work lists, copies them to the
// device, and integrates the lights that no parameter moves once.  The
// evaluation calls schedule the kernels of lensed_kernels.cu:
//
//   batched:  prologue(all points) -> for each point chunk: trace (and, in
//             MIXED_FF when the configuration asks for it, the second pass
//             of the float-float re-traces), the MIXED fix-up, psf ->
//             finalize, captured once per (P, pointers, launch
//             configuration) into a CUDA graph and replayed with one graph
//             launch;
//   plain:    for each system and point: prologue, trace, fix-up, psf,
//             finalize, each a separate launch (the per-point scheduling of
//             the paper's code), no graph.
//
// Both do the same arithmetic in the same order on the same per-pixel work,
// so their results are bit-identical.
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <atomic>
#include <mutex>
#include <string>
#include <vector>

#include "lensed_internal.cuh"

using namespace lensed;

// Allocation-failure injection for tests (lensed_debug_fail_alloc): -1 off,
// else how many more device allocations may succeed before every later one
// is refused.
static std::atomic<long long> g_alloc_budget{-1};
// Device buffers the library holds (models and networks), for leak checks.
static std::atomic<long long> g_live_buffers{0};

void lensed::note_buffers(int delta) { g_live_buffers += delta; }

bool lensed::alloc_failure_injected()
{
    long long b = g_alloc_budget.load();
    while (b >= 0) {
        if (b == 0) return true;
        if (g_alloc_budget.compare_exchange_weak(b, b - 1)) return false;
    }
    return false;
}

namespace {

thread_local std::string g_last_error;

int fail(int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return code;
}

#define CUDA_OK(call)                                                                       \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess)                                                              \
            return fail(e_ == cudaErrorMemoryAllocation ? LENSED_E_NOMEM : LENSED_E_CUDA,   \
                        "%s: %s", #call, cudaGetErrorString(e_));                           \
    } while (0)

// Algorithmic operation count of one ray through a component, counted from
// the formulas (add/sub/mul/div/sqrt/transcendental = 1, a multiply-add
// pair = 2) -- not from the compiled code.  {flops, transcendentals}:
//   SIE: translate 2, rotate 6, psi 6 (incl. sqrt), two quotients 4, e*z 2,
//        atan + atanh 2, prefactor 2, rotate back 6, accumulate 2 -> 32, 3
//   shear / point mass: translate 2, two linear forms 6 / r^2 3 + div 1 +
//        scale 2, accumulate 2 -> 10, 0
//   Sersic-type light: translate 2, rotate 6, R^2 5, log2 1, scale+shift 2,
//        exp2 1, negate+exp2 2, amplitude 1, accumulate 1 -> 21, 3
//   Gaussian light: translate 2, rotate 6, R^2 5, scale 1, negate+exp2 2,
//        amplitude 1, accumulate 1 -> 18, 1
//   per ray: position 2, lens equation 2, weight product + accumulate 2 -> 6
// MIXED and MIXED_FF both run the FP64 SIE fix-up pass.
bool is_mixed(int precision)
{
    return precision == LENSED_PREC_MIXED || precision == LENSED_PREC_MIXED_FF;
}

void component_ops(int type, double &flops, double &transc)
{
    switch (type) {
    case LENSED_SIE: flops += 32; transc += 3; break;
    case LENSED_SHEAR: flops += 10; break;
    case LENSED_POINTMASS: flops += 10; break;
    case LENSED_GAUSS: flops += 18; transc += 1; break;
    case LENSED_SKY: flops += 1; break;
    default: flops += 21; transc += 3; break;
    }
}

int nparams_of(int type)
{
    switch (type) {
    case LENSED_SIE: return 6;
    case LENSED_SHEAR: return 4;
    case LENSED_POINTMASS: return 3;
    case LENSED_SERSIC: return 7;
    case LENSED_DEVAUC: return 6;
    case LENSED_GAUSS: return 6;
    case LENSED_SKY: return 1;
    }
    return -1;
}

// Gauss-Legendre nodes on [-1, 1] by Newton's method on P_n with the
// three-term recurrence, started from the Tricomi estimate; long double.
void gauss_legendre(int n, std::vector<double> &x, std::vector<double> &w)
{
    x.assign(n, 0.0);
    w.assign(n, 0.0);
    const long double pi = 3.141592653589793238462643383279502884L;
    for (int i = 0; i < (n + 1) / 2; ++i) {
        long double z = cosl(pi * (i + 0.75L) / (n + 0.5L)), dp = 0;
        for (int it = 0; it < 100; ++it) {
            long double p0 = 1, p1 = z;
            for (int k = 2; k <= n; ++k) {
                long double p2 = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            if (n == 1) { p1 = z; p0 = 1; }
            dp = n * (z * p1 - p0) / (z * z - 1);
            long double dz = p1 / dp;
            z -= dz;
            if (fabsl(dz) < 1e-19L) break;
        }
        // recompute the derivative at the converged root
        long double p0 = 1, p1 = z;
        for (int k = 2; k <= n; ++k) {
            long double p2 = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k;
            p0 = p1;
            p1 = p2;
        }
        dp = (n == 1) ? 1.0L : n * (z * p1 - p0) / (z * z - 1);
        const long double wt = 2 / ((1 - z * z) * dp * dp);
        x[n - 1 - i] = (double)z;
        x[i] = (double)-z;
        w[i] = w[n - 1 - i] = (double)wt;
    }
    if (n % 2 == 1) x[n / 2] = 0.0;
}

// Regularised lower incomplete gamma P(a, x) by its power series, long
// double, summed as one fraction (host side, for the b_n table).
long double host_gamma_p(long double a, long double x)
{
    if (x <= 0) return 0;
    long double N = 1, D = 1, xk = 1;
    for (int k = 1; k < 2000; ++k) {
        const long double f = a + k;
        xk *= x;
        N = N * f + xk;
        D *= f;
        if (xk < 1e-21L * N) break;
        if (D > 1e300L) {
            N *= 1e-300L;
            D *= 1e-300L;
            xk *= 1e-300L;
        }
    }
    return expl(a * logl(x) - x - lgammal(a + 1)) * (N / D);
}

// Sersic b_n (root of P(2n, b) = 1/2) by bisection in long double.
double host_sersic_b(double n)
{
    long double lo = 0, hi = 2.0L * n;
    for (int it = 0; it < 200; ++it) {
        const long double mid = 0.5L * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        if (host_gamma_p(2.0L * n, mid) < 0.5L) lo = mid;
        else hi = mid;
    }
    return (double)(0.5L * (lo + hi));
}

// Piecewise Chebyshev coefficients of b_n in log n (kBnSeg segments of
// degree kBnDeg over [kBnMin, kBnMax]), from values at the Chebyshev points.
std::vector<double> build_bn_table()
{
    std::vector<double> tab(kBnSeg * (kBnDeg + 1));
    const double l0 = log(kBnMin), dl = (log(kBnMax) - l0) / kBnSeg;
    const int N = kBnDeg + 1;
    const long double pi = 3.141592653589793238462643383279502884L;
    for (int k = 0; k < kBnSeg; ++k) {
        std::vector<long double> f(N);
        for (int i = 0; i < N; ++i) {
            const long double t = cosl(pi * (i + 0.5L) / N);
            f[i] = host_sersic_b((double)expl(l0 + dl * (k + 0.5L * (t + 1))));
        }
        for (int j = 0; j < N; ++j) {
            long double c = 0;
            for (int i = 0; i < N; ++i) c += f[i] * cosl(pi * j * (i + 0.5L) / N);
            c *= 2.0L / N;
            if (j == 0) c *= 0.5L;
            tab[k * N + j] = (double)c;
        }
    }
    return tab;
}

// Integral of x^k P_n(x) over [-1, 1]: zero unless k >= n and k - n even,
// then 2^(n+1) k! ((k+n)/2)! / (((k-n)/2)! (k+n+1)!) (Rodrigues' formula
// integrated by parts n times).
static long double legendre_moment(int n, int k)
{
    if (k < n || (k - n) % 2) return 0.0L;
    return expl((n + 1) * logl(2.0L) + lgammal(k + 1.0L) + lgammal((k + n) / 2 + 1.0L) -
                lgammal((k - n) / 2 + 1.0L) - lgammal(k + n + 2.0L));
}

// Kronrod's (2n+1)-point extension of the n-point Gauss rule on [-1, 1]
// (Sec. 3.1 default rule; Patterson 1968).  The n+1 added nodes are the
// roots of the Stieltjes polynomial E(x) = x^(n+1) + sum_j c_j x^j (j of the
// parity of n+1), fixed by integral P_n E x^k = 0 for odd k, with the
// moments in closed form; each root lies between consecutive Gauss nodes
// (or a Gauss node and an end point) and is found by bisection there.  The
// Kronrod weights integrate the Lagrange basis of the 2n+1 nodes with a
// Gauss-Legendre rule exact for its degree.  Long double throughout.
bool gauss_kronrod(int n, std::vector<double> &x, std::vector<double> &wk,
                   std::vector<double> &wg)
{
    if (n < 1 || n > LENSED_MAX_KRONROD_ORDER) return false;
    std::vector<int> js, ks;
    for (int j = n - 1; j >= 0; j -= 2) js.push_back(j);
    for (int k = 1; (int)ks.size() < (int)js.size(); k += 2) ks.push_back(k);
    const int m = (int)js.size();
    std::vector<long double> A(m * m), c(m);
    for (int r = 0; r < m; ++r) {
        for (int q = 0; q < m; ++q) A[r * m + q] = legendre_moment(n, js[q] + ks[r]);
        c[r] = -legendre_moment(n, n + 1 + ks[r]);
    }
    // Gauss-Jordan with partial pivoting (m <= 4)
    for (int col = 0; col < m; ++col) {
        int piv = col;
        for (int r = col + 1; r < m; ++r)
            if (fabsl(A[r * m + col]) > fabsl(A[piv * m + col])) piv = r;
        if (A[piv * m + col] == 0.0L) return false;
        for (int q = 0; q < m; ++q) std::swap(A[col * m + q], A[piv * m + q]);
        std::swap(c[col], c[piv]);
        for (int r = 0; r < m; ++r) {
            if (r == col) continue;
            const long double f = A[r * m + col] / A[col * m + col];
            for (int q = 0; q < m; ++q) A[r * m + q] -= f * A[col * m + q];
            c[r] -= f * c[col];
        }
    }
    for (int r = 0; r < m; ++r) c[r] /= A[r * m + r];
    auto E = [&](long double z) {
        long double v = powl(z, n + 1);
        for (int q = 0; q < m; ++q) v += c[q] * powl(z, js[q]);
        return v;
    };
    std::vector<double> gx, gw;
    gauss_legendre(n, gx, gw);
    std::vector<long double> edges(n + 2);
    edges[0] = -1.0L;
    for (int i = 0; i < n; ++i) edges[i + 1] = gx[i];
    edges[n + 1] = 1.0L;
    x.assign(2 * n + 1, 0.0);
    wg.assign(2 * n + 1, 0.0);
    std::vector<long double> xl(2 * n + 1);
    for (int i = 0; i <= n; ++i) {
        long double lo = edges[i], hi = edges[i + 1];
        const long double flo = E(lo);
        if ((flo < 0) == (E(hi) < 0)) return false;
        for (int it = 0; it < 200; ++it) {
            const long double mid = 0.5L * (lo + hi);
            if (mid <= lo || mid >= hi) break;
            if ((E(mid) < 0) == (flo < 0)) lo = mid;
            else hi = mid;
        }
        xl[2 * i] = 0.5L * (lo + hi);
        if (i < n) {
            xl[2 * i + 1] = gx[i];
            wg[2 * i + 1] = gw[i];
        }
    }
    xl[n] = 0.0L;  // the middle node (Gauss for odd n, added for even n) by symmetry
    std::vector<double> qx, qw;
    gauss_legendre(2 * n + 2, qx, qw);  // exact to degree 4n + 3 >= 2n
    wk.assign(2 * n + 1, 0.0);
    for (int i = 0; i < 2 * n + 1; ++i) {
        long double acc = 0.0L;
        for (size_t q = 0; q < qx.size(); ++q) {
            long double l = 1.0L;
            for (int k = 0; k < 2 * n + 1; ++k)
                if (k != i) l *= (qx[q] - xl[k]) / (xl[i] - xl[k]);
            acc += qw[q] * l;
        }
        wk[i] = (double)acc;
        x[i] = (double)xl[i];
    }
    return true;
}

// 1-D rule on the unit pixel: offsets t in (-1/2, 1/2), weights summing to 1.
// For LENSED_RULE_GK, wt_gauss (if given) receives the embedded Gauss
// weights (zero on the added nodes).
bool rule_nodes(int rule, int order, std::vector<double> &t, std::vector<double> &wt,
                std::vector<double> *wt_gauss = nullptr)
{
    if (rule == LENSED_RULE_POINT) {
        t = {0.0};
        wt = {1.0};
        return true;
    }
    if (order < 1 || order > LENSED_MAX_RULE_ORDER) return false;
    if (rule == LENSED_RULE_SUB) {
        t.resize(order);
        wt.assign(order, 1.0 / order);
        for (int a = 0; a < order; ++a) t[a] = (a + 0.5) / order - 0.5;
        return true;
    }
    if (rule == LENSED_RULE_GK) {
        std::vector<double> x, wk, wg;
        if (!gauss_kronrod(order, x, wk, wg)) return false;
        t.resize(x.size());
        wt.resize(x.size());
        if (wt_gauss) wt_gauss->resize(x.size());
        for (size_t a = 0; a < x.size(); ++a) {
            t[a] = 0.5 * x[a];
            wt[a] = 0.5 * wk[a];
            if (wt_gauss) (*wt_gauss)[a] = 0.5 * wg[a];
        }
        return true;
    }
    if (rule == LENSED_RULE_GL) {
        std::vector<double> x, w;
        gauss_legendre(order, x, w);
        t.resize(order);
        wt.resize(order);
        for (int a = 0; a < order; ++a) {
            t[a] = 0.5 * x[a];
            wt[a] = 0.5 * w[a];
        }
        return true;
    }
    return false;
}

template <typename T>
struct DevBuf {
    T *p = nullptr;
    size_t n = 0;
    ~DevBuf() { release(); }
    void release()
    {
        if (p) {
            cudaFree(p);
            note_buffers(-1);
        }
        p = nullptr;
        n = 0;
    }
    int alloc(size_t count)
    {
        release();
        if (count == 0) count = 1;
        if (lensed::alloc_failure_injected())
            return fail(LENSED_E_NOMEM, "cudaMalloc(%zu bytes): refused by the injected "
                                        "allocation failure", count * sizeof(T));
        cudaError_t e = cudaMalloc(&p, count * sizeof(T));
        if (e != cudaSuccess) {
            p = nullptr;
            return fail(LENSED_E_NOMEM, "cudaMalloc(%zu bytes): %s", count * sizeof(T),
                        cudaGetErrorString(e));
        }
        note_buffers(1);
        n = count;
        return LENSED_OK;
    }
    int upload(const std::vector<T> &v)
    {
        int rc = alloc(v.size());
        if (rc) return rc;
        if (!v.empty()) CUDA_OK(cudaMemcpy(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
        return LENSED_OK;
    }
};

struct PsfGroup {
    int q, p_max;
    int off, count;  // into the PSF block table
    int sep;         // largest separable rank in the group (0: direct convolution)
};

struct TraceGroup {
    int nn;          // nodes per row of the rule of every system in the group
    int off, count;  // into the trace block table
};

struct GraphEntry {
    int P;
    const void *params;
    void *out;
    int cfg;
    int chunk;  // points per scratch chunk the graph was captured with
    cudaGraphExec_t exec;
    unsigned long long age;
};

struct Candidate {
    LaunchCfg cfg;
    const char *name;
};

// Launch configurations the autotuner tries: trace block size x PSF form
// (0-5), the same with the trace as a persistent, work-queued launch (6-11);
// for MIXED_FF also 0-11 with the float-float re-traces in a second kernel
// (12-23).  The first kBaseCandidates apply to every precision.
struct CandidateTable {
    Candidate c[24];
    char names[24][160];
};
static CandidateTable make_candidates()
{
    CandidateTable t{};
    const int threads[3] = {128, 256, 64};
    for (int split = 0; split < 2; ++split)
        for (int pq = 0; pq < 2; ++pq)
            for (int sep = 0; sep < 2; ++sep)
                for (int b = 0; b < 3; ++b) {
                    const int k = split * 12 + pq * 6 + sep * 3 + b;
                    snprintf(t.names[k], sizeof(t.names[k]), "trace blocks of %d pixels%s, %s%s",
                             threads[b], pq ? " (persistent, work-queued launch)" : "",
                             sep ? "separable PSF where its rank allows" : "direct PSF",
                             split ? ", float-float re-trace as a second pass" : "");
                    t.c[k] = Candidate{LaunchCfg{threads[b], sep, split, pq}, t.names[k]};
                }
    return t;
}
static const CandidateTable g_candidates = make_candidates();
static const Candidate *const kCandidates = g_candidates.c;
constexpr int kAllCandidates = 24;
constexpr int kBaseCandidates = 12;

// Instantiated graphs kept per model (keyed by point count, buffers and
// configuration; the least recently used is dropped beyond this).
constexpr size_t kGraphCache = 32;

// Second-pass queue entries per scratch chunk are capped at this many
// (4 bytes each); blocks that find it full re-trace their rays themselves.
constexpr long long kFfEntryCap = 64LL << 20;

}  // namespace

struct lensed_model {
    int device = 0;
    int precision = LENSED_PREC_MIXED;
    int n_sys = 0;
    int n_par_max = 0;
    int C_total = 0;
    long long total_pix = 0;
    int T_total = 0;  // active (chi^2) tiles over all systems
    size_t scratch_budget = (size_t)2 << 30;  // bytes of per-point image scratch

    std::vector<SysDev> sys_h;
    std::vector<SysDev> sys_gauss_h;  // per system: its embedded Gauss rule (GK systems)
    std::vector<int> need_count;      // per system
    std::vector<int> n_nodes;         // per system
    std::vector<int> n_nodes_gauss;   // per system: Gauss nodes per axis (GK), else 0
    std::vector<int> psf_p, psf_q;    // per system
    std::vector<int> psf_sep;         // per system: separable PSF rank, 0 = direct
    std::vector<int> tiles_all;       // per system: tiles_x * tiles_y
    std::vector<double> ray_flops, ray_transc;  // per system, per ray

    // device tables
    DevBuf<SysDev> sys, sys_gauss;
    DevBuf<int> comp_type, comp_plane, comp_free, comp_sys;
    DevBuf<int> comp_plane_pre;        // planes for the one-off integration of fixed lights
    DevBuf<float> pre_f;               // precomputed luminosities (FP32 modes)
    DevBuf<double> pre_d;              // precomputed luminosities (FP64), then its float copy
    DevBuf<double> comp_value;
    DevBuf<float> data, weight;
    DevBuf<double> data_d, weight_d;  // FP64 mode
    DevBuf<float> psf_f;
    DevBuf<double> psf_d;
    DevBuf<float> node_u, node_w;
    DevBuf<double> node_ud, node_wd;
    DevBuf<int> need;
    DevBuf<double> bn_table;

    // chi^2 PSF blocks (grouped by q, systems contiguous) and render tables
    std::vector<PsfBlock> psf_blocks_h;
    DevBuf<PsfBlock> psf_blocks;
    std::vector<PsfGroup> psf_groups;
    std::vector<int> psf_sys_off, psf_sys_cnt;  // per system range in psf_blocks
    std::vector<int> render_psf_off, render_psf_cnt;
    std::vector<PsfBlock> render_psf_h;
    DevBuf<PsfBlock> render_psf;

    // trace block tables, rebuilt when the items per block change
    int trace_items = 0;
    std::vector<int> trace_sys_off, trace_sys_cnt;
    std::vector<TraceGroup> trace_groups;
    DevBuf<TraceBlock> trace_blocks;
    int n_trace_blocks = 0;
    std::vector<int> render_trace_off, render_trace_cnt;
    DevBuf<TraceBlock> render_trace;

    // per-batch buffers
    int cap_P = 0;
    DevBuf<float> cf;
    DevBuf<double> cd;
    DevBuf<unsigned char> valid, cvalid;
    DevBuf<double> partial;
    DevBuf<unsigned char> Lbuf;
    int chunk_P = 0;      // points per chunk that the scratch budget holds
    int chunk_limit = 0;  // if > 0, at most this many points per chunk
    // MIXED_FF second-pass queue (one trace launch at a time)
    DevBuf<unsigned long long> ffq_cnt;
    DevBuf<FfEntry> ffq_ent;
    DevBuf<float> ffq_val;
    DevBuf<FfEntry> ffq_pix;
    DevBuf<uint2> ffq_prun;
    DevBuf<unsigned long long> work;  // item counter of a persistent trace launch
    // render buffers (one point)
    DevBuf<float> rcf;
    DevBuf<double> rcd;
    DevBuf<unsigned char> rvalid, rcvalid;
    DevBuf<unsigned char> rL, rLg;  // rLg: the embedded-Gauss luminosities (GK systems)
    // host-API staging
    DevBuf<double> stage_params, stage_out;

    int cfg_index = -1;  // autotuned candidate, -1 = default
    long long ffq_limit = -1;  // test hook: entries the second pass may take (-1: all)
    cudaStream_t cap_stream = nullptr;
    std::vector<GraphEntry> graphs;
    unsigned long long graph_clock = 0;

    LaunchCfg cfg() const { return kCandidates[cfg_index < 0 ? 0 : cfg_index].cfg; }
    // points per chunk of the batched schedule (after ensure_capacity)
    int chunk() const { return chunk_limit > 0 ? std::min(chunk_P, chunk_limit) : chunk_P; }
    int n_candidates() const
    {
        return precision == LENSED_PREC_MIXED_FF ? kAllCandidates : kBaseCandidates;
    }
    FfQueue ffq() const
    {
        if (!ffq_cnt.p) return FfQueue{};
        const long long n = (long long)ffq_ent.n;
        return {ffq_cnt.p, ffq_ent.p, ffq_val.p, ffq_limit >= 0 ? std::min(ffq_limit, n) : n,
                ffq_pix.p, (long long)ffq_pix.n, ffq_prun.p};
    }
    size_t elem() const { return precision == LENSED_PREC_FP64 ? sizeof(double) : sizeof(float); }
    // FP32 modes with fixed lights: the chi^2 path traces without them and
    // compares with data from which their convolved image was removed
    bool fold_fixed = false;
    NodeTables nodes_chi() const
    {
        NodeTables n = nodes();
        if (fold_fixed) n.pre_f = nullptr;
        return n;
    }
    NodeTables nodes() const
    {
        return {node_u.p, node_w.p, node_ud.p, node_wd.p, pre_f.p, pre_d.p,
                precision == LENSED_PREC_MIXED_FF ? 1 : 0};
    }

    void clear_graphs()
    {
        for (auto &g : graphs) cudaGraphExecDestroy(g.exec);
        graphs.clear();
    }
    ~lensed_model()
    {
        cudaDeviceSynchronize();
        clear_graphs();
        if (cap_stream) cudaStreamDestroy(cap_stream);
    }
};

namespace {

int build_trace_tables(lensed_model *m, int items)
{
    if (m->trace_items == items) return LENSED_OK;
    // systems ordered by nodes per row, so each group is one launch
    std::vector<int> order(m->n_sys);
    for (int s = 0; s < m->n_sys; ++s) order[s] = s;
    std::stable_sort(order.begin(), order.end(),
                     [&](int a, int b) { return m->n_nodes[a] < m->n_nodes[b]; });
    std::vector<TraceBlock> tb, rb;
    m->trace_sys_off.assign(m->n_sys, 0);
    m->trace_sys_cnt.assign(m->n_sys, 0);
    m->render_trace_off.assign(m->n_sys, 0);
    m->render_trace_cnt.assign(m->n_sys, 0);
    m->trace_groups.clear();
    for (int s : order) {
        if (m->trace_groups.empty() || m->trace_groups.back().nn != m->n_nodes[s])
            m->trace_groups.push_back({m->n_nodes[s], (int)tb.size(), 0});
        m->trace_sys_off[s] = (int)tb.size();
        for (int a = 0; a < m->need_count[s]; a += items)
            tb.push_back({s, a, std::min(a + items, m->need_count[s])});
        m->trace_sys_cnt[s] = (int)tb.size() - m->trace_sys_off[s];
        m->trace_groups.back().count = (int)tb.size() - m->trace_groups.back().off;
    }
    for (int s = 0; s < m->n_sys; ++s) {
        m->render_trace_off[s] = (int)rb.size();
        const int npix = m->sys_h[s].npix;
        for (int a = 0; a < npix; a += items) rb.push_back({s, a, std::min(a + items, npix)});
        m->render_trace_cnt[s] = (int)rb.size() - m->render_trace_off[s];
    }
    int rc = m->trace_blocks.upload(tb);
    if (rc) return rc;
    rc = m->render_trace.upload(rb);
    if (rc) return rc;
    m->n_trace_blocks = (int)tb.size();
    m->trace_items = items;
    m->clear_graphs();
    return LENSED_OK;
}

int ensure_capacity(lensed_model *m, int P)
{
    if (P <= m->cap_P) return LENSED_OK;
    cudaDeviceSynchronize();
    m->clear_graphs();
    // no capacity until every buffer below is in place: a failed allocation
    // leaves the model valid, and the next call allocates again
    m->cap_P = 0;
    m->chunk_P = 0;
    int rc;
    if ((rc = m->cf.alloc((size_t)P * m->C_total * kNC))) return rc;
    if ((rc = m->cd.alloc((size_t)P * m->C_total * kNC))) return rc;
    if ((rc = m->valid.alloc((size_t)P * m->n_sys))) return rc;
    if ((rc = m->cvalid.alloc((size_t)P * m->C_total))) return rc;
    if ((rc = m->partial.alloc((size_t)P * std::max(m->T_total, 1)))) return rc;
    // per point: its pixel luminosities, and in MIXED_FF room for every
    // needed pixel in the second pass's pixel queue
    long long need_total = 0;
    for (int s = 0; s < m->n_sys; ++s) need_total += m->need_count[s];
    const size_t per_point =
        (size_t)m->total_pix * m->elem() +
        (m->precision == LENSED_PREC_MIXED_FF ? (size_t)need_total * (sizeof(FfEntry) + sizeof(uint2))
                                               : 0);
    size_t chunk = std::max<size_t>(1, m->scratch_budget / std::max<size_t>(per_point, 1));
    chunk = std::min<size_t>(chunk, (size_t)P);
    if ((rc = m->Lbuf.alloc(chunk * (size_t)m->total_pix * m->elem()))) return rc;
    if ((rc = m->work.alloc(1))) return rc;
    if (m->precision == LENSED_PREC_MIXED_FF) {
        // the second pass's queue: room for every traced ray of a chunk, capped
        long long rays = 0;
        for (int s = 0; s < m->n_sys; ++s)
            rays += (long long)m->need_count[s] * m->n_nodes[s] * m->n_nodes[s];
        const size_t cap = (size_t)std::max(1LL, std::min(rays * (long long)chunk, kFfEntryCap));
        if ((rc = m->ffq_cnt.alloc(2))) return rc;
        if ((rc = m->ffq_ent.alloc(cap))) return rc;
        if ((rc = m->ffq_val.alloc(cap))) return rc;
        const size_t pcap = (size_t)std::max(1LL, need_total * (long long)chunk);
        if ((rc = m->ffq_pix.alloc(pcap))) return rc;
        if ((rc = m->ffq_prun.alloc(pcap))) return rc;
    }
    m->chunk_P = (int)chunk;
    m->cap_P = P;
    return LENSED_OK;
}

// Optional per-stage timing of enqueue_batch: events recorded around every
// launch (stage 0 prologue, 1 trace, 2 psf, 3 finalize).
struct StageTimer {
    std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> marks;
    cudaStream_t st;
    void begin(int stage)
    {
        cudaEvent_t a, b;
        cudaEventCreate(&a);
        cudaEventCreate(&b);
        cudaEventRecord(a, st);
        marks.push_back({stage, {a, b}});
    }
    void end() { cudaEventRecord(marks.back().second.second, st); }
    ~StageTimer()
    {
        for (auto &mk : marks) {
            cudaEventDestroy(mk.second.first);
            cudaEventDestroy(mk.second.second);
        }
    }
};

// Enqueue the batched evaluation (no graph) on stream st.
void enqueue_batch(lensed_model *m, const double *params, int P, double *out, LaunchCfg cfg,
                   cudaStream_t st, StageTimer *tm = nullptr)
{
    if (tm) tm->begin(0);
    launch_prologue(m->sys.p, m->comp_sys.p, 0, m->n_sys, 0, m->C_total, m->comp_type.p,
                    m->comp_free.p, m->comp_value.p, params, false, P, 0, P, m->n_par_max,
                    m->C_total, m->bn_table.p, m->cf.p, m->cd.p, m->cvalid.p, m->valid.p, st);
    if (tm) tm->end();
    const int chunk = m->chunk();
    for (int p0 = 0; p0 < P; p0 += chunk) {
        const int nP = std::min(chunk, P - p0);
        if (tm) tm->begin(1);
        // (a second pass, where launch_trace runs one, completes before the
        // MIXED fix-up overwrites its pixels: both are on stream st)
        for (const TraceGroup &g : m->trace_groups)
            launch_trace(m->precision, cfg, g.nn, m->sys.p, m->comp_type.p, m->comp_plane.p,
                         m->cf.p, m->cd.p, m->valid.p, P, m->C_total, m->trace_blocks.p + g.off,
                         g.count, m->need.p, m->nodes_chi(), p0, nP, m->Lbuf.p, m->total_pix, st,
                         m->ffq(), m->work.p);
        if (is_mixed(m->precision))
            launch_fix64(cfg, m->sys.p, 0, m->n_sys, m->comp_type.p, m->comp_plane.p, m->cf.p,
                         m->cd.p, m->valid.p, P, m->C_total, m->need.p, m->nodes_chi(), p0, nP,
                         m->Lbuf.p, m->total_pix, st);
        if (tm) tm->end();
        if (tm) tm->begin(2);
        for (const PsfGroup &g : m->psf_groups)
            launch_psf(m->precision, g.q, cfg.psf_sep ? g.sep : 0, g.p_max, m->sys.p, m->psf_f.p, m->psf_d.p, m->data.p,
                       m->weight.p, m->data_d.p, m->weight_d.p, m->valid.p, P, m->psf_blocks.p + g.off, g.count, p0, nP,
                       m->Lbuf.p, m->total_pix, m->partial.p, m->T_total, nullptr, st);
        if (tm) tm->end();
    }
    if (tm) tm->begin(3);
    launch_finalize(m->sys.p, m->valid.p, P, m->partial.p, m->T_total, out, 0, 0, m->n_sys, P,
                    st);
    if (tm) tm->end();
}

int check_model(const lensed_model *m)
{
    if (!m) return fail(LENSED_E_ARG, "model is NULL");
    return LENSED_OK;
}

}  // namespace

// ===========================================================================
// C ABI

extern "C" const char *lensed_last_error(void) { return g_last_error.c_str(); }

extern "C" long long lensed_debug_fail_alloc(long long after)
{
    g_alloc_budget.store(after < 0 ? -1 : after);
    return g_live_buffers.load();
}

extern "C" int lensed_debug_ff_queue_cap(lensed_model *m, long long cap)
{
    if (check_model(m)) return LENSED_E_ARG;
    cudaDeviceSynchronize();
    m->clear_graphs();  // captured launches hold the queue's capacity
    m->ffq_limit = cap < 0 ? -1 : cap;
    return LENSED_OK;
}

// Low-rank form of a normalised, flipped PSF F [m][n] (m = 2p+1 rows):
// singular value decomposition by one-sided Jacobi rotations (Hestenes) in
// double, then the fewest terms F ~ sum_k c_k r_k^T (c_k = sigma_k u_k,
// r_k = v_k, at most kMaxSepRank) whose residual sum_ij |F - F_R| stays below
// 1e-7 (the float rounding of the taps themselves).  Returns the number of
// terms, 0 if none qualifies or the separable passes would not be cheaper.
constexpr int kMaxSepRank = 3;
static int psf_low_rank(const double *F, int m, int n, std::vector<double> &c,
                        std::vector<double> &r)
{
    std::vector<double> U(F, F + (size_t)m * n), V((size_t)n * n, 0.0);
    for (int j = 0; j < n; ++j) V[(size_t)j * n + j] = 1.0;
    for (int sweep = 0; sweep < 60; ++sweep) {
        bool rotated = false;
        for (int a = 0; a < n - 1; ++a)
            for (int b = a + 1; b < n; ++b) {
                double al = 0, be = 0, ga = 0;
                for (int i = 0; i < m; ++i) {
                    const double x = U[(size_t)i * n + a], y = U[(size_t)i * n + b];
                    al += x * x;
                    be += y * y;
                    ga += x * y;
                }
                if (!(fabs(ga) > 1e-15 * sqrt(al * be))) continue;
                rotated = true;
                const double ze = (be - al) / (2 * ga);
                const double t = (ze >= 0 ? 1.0 : -1.0) / (fabs(ze) + sqrt(1 + ze * ze));
                const double cs = 1 / sqrt(1 + t * t), sn = cs * t;
                for (int i = 0; i < m; ++i) {
                    const double x = U[(size_t)i * n + a], y = U[(size_t)i * n + b];
                    U[(size_t)i * n + a] = cs * x - sn * y;
                    U[(size_t)i * n + b] = sn * x + cs * y;
                }
                for (int i = 0; i < n; ++i) {
                    const double x = V[(size_t)i * n + a], y = V[(size_t)i * n + b];
                    V[(size_t)i * n + a] = cs * x - sn * y;
                    V[(size_t)i * n + b] = sn * x + cs * y;
                }
            }
        if (!rotated) break;
    }
    // columns of U are sigma_j u_j; order by sigma
    std::vector<int> ord(n);
    std::vector<double> sig(n);
    for (int j = 0; j < n; ++j) {
        double s2 = 0;
        for (int i = 0; i < m; ++i) s2 += U[(size_t)i * n + j] * U[(size_t)i * n + j];
        sig[j] = sqrt(s2);
        ord[j] = j;
    }
    std::sort(ord.begin(), ord.end(), [&](int x, int y) { return sig[x] > sig[y]; });
    const int P = m / 2;
    const double direct = (double)m * n;
    for (int R = 1; R <= std::min(kMaxSepRank, n); ++R) {
        double res = 0;
        for (int i = 0; i < m; ++i)
            for (int j = 0; j < n; ++j) {
                double v = F[(size_t)i * n + j];
                for (int k = 0; k < R; ++k)
                    v -= U[(size_t)i * n + ord[k]] * V[(size_t)j * n + ord[k]];
                res += fabs(v);
            }
        if (res > 1e-7) continue;
        const double cost = R * (n * (kTileH + 2.0 * P) / kTileH + m);
        if (cost > 0.6 * direct) return 0;
        c.assign((size_t)R * m, 0.0);
        r.assign((size_t)R * n, 0.0);
        for (int k = 0; k < R; ++k) {
            for (int i = 0; i < m; ++i) c[(size_t)k * m + i] = U[(size_t)i * n + ord[k]];
            for (int j = 0; j < n; ++j) r[(size_t)k * n + j] = V[(size_t)j * n + ord[k]];
        }
        return R;
    }
    return 0;
}

// One-off FP64 pixel integrals of the foreground lights whose parameters are
// all fixed (device plane kPlanePrecomputed): every evaluation starts each
// pixel's sum from them instead of tracing those components again.  For a
// Gauss-Kronrod system the embedded Gauss rule gets a table of its own.
// Eq. 15 on the host in FP64, with the kernels' indexing: L*_ij =
// sum_kl Fs[k][l] L[clamp(i + k - p)][clamp(j + l - q)], Fs the stored
// (flipped, unit-sum) PSF of the system.
static void convolve_host(const SysDev &S, const double *L, const double *Fs, double *out)
{
    const int p = S.psf_p, q = S.psf_q, W = 2 * q + 1;
    for (int i = 0; i < S.ny; ++i)
        for (int j = 0; j < S.nx; ++j) {
            double acc = 0.0;
            for (int k = 0; k <= 2 * p; ++k) {
                const int gi = std::min(std::max(i + k - p, 0), S.ny - 1);
                for (int l = 0; l < W; ++l) {
                    const int gj = std::min(std::max(j + l - q, 0), S.nx - 1);
                    acc += Fs[k * W + l] * L[(size_t)gi * S.nx + gj];
                }
            }
            out[(size_t)i * S.nx + j] = acc;
        }
}

static int precompute_fixed_light(lensed_model *m, const std::vector<int> &cplane_pre,
                                  const std::vector<double> &data_d,
                                  const std::vector<double> &psf_d,
                                  const std::vector<size_t> &psfd_off)
{
    bool any = false;
    for (auto &S : m->sys_h) any |= S.pre_off >= 0;
    if (!any) return LENSED_OK;
    const long long T = m->total_pix;
    int rc;
    DevBuf<double> zeros;
    if ((rc = m->comp_plane_pre.upload(cplane_pre)) ||
        (rc = zeros.upload(std::vector<double>(std::max(m->n_par_max, 1), 0.0))) ||
        (rc = m->pre_d.alloc(2 * T)))
        return rc;
    CUDA_OK(cudaMemset(m->pre_d.p, 0, sizeof(double) * 2 * T));
    // constants of every component at a dummy point (the fixed lights read
    // no parameter), all systems marked valid for this pass
    launch_prologue(m->sys.p, m->comp_sys.p, 0, m->n_sys, 0, m->C_total, m->comp_type.p,
                    m->comp_free.p, m->comp_value.p, zeros.p, true, 1, 0, 1, m->n_par_max,
                    m->C_total, m->bn_table.p, m->rcf.p, m->rcd.p, m->rcvalid.p, m->rvalid.p, 0);
    CUDA_OK(cudaMemset(m->rvalid.p, 1, m->n_sys));
    const NodeTables nodes{m->node_u.p, m->node_w.p, m->node_ud.p, m->node_wd.p, nullptr,
                           nullptr, 0};
    const int n_blocks = m->render_trace_off.back() + m->render_trace_cnt.back();
    for (int g = 0; g < 2; ++g) {
        if (g == 1 && m->rLg.p == nullptr) break;  // no Gauss-Kronrod system
        launch_trace(LENSED_PREC_FP64, m->cfg(), 1, g ? m->sys_gauss.p : m->sys.p,
                     m->comp_type.p, m->comp_plane_pre.p, m->rcf.p, m->rcd.p, m->rvalid.p, 1,
                     m->C_total, m->render_trace.p, n_blocks, nullptr, nodes, 0, 1,
                     m->pre_d.p + g * T, 0, 0);
    }
    CUDA_OK(cudaGetLastError());
    CUDA_OK(cudaDeviceSynchronize());
    std::vector<double> hd(2 * T);
    CUDA_OK(cudaMemcpy(hd.data(), m->pre_d.p, sizeof(double) * 2 * T, cudaMemcpyDeviceToHost));
    std::vector<float> hf(hd.begin(), hd.end());
    if ((rc = m->pre_f.upload(hf))) return rc;
    if (m->precision != LENSED_PREC_FP64) {
        // FP32 modes: the chi^2 path leaves the fixed lights out of the float
        // arithmetic.  Eq. 15 is linear, so L* = F * L_fixed + F * L_rest;
        // the first term is the same for every point and is taken off the
        // data here in FP64, the kernels convolve only the rest in float.
        // (Renders still start from the fixed lights and convolve the sum.)
        std::vector<float> dres(T);
        std::vector<double> conv;
        for (int s = 0; s < m->n_sys; ++s) {
            const SysDev &S = m->sys_h[s];
            const double *d = data_d.data() + S.pix_off;
            float *o = dres.data() + S.pix_off;
            if (S.pre_off < 0) {
                for (int k = 0; k < S.npix; ++k) o[k] = (float)d[k];
                continue;
            }
            const double *Lf = hd.data() + S.pix_off;
            conv.assign(S.npix, 0.0);
            if (S.psf_p > 0 || S.psf_q > 0)
                convolve_host(S, Lf, psf_d.data() + psfd_off[s], conv.data());
            else
                std::copy(Lf, Lf + S.npix, conv.begin());
            for (int k = 0; k < S.npix; ++k) o[k] = (float)(d[k] - conv[k]);
        }
        if ((rc = m->data.upload(dres))) return rc;
        m->fold_fixed = true;
    }
    // point the systems (and their Gauss shadows) at their tables
    for (int s = 0; s < m->n_sys; ++s) {
        if (m->sys_h[s].pre_off < 0) continue;
        m->sys_h[s].pre_off = m->sys_h[s].pix_off;
        m->sys_gauss_h[s].pre_off = m->n_nodes_gauss[s] > 0 ? T + m->sys_h[s].pix_off : -1;
    }
    if ((rc = m->sys.upload(m->sys_h)) || (rc = m->sys_gauss.upload(m->sys_gauss_h))) return rc;
    if (m->precision != LENSED_PREC_FP64) m->pre_d.release();
    return LENSED_OK;
}

extern "C" int lensed_create_model(const lensed_system_desc *systems, int n_systems,
                                   int precision, lensed_model **out)
{
    g_last_error.clear();
    if (!out) return fail(LENSED_E_ARG, "out is NULL");
    if (!systems || n_systems < 1) return fail(LENSED_E_ARG, "need at least one system");
    if (precision < LENSED_PREC_FP32 || precision > LENSED_PREC_MIXED_FF)
        return fail(LENSED_E_ARG, "unknown precision %d", precision);

    // ---- validate every descriptor before touching the device
    int n_par_max = 0, C_total = 0;
    long long total_pix = 0;
    for (int s = 0; s < n_systems; ++s) {
        const lensed_system_desc &d = systems[s];
        if (d.nx < 1 || d.ny < 1 || d.nx > LENSED_MAX_IMAGE_SIDE || d.ny > LENSED_MAX_IMAGE_SIDE)
            return fail(LENSED_E_ARG, "system %d: image size %d x %d out of range", s, d.nx, d.ny);
        if (!(d.pixel_scale > 0.0) || !isfinite(d.pixel_scale))
            return fail(LENSED_E_ARG, "system %d: pixel_scale must be > 0", s);
        if (!d.data) return fail(LENSED_E_ARG, "system %d: data is NULL", s);
        if (!d.variance && !(d.gain > 0.0 && isfinite(d.gain) && isfinite(d.offset)))
            return fail(LENSED_E_ARG, "system %d: need a variance map or gain > 0", s);
        if (d.psf) {
            if (d.psf_nx < 1 || d.psf_ny < 1 || d.psf_nx % 2 == 0 || d.psf_ny % 2 == 0)
                return fail(LENSED_E_ARG, "system %d: PSF size %d x %d must be odd", s, d.psf_nx,
                            d.psf_ny);
            if (d.psf_nx > 2 * LENSED_MAX_PSF_HALF + 1 || d.psf_ny > 2 * LENSED_MAX_PSF_HALF + 1)
                return fail(LENSED_E_UNSUPPORTED, "system %d: PSF larger than %d x %d", s,
                            2 * LENSED_MAX_PSF_HALF + 1, 2 * LENSED_MAX_PSF_HALF + 1);
        }
        if (d.rule != LENSED_RULE_POINT &&
            (d.rule_order < 1 || d.rule_order > LENSED_MAX_RULE_ORDER))
            return fail(LENSED_E_ARG, "system %d: rule order %d out of range", s, d.rule_order);
        if (d.rule < LENSED_RULE_POINT || d.rule > LENSED_RULE_GK)
            return fail(LENSED_E_ARG, "system %d: unknown rule %d", s, d.rule);
        if (d.rule == LENSED_RULE_GK && d.rule_order > LENSED_MAX_KRONROD_ORDER)
            return fail(LENSED_E_ARG, "system %d: Gauss-Kronrod order %d out of range (1..%d)", s,
                        d.rule_order, LENSED_MAX_KRONROD_ORDER);
        if (d.n_components < 1 || d.n_components > LENSED_MAX_COMPONENTS || !d.components)
            return fail(LENSED_E_ARG, "system %d: %d components (1..%d)", s, d.n_components,
                        LENSED_MAX_COMPONENTS);
        if (d.n_params < 0) return fail(LENSED_E_ARG, "system %d: n_params < 0", s);
        if (!isfinite(d.zeropoint)) return fail(LENSED_E_ARG, "system %d: zeropoint", s);
        for (int c = 0; c < d.n_components; ++c) {
            const lensed_component &cp = d.components[c];
            const int np = nparams_of(cp.type);
            if (np < 0) return fail(LENSED_E_ARG, "system %d comp %d: unknown type %d", s, c, cp.type);
            const bool mass = cp.type <= LENSED_POINTMASS;
            if (mass && cp.plane != LENSED_PLANE_LENS)
                return fail(LENSED_E_ARG, "system %d comp %d: mass must be on the lens plane", s, c);
            if (!mass && cp.plane != LENSED_PLANE_FOREGROUND && cp.plane != LENSED_PLANE_SOURCE &&
                !(cp.plane == LENSED_PLANE_SOURCE_IMAGE && cp.type != LENSED_SKY))
                return fail(LENSED_E_ARG, "system %d comp %d: bad plane %d", s, c, cp.plane);
            for (int k = 0; k < np; ++k) {
                if (cp.free_index[k] >= d.n_params)
                    return fail(LENSED_E_ARG, "system %d comp %d: free index %d >= n_params %d",
                                s, c, cp.free_index[k], d.n_params);
                if (cp.free_index[k] < 0 && !isfinite(cp.value[k]))
                    return fail(LENSED_E_NONFINITE, "system %d comp %d: fixed value %d not finite",
                                s, c, k);
            }
        }
        n_par_max = std::max(n_par_max, d.n_params);
        C_total += d.n_components;
        total_pix += (long long)d.nx * d.ny;
    }

    // ---- host tables
    std::vector<SysDev> sh(n_systems), shg(n_systems);
    std::vector<int> sep_v(n_systems, 0);
    std::vector<int> nng_v(n_systems);
    std::vector<int> ctype, cplane, cplane_pre, cfree, csys;
    std::vector<double> cval;
    std::vector<float> data, weight, psf_f, node_u, node_w;
    std::vector<double> data_d, weight_d, psf_d, node_ud, node_wd;
    std::vector<size_t> psfd_off(n_systems);
    std::vector<int> need;
    std::vector<std::vector<PsfBlock>> chi_tiles(n_systems);
    std::vector<int> need_count(n_systems), nn_v(n_systems), pp(n_systems), qq(n_systems),
        tiles_all(n_systems);
    long long pix_off = 0;
    int comp_off = 0, T_total = 0;
    std::vector<double> ray_flops_v, ray_transc_v;
    for (int s = 0; s < n_systems; ++s) {
        const lensed_system_desc &d = systems[s];
        const int nx = d.nx, ny = d.ny, npix = nx * ny;
        SysDev &S = sh[s];
        memset(&S, 0, sizeof(S));
        S.pre_off = -1;
        S.nx = nx;
        S.ny = ny;
        S.npix = npix;
        S.h = (float)d.pixel_scale;
        S.h_lo = (float)(d.pixel_scale - (double)S.h);
        S.hd = d.pixel_scale;
        S.cx = 0.5f * (nx - 1);
        S.cy = 0.5f * (ny - 1);
        S.zeropoint = d.zeropoint;
        // weights (Sec. 3.2-3.3): w = extra / s^2, zero where masked
        std::vector<double> w(npix);
        for (int k = 0; k < npix; ++k) {
            const bool masked = d.mask && d.mask[k];
            if (masked) {
                w[k] = 0.0;
                data.push_back(0.f);
                data_d.push_back(0.0);
                continue;
            }
            const double dv = d.data[k];
            if (!isfinite(dv))
                return fail(LENSED_E_NONFINITE, "system %d: data[%d] not finite", s, k);
            const double s2 = d.variance ? d.variance[k] : (dv + d.offset) / d.gain;
            if (!(s2 > 0.0) || !isfinite(s2))
                return fail(LENSED_E_NONFINITE, "system %d: variance[%d] = %g not > 0", s, k, s2);
            const double ex = d.extra_weight ? d.extra_weight[k] : 1.0;
            if (!isfinite(ex) || ex < 0.0)
                return fail(LENSED_E_NONFINITE, "system %d: extra_weight[%d] invalid", s, k);
            w[k] = ex / s2;
            data.push_back((float)dv);
            data_d.push_back(dv);
        }
        double wmax = 0.0;
        for (int k = 0; k < npix; ++k) wmax = std::max(wmax, w[k]);
        S.wscale = wmax > 0.0 ? wmax : 1.0;
        for (int k = 0; k < npix; ++k) {
            const double rel = w[k] / S.wscale;
            weight.push_back((float)rel);
            weight_d.push_back(rel);
        }
        // PSF (Sec. 3.1): normalised to unit sum, stored flipped (F_{-k,-l})
        int P = 0, Q = 0;
        S.psf_off = (int)psf_f.size();
        psfd_off[s] = psf_d.size();  // the FP64 table holds no separable factors
        if (d.psf) {
            P = d.psf_ny / 2;
            Q = d.psf_nx / 2;
            double sum = 0.0;
            for (int k = 0; k < d.psf_nx * d.psf_ny; ++k) {
                if (!isfinite(d.psf[k]))
                    return fail(LENSED_E_NONFINITE, "system %d: psf[%d] not finite", s, k);
                sum += d.psf[k];
            }
            if (!(sum != 0.0) || !isfinite(sum))
                return fail(LENSED_E_NONFINITE, "system %d: PSF sums to %g", s, sum);
            // normalised, flipped; the float copy is adjusted at its largest tap
            // so that it sums to one in exact arithmetic
            const size_t f0 = psf_f.size();
            size_t imax = f0;
            for (int kk = 0; kk <= 2 * P; ++kk)
                for (int ll = 0; ll <= 2 * Q; ++ll) {
                    const double f = d.psf[(2 * P - kk) * d.psf_nx + (2 * Q - ll)] / sum;
                    psf_d.push_back(f);
                    psf_f.push_back((float)f);
                    if (fabs(f) > fabs(psf_d[imax])) imax = psf_f.size() - 1;
                }
            double rest = 0.0;
            for (size_t k = f0; k < psf_f.size(); ++k)
                if (k != imax) rest += (double)psf_f[k];
            psf_f[imax] = (float)(1.0 - rest);
        } else {
            psf_d.push_back(1.0);
            psf_f.push_back(1.f);
        }
        S.psf_p = P;
        S.psf_q = Q;
        pp[s] = P;
        qq[s] = Q;
        // low-rank PSF (FP32 modes): float factors appended to the table, the
        // first column factor adjusted so that the float terms sum to one
        S.psf_rank = 0;
        if (d.psf && precision != LENSED_PREC_FP64) {
            std::vector<double> cf_, rf_;
            const int m_ = 2 * P + 1, n_ = 2 * Q + 1;
            const int R = psf_low_rank(psf_d.data() + (psf_d.size() - (size_t)m_ * n_), m_, n_,
                                       cf_, rf_);
            if (R > 0) {
                S.psf_rank = R;
                S.psf_sep_off = (int)psf_f.size();
                std::vector<float> cfl(cf_.begin(), cf_.end()), rfl(rf_.begin(), rf_.end());
                double tot = 0, s_r0 = 0, s_c0 = 0;
                for (int k = 0; k < R; ++k) {
                    double sc = 0, sr = 0;
                    for (int i = 0; i < m_; ++i) sc += cfl[(size_t)k * m_ + i];
                    for (int j = 0; j < n_; ++j) sr += rfl[(size_t)k * n_ + j];
                    tot += sc * sr;
                    if (k == 0) s_r0 = sr, s_c0 = sc;
                }
                int imax = 0;
                for (int i = 1; i < m_; ++i)
                    if (fabs(cfl[i]) > fabs(cfl[imax])) imax = i;
                if (s_r0 != 0.0) cfl[imax] = (float)(cfl[imax] - (tot - 1.0) / s_r0);
                (void)s_c0;
                for (int k = 0; k < R; ++k) {
                    psf_f.insert(psf_f.end(), cfl.begin() + (size_t)k * m_,
                                 cfl.begin() + (size_t)(k + 1) * m_);
                    psf_f.insert(psf_f.end(), rfl.begin() + (size_t)k * n_,
                                 rfl.begin() + (size_t)(k + 1) * n_);
                }
                sep_v[s] = R;
            }
        }
        // quadrature (Eq. 14): 1-D offsets t*h, 2-D weights W_a W_b; the float
        // weights are adjusted at the largest one so they sum to one in exact
        // arithmetic, leaving no coherent scale error
        std::vector<double> t, wt, wtg;
        rule_nodes(d.rule, d.rule_order, t, wt, &wtg);
        auto append_rule = [&](const std::vector<double> &tt, const std::vector<double> &ww,
                               SysDev &D) {
            const int nn = (int)tt.size();
            D.nn = nn;
            D.node_off = (int)node_u.size();
            D.w2_off = (int)node_w.size();
            for (int a = 0; a < nn; ++a) {
                node_ud.push_back(tt[a] * d.pixel_scale);
                node_u.push_back((float)(tt[a] * d.pixel_scale));
            }
            std::vector<float> w2f(nn * nn);
            int kmax = 0;
            for (int b = 0; b < nn; ++b)
                for (int a = 0; a < nn; ++a) {
                    const double v = ww[a] * ww[b];
                    node_wd.push_back(v);
                    w2f[b * nn + a] = (float)v;
                    if (v > ww[kmax % nn] * ww[kmax / nn]) kmax = b * nn + a;
                }
            double rest = 0.0;
            for (int k = 0; k < nn * nn; ++k)
                if (k != kmax) rest += (double)w2f[k];
            w2f[kmax] = (float)(1.0 - rest);
            node_w.insert(node_w.end(), w2f.begin(), w2f.end());
        };
        append_rule(t, wt, S);
        const int nn = S.nn;
        nn_v[s] = nn;
        // needed pixels: every pixel an unmasked output reads through the
        // (clamped) PSF footprint
        std::vector<unsigned char> nd(npix, 0);
        for (int i = 0; i < ny; ++i)
            for (int j = 0; j < nx; ++j) {
                if (!(w[(size_t)i * nx + j] > 0.0)) continue;
                for (int k = -P; k <= P; ++k) {
                    const int ii = std::min(std::max(i + k, 0), ny - 1);
                    for (int l = -Q; l <= Q; ++l) {
                        const int jj = std::min(std::max(j + l, 0), nx - 1);
                        nd[(size_t)ii * nx + jj] = 1;
                    }
                }
            }
        S.need_off = (long long)need.size();
        int cnt = 0;
        for (int k = 0; k < npix; ++k)
            if (nd[k]) {
                need.push_back(k);
                ++cnt;
            }
        need_count[s] = cnt;
        S.n_need = cnt;
        // tiles of the chi^2 pass: those holding an output with w > 0
        S.tiles_x = (nx + kTileW - 1) / kTileW;
        S.tiles_y = (ny + kTileH - 1) / kTileH;
        tiles_all[s] = S.tiles_x * S.tiles_y;
        S.tile_off = T_total;
        for (int ty = 0; ty < S.tiles_y; ++ty)
            for (int tx = 0; tx < S.tiles_x; ++tx) {
                unsigned live_rows = 0u, live_warps = 0u;
                for (int r = 0; r < kTileH; ++r) {
                    const int i = ty * kTileH + r;
                    if (i >= ny) break;
                    for (int c = 0; c < kTileW; ++c) {
                        const int j = tx * kTileW + c;
                        if (j >= nx) break;
                        if (w[(size_t)i * nx + j] > 0.0) {
                            live_rows |= 1u << r;
                            live_warps |= 1u << ((r / 16) * 4 + c / 16);
                        }
                    }
                }
                if (live_rows)
                    chi_tiles[s].push_back({s, T_total + (int)chi_tiles[s].size(), ty * kTileH,
                                            tx * kTileW, live_rows, live_warps});
            }
        S.n_tiles = (int)chi_tiles[s].size();
        T_total += S.n_tiles;
        // components
        S.comp_off = comp_off;
        S.ncomp = d.n_components;
        S.n_params = d.n_params;
        for (int c = 0; c < d.n_components; ++c) {
            const lensed_component &cp = d.components[c];
            ctype.push_back(cp.type);
            const int np = nparams_of(cp.type);
            // a foreground light with no free parameter is integrated once
            // per model; the ray kernels skip it
            bool fixed_fg = cp.plane == LENSED_PLANE_FOREGROUND;
            for (int k = 0; k < np; ++k) fixed_fg = fixed_fg && cp.free_index[k] < 0;
            // the kernels see an image-plane-prior source as a source; the
            // prologue moves it (bit c of imgpos_mask)
            cplane.push_back(fixed_fg ? kPlanePrecomputed
                             : cp.plane == LENSED_PLANE_SOURCE_IMAGE ? LENSED_PLANE_SOURCE
                                                                      : cp.plane);
            cplane_pre.push_back(fixed_fg ? LENSED_PLANE_FOREGROUND : kPlanePrecomputed);
            if (fixed_fg) S.pre_off = 0;  // placed below
            if (cp.plane == LENSED_PLANE_SOURCE_IMAGE) S.imgpos_mask |= 1 << c;
            csys.push_back(s);
            for (int k = 0; k < LENSED_MAX_COMPONENT_PARAMS; ++k) {
                cfree.push_back(k < np ? cp.free_index[k] : -1);
                cval.push_back(k < np && cp.free_index[k] < 0 ? cp.value[k] : 0.0);
            }
        }
        comp_off += d.n_components;
        {
            double f = 6.0, tr = 0.0;
            for (int c = 0; c < d.n_components; ++c)
                if (cplane[comp_off - d.n_components + c] != kPlanePrecomputed)
                    component_ops(d.components[c].type, f, tr);
            ray_flops_v.push_back(f);
            ray_transc_v.push_back(tr);
        }
        S.pix_off = pix_off;
        if (S.pre_off >= 0) S.pre_off = pix_off;
        pix_off += npix;
        // the embedded Gauss rule of a Gauss-Kronrod system as a system of
        // its own (same image, components and tables, Gauss nodes only) for
        // the per-pixel error estimate
        shg[s] = S;
        nng_v[s] = 0;
        if (d.rule == LENSED_RULE_GK) {
            std::vector<double> tg, wg;
            for (size_t a = 0; a < t.size(); ++a)
                if (wtg[a] != 0.0) {
                    tg.push_back(t[a]);
                    wg.push_back(wtg[a]);
                }
            append_rule(tg, wg, shg[s]);
            nng_v[s] = shg[s].nn;
            if (shg[s].pre_off >= 0) shg[s].pre_off = -2;  // second table, placed after the loop
        }
    }

    lensed_model *m = new lensed_model();
    m->sys_gauss_h = shg;
    m->n_nodes_gauss = nng_v;
    m->precision = precision;
    m->n_sys = n_systems;
    m->n_par_max = n_par_max;
    m->C_total = C_total;
    m->total_pix = total_pix;
    m->T_total = T_total;
    m->sys_h = sh;
    m->need_count = need_count;
    m->n_nodes = nn_v;
    m->psf_p = pp;
    m->psf_q = qq;
    m->tiles_all = tiles_all;
    m->ray_flops = ray_flops_v;
    m->ray_transc = ray_transc_v;
    cudaGetDevice(&m->device);

    // PSF block tables: chi^2 tiles grouped by q (systems contiguous);
    // render tiles per system (all tiles)
    m->psf_sys_off.assign(n_systems, 0);
    m->psf_sys_cnt.assign(n_systems, 0);
    for (int q = 0; q <= LENSED_MAX_PSF_HALF; ++q)
        for (int sep = 0; sep <= 1; ++sep) {
            PsfGroup g{q, 0, (int)m->psf_blocks_h.size(), 0, 0};
            for (int s = 0; s < n_systems; ++s) {
                if (qq[s] != q || (sep_v[s] > 0) != (sep == 1) || chi_tiles[s].empty()) continue;
                m->psf_sys_off[s] = (int)m->psf_blocks_h.size();
                m->psf_sys_cnt[s] = (int)chi_tiles[s].size();
                m->psf_blocks_h.insert(m->psf_blocks_h.end(), chi_tiles[s].begin(),
                                       chi_tiles[s].end());
                g.p_max = std::max(g.p_max, pp[s]);
                g.sep = std::max(g.sep, sep_v[s]);
            }
            g.count = (int)m->psf_blocks_h.size() - g.off;
            if (g.count > 0) m->psf_groups.push_back(g);
        }
    m->psf_sep = sep_v;
    m->render_psf_off.assign(n_systems, 0);
    m->render_psf_cnt.assign(n_systems, 0);
    for (int s = 0; s < n_systems; ++s) {
        m->render_psf_off[s] = (int)m->render_psf_h.size();
        for (int ty = 0; ty < sh[s].tiles_y; ++ty)
            for (int tx = 0; tx < sh[s].tiles_x; ++tx)
                m->render_psf_h.push_back({s, 0, ty * kTileH, tx * kTileW, ~0u, ~0u});
        m->render_psf_cnt[s] = (int)m->render_psf_h.size() - m->render_psf_off[s];
    }

    int rc;
    init_kernel_attributes();
    if ((rc = m->sys.upload(sh)) || (rc = m->sys_gauss.upload(shg)) || (rc = m->comp_type.upload(ctype)) ||
        (rc = m->comp_plane.upload(cplane)) || (rc = m->comp_free.upload(cfree)) || (rc = m->comp_sys.upload(csys)) ||
        (rc = m->comp_value.upload(cval)) || (rc = m->data.upload(data)) ||
        (rc = m->weight.upload(weight)) ||
        (rc = m->data_d.upload(precision == LENSED_PREC_FP64 ? data_d : std::vector<double>())) ||
        (rc = m->weight_d.upload(precision == LENSED_PREC_FP64 ? weight_d : std::vector<double>())) || (rc = m->psf_f.upload(psf_f)) ||
        (rc = m->psf_d.upload(psf_d)) || (rc = m->node_u.upload(node_u)) ||
        (rc = m->node_w.upload(node_w)) || (rc = m->node_ud.upload(node_ud)) ||
        (rc = m->node_wd.upload(node_wd)) || (rc = m->need.upload(need)) ||
        (rc = m->psf_blocks.upload(m->psf_blocks_h)) || (rc = m->bn_table.upload(build_bn_table())) ||
        (rc = m->render_psf.upload(m->render_psf_h))) {
        std::string msg = g_last_error;
        delete m;
        g_last_error = msg;
        return rc;
    }
    if ((rc = build_trace_tables(m, m->cfg().trace_threads)) ||
        (rc = m->rcf.alloc((size_t)C_total * kNC)) || (rc = m->rcd.alloc((size_t)C_total * kNC)) ||
        (rc = m->rvalid.alloc(n_systems)) || (rc = m->rcvalid.alloc((size_t)C_total))) {
        std::string msg = g_last_error;
        delete m;
        g_last_error = msg;
        return rc;
    }
    size_t max_npix = 0;
    for (auto &S : sh) max_npix = std::max(max_npix, (size_t)S.npix);
    bool any_gk = false;
    for (int s = 0; s < n_systems; ++s) any_gk |= systems[s].rule == LENSED_RULE_GK;
    if ((rc = m->rL.alloc(total_pix * m->elem())) ||
        (any_gk && (rc = m->rLg.alloc(total_pix * m->elem())))) {
        std::string msg = g_last_error;
        delete m;
        g_last_error = msg;
        return rc;
    }
    if ((rc = precompute_fixed_light(m, cplane_pre, data_d, psf_d, psfd_off))) {
        std::string msg = g_last_error;
        delete m;
        g_last_error = msg;
        return rc;
    }
    cudaError_t e = cudaStreamCreateWithFlags(&m->cap_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        delete m;
        return fail(LENSED_E_CUDA, "create: %s", cudaGetErrorString(e));
    }
    *out = m;
    return LENSED_OK;
}

extern "C" void lensed_destroy(lensed_model *m) { delete m; }

extern "C" int lensed_model_info_get(const lensed_model *m, lensed_model_info *info)
{
    if (check_model(m)) return LENSED_E_ARG;
    if (!info) return fail(LENSED_E_ARG, "info is NULL");
    info->n_systems = m->n_sys;
    info->n_params_max = m->n_par_max;
    info->precision = m->precision;
    info->total_pixels = m->total_pix;
    long long all = 0, traced = 0, taps = 0;
    double fl = 0.0, tr = 0.0;
    for (int s = 0; s < m->n_sys; ++s) {
        const long long rays = (long long)m->n_nodes[s] * m->n_nodes[s];
        all += (long long)m->sys_h[s].npix * rays;
        traced += (long long)m->need_count[s] * rays;
        fl += (double)m->need_count[s] * rays * m->ray_flops[s];
        tr += (double)m->need_count[s] * rays * m->ray_transc[s];
        taps += (long long)m->psf_sys_cnt[s] * kTileW * kTileH * (2 * m->psf_p[s] + 1) *
                (2 * m->psf_q[s] + 1);
    }
    info->rays_per_eval_all = all;
    info->rays_per_eval_traced = traced;
    info->psf_taps_per_eval = taps;
    info->flops_per_ray = traced > 0 ? fl / traced : 0.0;
    info->transcendentals_per_ray = traced > 0 ? tr / traced : 0.0;
    return LENSED_OK;
}

extern "C" int lensed_render(lensed_model *m, int system, const double *params, int flags,
                             float *out_image, void *stream)
{
    if (check_model(m)) return LENSED_E_ARG;
    if (system < 0 || system >= m->n_sys) return fail(LENSED_E_ARG, "system %d out of range", system);
    if (!params || !out_image) return fail(LENSED_E_ARG, "params/out_image is NULL");
    if (flags != LENSED_RENDER_CONVOLVED && flags != LENSED_RENDER_UNCONVOLVED)
        return fail(LENSED_E_ARG, "unknown flags %d", flags);
    cudaStream_t st = (cudaStream_t)stream;
    const SysDev &S = m->sys_h[system];
    // one point: consts at p = 0, valid at index system (P = 1)
    launch_prologue(m->sys.p, m->comp_sys.p, system, 1, S.comp_off, S.ncomp, m->comp_type.p,
                    m->comp_free.p, m->comp_value.p, params, true, 1, 0, 1, m->n_par_max,
                    m->C_total, m->bn_table.p, m->rcf.p, m->rcd.p, m->rcvalid.p, m->rvalid.p, st);
    launch_trace(m->precision, m->cfg(), m->n_nodes[system], m->sys.p, m->comp_type.p,
                 m->comp_plane.p, m->rcf.p,
                 m->rcd.p, m->rvalid.p, 1, m->C_total,
                 m->render_trace.p + m->render_trace_off[system], m->render_trace_cnt[system],
                 nullptr, m->nodes(), 0, 1, m->rL.p, m->total_pix, st);
    if (is_mixed(m->precision))
        launch_fix64(m->cfg(), m->sys.p, system, 1, m->comp_type.p, m->comp_plane.p, m->rcf.p,
                     m->rcd.p, m->rvalid.p, 1, m->C_total, nullptr, m->nodes(), 0, 1, m->rL.p,
                     m->total_pix, st);
    if (flags == LENSED_RENDER_UNCONVOLVED) {
        launch_copy_image(m->precision, m->rL.p, S.pix_off, S.npix, m->rvalid.p + system,
                          out_image, st);
    } else {
        launch_psf(m->precision, m->psf_q[system], m->cfg().psf_sep ? m->psf_sep[system] : 0,
                   m->psf_p[system],
                   m->sys.p, m->psf_f.p,
                   m->psf_d.p, m->data.p, m->weight.p, m->data_d.p, m->weight_d.p, m->rvalid.p, 1,
                   m->render_psf.p + m->render_psf_off[system], m->render_psf_cnt[system], 0, 1,
                   m->rL.p, m->total_pix, nullptr, 0, out_image, st);
    }
    CUDA_OK(cudaGetLastError());
    return LENSED_OK;
}

extern "C" int lensed_measure_alu_peaks(double *fma_tflops, double *mufu_tops, void *stream)
{
    if (!fma_tflops || !mufu_tops) return fail(LENSED_E_ARG, "NULL output");
    int dev = 0, sms = 0;
    CUDA_OK(cudaGetDevice(&dev));
    CUDA_OK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    cudaStream_t st = (cudaStream_t)stream;
    DevBuf<float> sink;
    int rc = sink.alloc((size_t)sms * 8);
    if (rc) return rc;
    cudaEvent_t e0, e1;
    CUDA_OK(cudaEventCreate(&e0));
    CUDA_OK(cudaEventCreate(&e1));
    const int blocks = sms * 8, threads = 256;
    const int iters[2] = {1 << 14, 1 << 12};
    double out[2];
    for (int mufu = 0; mufu < 2; ++mufu) {
        float best = 1e30f;
        for (int rep = 0; rep < 4; ++rep) {
            cudaEventRecord(e0, st);
            launch_probe(mufu, blocks, threads, iters[mufu], sink.p, st);
            cudaEventRecord(e1, st);
            CUDA_OK(cudaEventSynchronize(e1));
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (rep > 0) best = std::min(best, ms);  // the first launch warms up
        }
        const double ops = (double)blocks * threads * iters[mufu] * 8;
        out[mufu] = ops * (mufu ? 1.0 : 2.0) / (best * 1e-3) / 1e12;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    CUDA_OK(cudaGetLastError());
    *fma_tflops = out[0];
    *mufu_tops = out[1];
    return LENSED_OK;
}

extern "C" int lensed_eval_sie_trig(const float *n, const float *d, long long count, float *out,
                                    void *stream)
{
    if (count < 0) return fail(LENSED_E_ARG, "negative count");
    if (count > 0 && (!n || !d || !out)) return fail(LENSED_E_ARG, "NULL pointer");
    launch_trig_probe(n, d, count, out, (cudaStream_t)stream);
    CUDA_OK(cudaGetLastError());
    return LENSED_OK;
}

extern "C" int lensed_rule_nodes(int rule, int order, double *t, double *w, double *w_gauss)
{
    if (!t || !w) return fail(LENSED_E_ARG, "t/w is NULL");
    if (rule < LENSED_RULE_POINT || rule > LENSED_RULE_GK)
        return fail(LENSED_E_ARG, "unknown rule %d", rule);
    std::vector<double> tt, ww, wg;
    if (!rule_nodes(rule, order, tt, ww, &wg))
        return fail(LENSED_E_ARG, "rule %d: order %d out of range", rule, order);
    for (size_t a = 0; a < tt.size(); ++a) {
        t[a] = tt[a];
        w[a] = ww[a];
        if (w_gauss) w_gauss[a] = rule == LENSED_RULE_GK ? wg[a] : 0.0;
    }
    return (int)tt.size();
}

extern "C" int lensed_render_error(lensed_model *m, int system, const double *params,
                                   float *out_error, void *stream)
{
    if (check_model(m)) return LENSED_E_ARG;
    if (system < 0 || system >= m->n_sys) return fail(LENSED_E_ARG, "system %d out of range", system);
    if (!params || !out_error) return fail(LENSED_E_ARG, "params/out_error is NULL");
    if (m->n_nodes_gauss[system] == 0)
        return fail(LENSED_E_ARG, "system %d: rule is not Gauss-Kronrod (no error estimate)", system);
    cudaStream_t st = (cudaStream_t)stream;
    const SysDev &S = m->sys_h[system];
    launch_prologue(m->sys.p, m->comp_sys.p, system, 1, S.comp_off, S.ncomp, m->comp_type.p,
                    m->comp_free.p, m->comp_value.p, params, true, 1, 0, 1, m->n_par_max,
                    m->C_total, m->bn_table.p, m->rcf.p, m->rcd.p, m->rcvalid.p, m->rvalid.p, st);
    // the Kronrod and the embedded Gauss luminosities, each with the trace
    // (and MIXED fix-up) kernels of lensed_render
    for (int g = 0; g < 2; ++g) {
        const SysDev *sys = g ? m->sys_gauss.p : m->sys.p;
        void *L = g ? (void *)m->rLg.p : (void *)m->rL.p;
        const int nn = g ? m->n_nodes_gauss[system] : m->n_nodes[system];
        launch_trace(m->precision, m->cfg(), nn, sys, m->comp_type.p, m->comp_plane.p, m->rcf.p,
                     m->rcd.p, m->rvalid.p, 1, m->C_total,
                     m->render_trace.p + m->render_trace_off[system], m->render_trace_cnt[system],
                     nullptr, m->nodes(), 0, 1, L, m->total_pix, st);
        if (is_mixed(m->precision))
            launch_fix64(m->cfg(), sys, system, 1, m->comp_type.p, m->comp_plane.p, m->rcf.p,
                         m->rcd.p, m->rvalid.p, 1, m->C_total, nullptr, m->nodes(), 0, 1, L,
                         m->total_pix, st);
    }
    launch_error_image(m->precision, m->rL.p, m->rLg.p, S.pix_off, S.npix, m->rvalid.p + system,
                       out_error, st);
    CUDA_OK(cudaGetLastError());
    return LENSED_OK;
}

static int loglike_args(lensed_model *m, const double *params, int P, double *out)
{
    if (check_model(m)) return LENSED_E_ARG;
    if (!params || !out) return fail(LENSED_E_ARG, "params/out is NULL");
    if (P < 1) return fail(LENSED_E_ARG, "P = %d must be >= 1", P);
    return LENSED_OK;
}

static int run_batch(lensed_model *m, const double *params, int P, double *out, cudaStream_t st,
                     bool use_graph)
{
    int rc = ensure_capacity(m, P);
    if (rc) return rc;
    LaunchCfg cfg = m->cfg();
    if ((rc = build_trace_tables(m, cfg.trace_threads))) return rc;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (st) cudaStreamIsCapturing(st, &cs);
    if (!use_graph || cs != cudaStreamCaptureStatusNone) {
        enqueue_batch(m, params, P, out, cfg, st);
        CUDA_OK(cudaGetLastError());
        return LENSED_OK;
    }
    // graph cache keyed by (P, params, out, configuration)
    GraphEntry *hit = nullptr;
    for (auto &g : m->graphs)
        if (g.P == P && g.params == params && g.out == out && g.cfg == m->cfg_index &&
            g.chunk == m->chunk())
            hit = &g;
    if (!hit) {
        if (m->graphs.size() >= kGraphCache) {
            auto old = std::min_element(m->graphs.begin(), m->graphs.end(),
                                        [](const GraphEntry &a, const GraphEntry &b) {
                                            return a.age < b.age;
                                        });
            cudaGraphExecDestroy(old->exec);
            m->graphs.erase(old);
        }
        cudaGraph_t graph;
        CUDA_OK(cudaStreamBeginCapture(m->cap_stream, cudaStreamCaptureModeThreadLocal));
        enqueue_batch(m, params, P, out, cfg, m->cap_stream);
        cudaError_t e1 = cudaGetLastError();
        cudaError_t e2 = cudaStreamEndCapture(m->cap_stream, &graph);
        if (e1 != cudaSuccess || e2 != cudaSuccess)
            return fail(LENSED_E_CUDA, "graph capture: %s / %s", cudaGetErrorString(e1),
                        cudaGetErrorString(e2));
        cudaGraphExec_t exec;
        cudaError_t e3 = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e3 != cudaSuccess)
            return fail(LENSED_E_CUDA, "graph instantiate: %s", cudaGetErrorString(e3));
        m->graphs.push_back({P, params, out, m->cfg_index, m->chunk(), exec, 0});
        hit = &m->graphs.back();
    }
    hit->age = ++m->graph_clock;
    CUDA_OK(cudaGraphLaunch(hit->exec, st));
    return LENSED_OK;
}

extern "C" int lensed_loglike_batch(lensed_model *m, const double *params, int P,
                                    double *out_loglike, void *stream)
{
    int rc = loglike_args(m, params, P, out_loglike);
    if (rc) return rc;
    return run_batch(m, params, P, out_loglike, (cudaStream_t)stream, true);
}

extern "C" int lensed_loglike_plain(lensed_model *m, const double *params, int P,
                                    double *out_loglike, void *stream)
{
    int rc = loglike_args(m, params, P, out_loglike);
    if (rc) return rc;
    if ((rc = ensure_capacity(m, P))) return rc;
    LaunchCfg cfg = m->cfg();
    if ((rc = build_trace_tables(m, cfg.trace_threads))) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    for (int s = 0; s < m->n_sys; ++s) {
        for (int p = 0; p < P; ++p) {
            launch_prologue(m->sys.p, m->comp_sys.p, s, 1, m->sys_h[s].comp_off,
                            m->sys_h[s].ncomp, m->comp_type.p, m->comp_free.p, m->comp_value.p,
                            params, false, P, p, 1, m->n_par_max, m->C_total, m->bn_table.p,
                            m->cf.p, m->cd.p, m->cvalid.p, m->valid.p, st);
            launch_trace(m->precision, cfg, m->n_nodes[s], m->sys.p, m->comp_type.p,
                         m->comp_plane.p, m->cf.p,
                         m->cd.p, m->valid.p, P, m->C_total,
                         m->trace_blocks.p + m->trace_sys_off[s], m->trace_sys_cnt[s], m->need.p,
                         m->nodes_chi(), p, 1, m->Lbuf.p, m->total_pix, st);
            if (is_mixed(m->precision))
                launch_fix64(cfg, m->sys.p, s, 1, m->comp_type.p, m->comp_plane.p, m->cf.p,
                             m->cd.p, m->valid.p, P, m->C_total, m->need.p, m->nodes_chi(), p, 1,
                             m->Lbuf.p, m->total_pix, st);
            if (m->psf_sys_cnt[s] > 0)
                launch_psf(m->precision, m->psf_q[s], cfg.psf_sep ? m->psf_sep[s] : 0, m->psf_p[s],
                           m->sys.p,
                           m->psf_f.p,
                           m->psf_d.p, m->data.p, m->weight.p, m->data_d.p, m->weight_d.p, m->valid.p, P,
                           m->psf_blocks.p + m->psf_sys_off[s], m->psf_sys_cnt[s], p, 1,
                           m->Lbuf.p, m->total_pix, m->partial.p, m->T_total, nullptr, st);
            launch_finalize(m->sys.p, m->valid.p, P, m->partial.p, m->T_total, out_loglike, s,
                            p, 1, 1, st);
        }
    }
    CUDA_OK(cudaGetLastError());
    return LENSED_OK;
}

extern "C" int lensed_loglike_batch_host(lensed_model *m, const double *params_host, int P,
                                         double *out_host, void *stream)
{
    int rc = loglike_args(m, params_host, P, out_host);
    if (rc) return rc;
    const size_t np = (size_t)m->n_sys * P * m->n_par_max;
    const size_t no = (size_t)m->n_sys * P;
    if (m->stage_params.n < std::max<size_t>(np, 1) || m->stage_out.n < no) {
        cudaDeviceSynchronize();
        m->clear_graphs();
        if ((rc = m->stage_params.alloc(np)) || (rc = m->stage_out.alloc(no))) return rc;
    }
    cudaStream_t st = (cudaStream_t)stream;
    CUDA_OK(cudaMemcpyAsync(m->stage_params.p, params_host, np * sizeof(double),
                            cudaMemcpyHostToDevice, st));
    if ((rc = run_batch(m, m->stage_params.p, P, m->stage_out.p, st, true))) return rc;
    CUDA_OK(cudaMemcpyAsync(out_host, m->stage_out.p, no * sizeof(double), cudaMemcpyDeviceToHost,
                            st));
    CUDA_OK(cudaStreamSynchronize(st));
    return LENSED_OK;
}

extern "C" int lensed_autotune(lensed_model *m, const double *params, int P, void *stream)
{
    int rc = loglike_args(m, params, P, (double *)params);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    DevBuf<double> tmp;
    if ((rc = tmp.alloc((size_t)m->n_sys * P))) return rc;
    if ((rc = ensure_capacity(m, P))) return rc;
    cudaEvent_t e0, e1;
    CUDA_OK(cudaEventCreate(&e0));
    CUDA_OK(cudaEventCreate(&e1));
    // best of 3 timed runs (each after an untimed one) of the current setting
    auto time_batch = [&](float *t_min) -> int {
        *t_min = 1e30f;
        for (int rep = 0; rep < 3; ++rep) {
            int r = run_batch(m, params, P, tmp.p, st, false);
            if (r) return r;
            cudaEventRecord(e0, st);
            run_batch(m, params, P, tmp.p, st, false);
            cudaEventRecord(e1, st);
            if (cudaEventSynchronize(e1) != cudaSuccess)
                return fail(LENSED_E_CUDA, "autotune: %s", cudaGetErrorString(cudaGetLastError()));
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            *t_min = std::min(*t_min, ms);
        }
        return LENSED_OK;
    };
    const int saved = m->cfg_index, saved_limit = m->chunk_limit;
    // First stage: every launch configuration, each over whole scratch chunks.
    m->chunk_limit = 0;
    float best = 1e30f, t = 0.f;
    int best_i = 0;
    for (int i = 0; i < m->n_candidates() && !rc; ++i) {
        m->cfg_index = i;
        if ((rc = time_batch(&t))) break;
        if (t < best) {
            best = t;
            best_i = i;
        }
    }
    // Second stage, with the chosen configuration: whole scratch chunks, or
    // chunks whose pixel luminosities fit in half or a quarter of L2, so the
    // PSF pass reads what the trace pass left in L2 (smaller chunks also
    // mean more launches and more launch tails; timing decides).
    int best_limit = 0;
    if (!rc) {
        m->cfg_index = best_i;
        int l2_bytes = 0;
        cudaDeviceGetAttribute(&l2_bytes, cudaDevAttrL2CacheSize, m->device);
        const size_t per_point = std::max<size_t>(1, (size_t)m->total_pix * m->elem());
        const int limits[2] = {(int)std::max<size_t>(1, (size_t)std::max(l2_bytes, 0) / 2 / per_point),
                               (int)std::max<size_t>(1, (size_t)std::max(l2_bytes, 0) / 4 / per_point)};
        for (int li = 0; li < 2 && !rc && l2_bytes > 0; ++li) {
            if (limits[li] >= std::min(m->chunk_P, P)) continue;  // one chunk already
            if (li > 0 && limits[li] == limits[li - 1]) continue;  // timed already
            m->chunk_limit = limits[li];
            if ((rc = time_batch(&t))) break;
            if (t < best) {
                best = t;
                best_limit = limits[li];
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) {
        m->cfg_index = saved;
        m->chunk_limit = saved_limit;
        return rc;
    }
    m->chunk_limit = best_limit;
    LaunchCfg cfg = m->cfg();
    if ((rc = build_trace_tables(m, cfg.trace_threads))) return rc;
    CUDA_OK(cudaStreamSynchronize(st));
    return LENSED_OK;
}

extern "C" int lensed_batch_plan(lensed_model *m, int P, int *launches, int *chunk_points)
{
    if (check_model(m)) return LENSED_E_ARG;
    if (P < 1 || !launches || !chunk_points) return fail(LENSED_E_ARG, "bad arguments");
    int rc = ensure_capacity(m, P);
    if (rc) return rc;
    const int chunks = (P + m->chunk() - 1) / m->chunk();
    // a MIXED_FF second pass: three more kernels (pixel refinement, re-trace,
    // apply) per trace group of at most 8 nodes per row
    int second = 0;
    if (m->precision == LENSED_PREC_MIXED_FF && m->cfg().ff_split && m->ffq_cnt.p)
        for (const TraceGroup &g : m->trace_groups) second += 3 * (g.nn >= 1 && g.nn <= 8);
    *launches = 3 + chunks * ((int)m->trace_groups.size() + (int)m->psf_groups.size() +
                              (is_mixed(m->precision) ? 1 : 0) + second);
    *chunk_points = m->chunk();
    return LENSED_OK;
}

extern "C" int lensed_profile_batch(lensed_model *m, const double *params, int P,
                                    double *out_loglike, void *stream, double *stage_ms,
                                    int *trace_launches)
{
    int rc = loglike_args(m, params, P, out_loglike);
    if (rc) return rc;
    if (!stage_ms) return fail(LENSED_E_ARG, "stage_ms is NULL");
    if ((rc = ensure_capacity(m, P))) return rc;
    LaunchCfg cfg = m->cfg();
    if ((rc = build_trace_tables(m, cfg.trace_threads))) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    StageTimer tm;
    tm.st = st;
    enqueue_batch(m, params, P, out_loglike, cfg, st, &tm);
    CUDA_OK(cudaGetLastError());
    CUDA_OK(cudaStreamSynchronize(st));
    for (int k = 0; k < 4; ++k) stage_ms[k] = 0.0;
    int nt = 0;
    for (auto &mk : tm.marks) {
        float ms = 0.f;
        CUDA_OK(cudaEventElapsedTime(&ms, mk.second.first, mk.second.second));
        stage_ms[mk.first] += ms;
        nt += mk.first == 1;
    }
    if (trace_launches) *trace_launches = nt;
    return LENSED_OK;
}

extern "C" int lensed_set_config(lensed_model *m, int index)
{
    if (check_model(m)) return LENSED_E_ARG;
    if (index < -1 || index >= m->n_candidates())
        return fail(LENSED_E_ARG, "configuration %d out of range (-1..%d)", index,
                    m->n_candidates() - 1);
    m->cfg_index = index;
    int rc = build_trace_tables(m, m->cfg().trace_threads);
    if (rc) return rc;
    return m->n_candidates();
}

extern "C" int lensed_set_chunk_points(lensed_model *m, int points)
{
    if (check_model(m)) return LENSED_E_ARG;
    if (points < 0) return fail(LENSED_E_ARG, "points per chunk = %d must be >= 0", points);
    m->chunk_limit = points;
    return LENSED_OK;
}

extern "C" int lensed_tuned_config(const lensed_model *m, char *buf, int buflen)
{
    if (check_model(m)) return -1;
    if (buf && buflen > 0) {
        const char *name = kCandidates[m->cfg_index < 0 ? 0 : m->cfg_index].name;
        char lim[64] = "";
        if (m->chunk_limit > 0)
            snprintf(lim, sizeof(lim), ", at most %d points per scratch chunk", m->chunk_limit);
        snprintf(buf, (size_t)buflen, "%s%s%s", name, lim, m->cfg_index < 0 ? " (default)" : "");
    }
    return m->cfg_index;
}

// ===========================================================================
// Allocation-free evaluation (lensed_loglike_batch_noalloc)
//
// Its scratch is this file-scope device array.  In host code the symbol is
// only a stand-in: the device address comes from cudaGetSymbolAddress, once
// per device, with that device current.

namespace {

constexpr size_t kStaticScratchBytes = (size_t)32 << 20;  // 32 MiB
__device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

std::mutex g_static_mu;
void *g_static_ptr[256] = {nullptr};

int static_scratch_address(void **out)
{
    int dev = 0;
    CUDA_OK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 256) return fail(LENSED_E_UNSUPPORTED, "device index %d", dev);
    std::lock_guard<std::mutex> lock(g_static_mu);
    if (!g_static_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess || !p)
            return fail(LENSED_E_CUDA, "cudaGetSymbolAddress(static scratch): %s",
                        cudaGetErrorString(e));
        g_static_ptr[dev] = p;
    }
    *out = g_static_ptr[dev];
    return LENSED_OK;
}

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

}  // namespace

extern "C" int lensed_loglike_batch_noalloc(lensed_model *m, const double *params, int P,
                                            double *out_loglike, void *stream)
{
    int rc = loglike_args(m, params, P, out_loglike);
    if (rc) return rc;
    // carve the fixed array: constants, validity, partials, then as many
    // points' pixel luminosities as fit
    const size_t Pz = (size_t)P;
    const size_t b_cf = align256(Pz * m->C_total * kNC * sizeof(float));
    const size_t b_cd = align256(Pz * m->C_total * kNC * sizeof(double));
    const size_t b_cv = align256(Pz * m->C_total);
    const size_t b_v = align256(Pz * m->n_sys);
    const size_t b_part = align256(Pz * std::max(m->T_total, 1) * sizeof(double));
    const size_t fixed = b_cf + b_cd + b_cv + b_v + b_part;
    const size_t per_point = (size_t)m->total_pix * m->elem();
    if (fixed >= kStaticScratchBytes || (kStaticScratchBytes - fixed) / per_point < 1) {
        const size_t per = (size_t)m->C_total * kNC * 12 + m->C_total + m->n_sys +
                           (size_t)std::max(m->T_total, 1) * 8;
        const size_t pmax = kStaticScratchBytes > per_point + 5 * 256
                                ? (kStaticScratchBytes - per_point - 5 * 256) / per
                                : 0;
        return fail(LENSED_E_ARG,
                    "P = %d needs more than the %zu bytes of fixed scratch of "
                    "lensed_loglike_batch_noalloc (about %zu points fit for this model)",
                    P, kStaticScratchBytes, pmax);
    }
    const int chunk = (int)std::min<size_t>(Pz, (kStaticScratchBytes - fixed) / per_point);
    void *base = nullptr;
    if ((rc = static_scratch_address(&base))) return rc;
    unsigned char *b = (unsigned char *)base;
    float *cf = (float *)b;
    double *cd = (double *)(b + b_cf);
    unsigned char *cvalid = b + b_cf + b_cd;
    unsigned char *valid = cvalid + b_cv;
    double *partial = (double *)(valid + b_v);
    void *Lbuf = (unsigned char *)partial + b_part;

    cudaStream_t st = (cudaStream_t)stream;
    const LaunchCfg cfg = m->cfg();
    launch_prologue(m->sys.p, m->comp_sys.p, 0, m->n_sys, 0, m->C_total, m->comp_type.p,
                    m->comp_free.p, m->comp_value.p, params, false, P, 0, P, m->n_par_max,
                    m->C_total, m->bn_table.p, cf, cd, cvalid, valid, st);
    for (int p0 = 0; p0 < P; p0 += chunk) {
        const int nP = std::min(chunk, P - p0);
        // no second-pass queue here (it lives in model-owned memory): in
        // MIXED_FF the trace blocks always re-trace their own rays, which
        // gives the same bits as the second pass would
        for (const TraceGroup &g : m->trace_groups)
            launch_trace(m->precision, cfg, g.nn, m->sys.p, m->comp_type.p, m->comp_plane.p, cf,
                         cd, valid, P, m->C_total, m->trace_blocks.p + g.off, g.count, m->need.p,
                         m->nodes_chi(), p0, nP, Lbuf, m->total_pix, st);
        if (is_mixed(m->precision))
            launch_fix64(cfg, m->sys.p, 0, m->n_sys, m->comp_type.p, m->comp_plane.p, cf, cd,
                         valid, P, m->C_total, m->need.p, m->nodes_chi(), p0, nP, Lbuf,
                         m->total_pix, st);
        for (const PsfGroup &g : m->psf_groups)
            launch_psf(m->precision, g.q, cfg.psf_sep ? g.sep : 0, g.p_max, m->sys.p, m->psf_f.p, m->psf_d.p, m->data.p,
                       m->weight.p, m->data_d.p, m->weight_d.p, valid, P,
                       m->psf_blocks.p + g.off, g.count, p0, nP, Lbuf, m->total_pix, partial,
                       m->T_total, nullptr, st);
    }
    launch_finalize(m->sys.p, valid, P, partial, m->T_total, out_loglike, 0, 0, m->n_sys, P, st);
    CUDA_OK(cudaGetLastError());
    return LENSED_OK;
}
