/*
 * Plain FP64 CPU oracle of the Lensed forward model and likelihood
 * (Tessore, Bellagamba & Metcalf, "Lensed: a code for the forward
 * reconstruction of lenses and sources from strong lensing observations").
 *
 * TEST INFRASTRUCTURE ONLY.  The test suite, the smoke check and the CPU
 * baseline leg of the benchmark are the only code that may load this file.
 * It shares no code, header, table or helper with the CUDA library, and the
 * CUDA library never calls it.
 *
 * Everything is written as the paper states it, in the paper's order, with
 * no blocking, fusion or reordering:
 *   Sec. 2.1  Eq. 1  lens equation          y = x - alpha(x)
 *             Eq. 2  image-plane brightness I(x) = I_L(x) + I_S(y(x))
 *             Eq. 3  pixel luminosity       L_i = integral of I over pixel i
 *   Sec. 3.1  Eq. 14 quadrature             L_i ~ sum_k w_k I(x_k)
 *                    (rules of Sec. 4.5: point, subN, Gauss-Kronrod gNk(2N+1)
 *                     as the Cartesian square of the 1-D rule; the embedded
 *                     N x N Gauss rule gives the per-pixel error estimate
 *                     |L_Kronrod - L_Gauss| of the unconvolved luminosity)
 *             Eq. 15 discrete PSF           L*_ij = sum_kl F_{-k,-l} L_{i+k,j+l}
 *                    (PSF normalised to unit sum; border padded by repeating
 *                     the nearest pixel)
 *   Sec. 3.2  Eq. 17 loglike = -1/2 sum_i w_i (d_i - L_i)^2, w_i = 1/s_i^2,
 *                    masked pixels have w_i = 0
 *   Sec. 3.3  Eq. 21 s_i^2 = (d_i + b_i)/g_i when no variance is given, plus a
 *                    multiplicative extra weight factor
 *   Sec. 4.1  Eqs. 22-23 elliptical Sersic law with geometric-mean radius
 *
 * Readings where the paper is silent (each also listed in the design notes):
 *   - pixel (i, j) has centre ((j - (nx-1)/2) h, (i - (ny-1)/2) h); row i runs
 *     along +y, column j along +x; the pixel is a square of side h;
 *   - position angles are counter-clockwise from +x to the major axis, in
 *     degrees;
 *   - SIE with core s in the geometric-mean convention:
 *       kappa = b sqrt(q) / (2 psi),  psi = sqrt(q^2 (s^2 + x^2) + y^2),
 *       alpha_x = (b sqrt(q)/e) atan (e x / (psi + s)),
 *       alpha_y = (b sqrt(q)/e) atanh(e y / (psi + q^2 s)),  e = sqrt(1 - q^2),
 *     with the series in e below e = 1e-3 (q = 1 is the softened SIS);
 *   - external shear alpha = (g1 dx + g2 dy, g2 dx - g1 dy), g1 = g cos 2phi,
 *     g2 = g sin 2phi, about its centre;
 *   - point mass alpha = thetaE^2 d / |d|^2, and alpha = 0 exactly at d = 0;
 *     likewise alpha = 0 exactly at the centre of a coreless SIE (s = 0);
 *   - Sersic b_n solves P(2n, b_n) = 1/2 exactly (regularised lower
 *     incomplete gamma); total flux F = 10^(-0.4 (mag - zp)) gives
 *     I_0 = F b_n^(2n) / (2 pi n r^2 Gamma(2n)); de Vaucouleurs is n = 4;
 *     the Gaussian profile is I_0 exp(-R^2 / (2 sigma^2)), I_0 = F/(2 pi sigma^2);
 *   - the flat sky (Sec. 5) is a constant surface brightness, in the image's
 *     flux units per arcsec^2 and of either sign (it absorbs residuals of
 *     the sky subtraction), on the foreground or source plane;
 *   - an image-plane prior (Sec. 5) gives a source's position parameters as
 *     an image-plane position theta; the source is centred on
 *     theta - alpha(theta) of the same parameter point's lens;
 *   - a parameter point with q outside (0, 1], a non-positive radius or
 *     Sersic index, a negative Einstein radius or core has loglike = -inf.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define ORA_PI 3.14159265358979323846

/* component types */
enum { ORA_SIE = 1, ORA_SHEAR = 2, ORA_POINTMASS = 3,
       ORA_SERSIC = 4, ORA_DEVAUC = 5, ORA_GAUSS = 6, ORA_SKY = 7 };
/* planes: mass on the lens plane, light on the lens plane (unlensed,
 * evaluated at x) or on the source plane (lensed, evaluated at y); a source
 * on ORA_PLANE_SOURCE_IMAGE gives its position as an image-plane position
 * (the image-plane prior of Sec. 5) */
enum { ORA_PLANE_LENS = 0, ORA_PLANE_FOREGROUND = 1, ORA_PLANE_SOURCE = 2,
       ORA_PLANE_SOURCE_IMAGE = 3 };
/* integration rules of Sec. 4.5 (point, subN, Gauss-Kronrod gNk(2N+1)) plus
 * Gauss-Legendre N x N */
enum { ORA_RULE_POINT = 0, ORA_RULE_SUB = 1, ORA_RULE_GL = 2, ORA_RULE_GK = 3 };

#define ORA_MAXPAR 8

typedef struct {
    int type;
    int plane;
    int free_index[ORA_MAXPAR]; /* index into xi, or -1 for a fixed value */
    double value[ORA_MAXPAR];   /* fixed values */
} ora_component;

typedef struct {
    int nx, ny;
    double h;                     /* pixel side, arcsec */
    const double *data;           /* [ny*nx], row-major, row i along +y */
    const double *variance;       /* [ny*nx] or NULL */
    double gain, offset;          /* Eq. 21, used when variance == NULL */
    const double *extra_weight;   /* [ny*nx] or NULL: multiplies w_i */
    const unsigned char *mask;    /* [ny*nx] or NULL: nonzero = excluded */
    const double *psf;            /* [psf_ny*psf_nx] or NULL (no PSF) */
    int psf_nx, psf_ny;           /* odd sizes 2q+1, 2p+1 */
    int rule, order;
    double zeropoint;
    int ncomp;
    const ora_component *comp;
    int nparam;
} ora_system;

int ora_nparams_of(int type)
{
    switch (type) {
    case ORA_SIE: return 6;       /* x, y, b, q, pa, s */
    case ORA_SHEAR: return 4;     /* x, y, gamma, phi */
    case ORA_POINTMASS: return 3; /* x, y, thetaE */
    case ORA_SERSIC: return 7;    /* x, y, r, mag, n, q, pa */
    case ORA_DEVAUC: return 6;    /* x, y, r, mag, q, pa */
    case ORA_GAUSS: return 6;     /* x, y, sigma, mag, q, pa */
    case ORA_SKY: return 1;       /* surface brightness per arcsec^2 */
    }
    return -1;
}

/* ------------------------------------------------------------------ */
/* Legendre polynomial P_n(x) and its derivative, three-term recurrence */
static void legendre(int n, double x, double *p, double *dp)
{
    double p0 = 1.0, p1 = x;
    if (n == 0) { *p = 1.0; *dp = 0.0; return; }
    for (int k = 2; k <= n; ++k) {
        double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
    }
    *p = p1;
    *dp = n * (x * p1 - p0) / (x * x - 1.0);
}

/* Gauss-Legendre nodes and weights on [-1, 1]: every root of P_n is found
 * by a sign change on a fine grid and refined by plain bisection; the
 * weight is 2 / ((1 - x^2) P_n'(x)^2).  Nodes are returned ascending.  The
 * grid has an odd number of intervals so that no grid point is x = 0. */
int ora_gauss_legendre(int n, double *x, double *w)
{
    if (n < 1 || n > 128) return -1;
    int grid = 256 * n + 1, found = 0;
    double a = -1.0, pa, dpa;
    legendre(n, a, &pa, &dpa);
    for (int g = 1; g <= grid && found < n; ++g) {
        double b = -1.0 + 2.0 * g / grid, pb, dpb;
        legendre(n, b, &pb, &dpb);
        if ((pa < 0.0) != (pb < 0.0)) {
            double lo = a, hi = b, plo = pa;
            for (int it = 0; it < 200; ++it) {
                double mid = 0.5 * (lo + hi), pm, dpm;
                if (mid <= lo || mid >= hi) break;
                legendre(n, mid, &pm, &dpm);
                if ((pm < 0.0) == (plo < 0.0)) { lo = mid; plo = pm; }
                else hi = mid;
            }
            double r = 0.5 * (lo + hi), pr, dpr;
            legendre(n, r, &pr, &dpr);
            x[found] = r;
            w[found] = 2.0 / ((1.0 - r * r) * dpr * dpr);
            ++found;
        }
        a = b;
        pa = pb;
    }
    return found == n ? 0 : -2;
}

/* Dense linear solve (Gaussian elimination with partial pivoting), n <= 64. */
static int solve(int n, double *A, double *b)
{
    for (int c = 0; c < n; ++c) {
        int piv = c;
        for (int r = c + 1; r < n; ++r)
            if (fabs(A[r * n + c]) > fabs(A[piv * n + c])) piv = r;
        if (A[piv * n + c] == 0.0) return -1;
        if (piv != c) {
            for (int k = 0; k < n; ++k) {
                double t = A[c * n + k]; A[c * n + k] = A[piv * n + k]; A[piv * n + k] = t;
            }
            double t = b[c]; b[c] = b[piv]; b[piv] = t;
        }
        for (int r = c + 1; r < n; ++r) {
            double f = A[r * n + c] / A[c * n + c];
            for (int k = c; k < n; ++k) A[r * n + k] -= f * A[c * n + k];
            b[r] -= f * b[c];
        }
    }
    for (int r = n - 1; r >= 0; --r) {
        double s = b[r];
        for (int k = r + 1; k < n; ++k) s -= A[r * n + k] * b[k];
        b[r] = s / A[r * n + r];
    }
    return 0;
}

/* Gauss-Kronrod rule with 2n+1 points on [-1, 1] (Kronrod's extension of the
 * n-point Gauss rule, the rules of Sec. 3.1 and Sec. 4.5, Patterson 1968).
 * The n+1 new nodes are the roots of the Stieltjes polynomial E_{n+1}: the
 * monic-in-P_{n+1} combination E = P_{n+1} + sum_j a_j P_j (j < n+1 of the
 * parity of n+1) with integral of P_n E P_k = 0 for k = 0..n, solved with the
 * integrals done by a 64-point Gauss-Legendre rule (exact here).  The
 * weights make the rule exact on P_0..P_{2n} (Legendre moments).  Outputs
 * the 2n+1 nodes ascending, the Kronrod weights wk and the embedded Gauss
 * weights wg (zero on the new nodes). */
int ora_gauss_kronrod(int n, double *x, double *wk, double *wg)
{
    if (n < 1 || n > 7) return -1;
    double gx[64], gw[64];
    if (ora_gauss_legendre(64, gx, gw) != 0) return -2;
    /* unknown coefficients a_j for j = n+1-2, n+1-4, ... >= 0 */
    int js[16], m = 0;
    for (int j = n - 1; j >= 0; j -= 2) js[m++] = j;
    /* conditions for k of the parity of n+1+n ... choose k with nonzero
     * integrals: k = 0..n with (n + k + j) even for some j; use the m
     * lowest such k */
    int ks[16], mk = 0;
    for (int k = 0; k <= n && mk < m; ++k)
        if ((n + k + (n + 1)) % 2 == 0) ks[mk++] = k;
    if (mk != m) return -3;
    double A[256], b[16];
    for (int r = 0; r < m; ++r) {
        double rhs = 0.0;
        for (int c = 0; c < m; ++c) A[r * m + c] = 0.0;
        for (int q = 0; q < 64; ++q) {
            double pn, d, pk, pj, pe;
            legendre(n, gx[q], &pn, &d);
            legendre(ks[r], gx[q], &pk, &d);
            legendre(n + 1, gx[q], &pe, &d);
            rhs -= gw[q] * pn * pk * pe;
            for (int c = 0; c < m; ++c) {
                legendre(js[c], gx[q], &pj, &d);
                A[r * m + c] += gw[q] * pn * pk * pj;
            }
        }
        b[r] = rhs;
    }
    if (m > 0 && solve(m, A, b) != 0) return -4;
    /* E(x) and its roots by sign changes + bisection */
    double ex[16];
    int found = 0, grid = 20001;
    double xa = -1.0, ea = 0.0, d;
    for (int g = 0; g <= grid; ++g) {
        double xb = -1.0 + 2.0 * g / grid, eb, t;
        legendre(n + 1, xb, &eb, &d);
        for (int c = 0; c < m; ++c) { legendre(js[c], xb, &t, &d); eb += b[c] * t; }
        if (g > 0 && (ea < 0.0) != (eb < 0.0)) {
            double lo = xa, hi = xb, elo = ea;
            for (int it = 0; it < 200; ++it) {
                double mid = 0.5 * (lo + hi), em;
                if (mid <= lo || mid >= hi) break;
                legendre(n + 1, mid, &em, &d);
                for (int c = 0; c < m; ++c) { legendre(js[c], mid, &t, &d); em += b[c] * t; }
                if ((em < 0.0) == (elo < 0.0)) { lo = mid; elo = em; } else hi = mid;
            }
            if (found < 16) ex[found++] = 0.5 * (lo + hi);
        }
        xa = xb;
        ea = eb;
    }
    if (found != n + 1) return -5;
    /* merge with the Gauss nodes, ascending */
    double gxn[16], gwn[16];
    if (ora_gauss_legendre(n, gxn, gwn) != 0) return -6;
    int N = 2 * n + 1, ig = 0, ie = 0;
    for (int k = 0; k < N; ++k) {
        if (ie < n + 1 && (ig >= n || ex[ie] < gxn[ig])) { x[k] = ex[ie++]; wg[k] = 0.0; }
        else { x[k] = gxn[ig]; wg[k] = gwn[ig]; ++ig; }
    }
    /* Kronrod weights: sum_i w_i P_k(x_i) = integral of P_k = 2 delta_k0 */
    double M[31 * 31], r[31];
    for (int k = 0; k < N; ++k) {
        for (int i = 0; i < N; ++i) { double p; legendre(k, x[i], &p, &d); M[k * N + i] = p; }
        r[k] = k == 0 ? 2.0 : 0.0;
    }
    if (solve(N, M, r) != 0) return -7;
    for (int i = 0; i < N; ++i) wk[i] = r[i];
    return 0;
}

/* 1-D rule on the unit pixel: abscissae t in (-1/2, 1/2), weights summing
 * to one (Eq. 14; the 2-D rule is the Cartesian square). */
int ora_rule_nodes(int rule, int order, double *t, double *wt)
{
    if (rule == ORA_RULE_POINT) { t[0] = 0.0; wt[0] = 1.0; return 1; }
    if (rule == ORA_RULE_SUB) {
        if (order < 1 || order > 64) return -1;
        for (int a = 0; a < order; ++a) {
            t[a] = (a + 0.5) / order - 0.5;
            wt[a] = 1.0 / order;
        }
        return order;
    }
    if (rule == ORA_RULE_GK) {
        double x[15], wk[15], wg[15];
        if (ora_gauss_kronrod(order, x, wk, wg) != 0) return -1;
        for (int a = 0; a < 2 * order + 1; ++a) { t[a] = 0.5 * x[a]; wt[a] = 0.5 * wk[a]; }
        return 2 * order + 1;
    }
    if (rule == ORA_RULE_GL) {
        if (order < 1 || order > 128) return -1;
        double *x = (double *)malloc(sizeof(double) * order);
        double *w = (double *)malloc(sizeof(double) * order);
        int rc = ora_gauss_legendre(order, x, w);
        for (int a = 0; a < order; ++a) { t[a] = 0.5 * x[a]; wt[a] = 0.5 * w[a]; }
        free(x);
        free(w);
        return rc == 0 ? order : -1;
    }
    return -1;
}

/* ------------------------------------------------------------------ */
/* Regularised lower incomplete gamma P(a, x) by its power series
 *   P(a, x) = x^a e^-x / Gamma(a+1) * sum_k x^k / ((a+1)...(a+k)),
 * which converges for every x >= 0 (used here only for x <= a). */
double ora_gammainc_lower(double a, double x)
{
    if (x <= 0.0) return 0.0;
    double term = 1.0, sum = 1.0;
    for (int k = 1; k < 100000; ++k) {
        term *= x / (a + k);
        sum += term;
        if (term < 1e-18 * sum) break;
    }
    return exp(a * log(x) - x - lgamma(a + 1.0)) * sum;
}

/* Sersic b_n: the root of P(2n, b) = 1/2 (r is the half-light radius,
 * Sec. 4.1), by bisection on [0, 2n]; P(2n, 0) = 0 and P(2n, 2n) > 1/2. */
double ora_sersic_bn(double n)
{
    double a = 2.0 * n, lo = 0.0, hi = 2.0 * n;
    for (int it = 0; it < 400; ++it) {
        double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        if (ora_gammainc_lower(a, mid) < 0.5) lo = mid;
        else hi = mid;
    }
    return 0.5 * (lo + hi);
}

/* ------------------------------------------------------------------ */
/* one component with its parameters resolved */
typedef struct {
    int type, plane;
    double p[ORA_MAXPAR];
    /* derived */
    double cos_pa, sin_pa, bn, inv_n, I0;
} ora_comp_eval;

static double deg2rad(double d) { return d * (ORA_PI / 180.0); }

void ora_deflection_one(int type, const double *p, double x, double y,
                        double *ax, double *ay);

/* Resolve parameters and derived constants; returns 0 if the point is
 * outside the valid domain of the component. */
static int resolve(const ora_system *sys, const double *xi, ora_comp_eval *ce)
{
    for (int c = 0; c < sys->ncomp; ++c) {
        const ora_component *cp = &sys->comp[c];
        ora_comp_eval *e = &ce[c];
        int np = ora_nparams_of(cp->type);
        if (np < 0) return 0;
        e->type = cp->type;
        e->plane = cp->plane;
        for (int k = 0; k < np; ++k)
            e->p[k] = cp->free_index[k] >= 0 ? xi[cp->free_index[k]] : cp->value[k];
        for (int k = 0; k < np; ++k)
            if (!isfinite(e->p[k])) return 0;
        double F, r, n, q, pa;
        switch (cp->type) {
        case ORA_SIE:
            q = e->p[3];
            if (!(q > 0.0 && q <= 1.0) || e->p[2] < 0.0 || e->p[5] < 0.0) return 0;
            e->cos_pa = cos(deg2rad(e->p[4]));
            e->sin_pa = sin(deg2rad(e->p[4]));
            break;
        case ORA_SHEAR:
            e->cos_pa = cos(2.0 * deg2rad(e->p[3]));
            e->sin_pa = sin(2.0 * deg2rad(e->p[3]));
            break;
        case ORA_POINTMASS:
            if (e->p[2] < 0.0) return 0;
            break;
        case ORA_SERSIC:
        case ORA_DEVAUC:
            r = e->p[2];
            F = pow(10.0, -0.4 * (e->p[3] - sys->zeropoint));
            if (cp->type == ORA_SERSIC) { n = e->p[4]; q = e->p[5]; pa = e->p[6]; }
            else { n = 4.0; q = e->p[4]; pa = e->p[5]; }
            if (!(r > 0.0) || !(n > 0.0) || !(q > 0.0 && q <= 1.0)) return 0;
            e->bn = ora_sersic_bn(n);
            e->inv_n = 1.0 / n;
            e->I0 = F * pow(e->bn, 2.0 * n) / (2.0 * ORA_PI * n * r * r * tgamma(2.0 * n));
            e->cos_pa = cos(deg2rad(pa));
            e->sin_pa = sin(deg2rad(pa));
            break;
        case ORA_GAUSS:
            r = e->p[2];
            q = e->p[4];
            if (!(r > 0.0) || !(q > 0.0 && q <= 1.0)) return 0;
            F = pow(10.0, -0.4 * (e->p[3] - sys->zeropoint));
            e->I0 = F / (2.0 * ORA_PI * r * r);
            e->cos_pa = cos(deg2rad(e->p[5]));
            e->sin_pa = sin(deg2rad(e->p[5]));
            break;
        case ORA_SKY:
            break;
        default:
            return 0;
        }
    }
    /* image-plane priors (Sec. 5): a source whose position parameters are an
     * image-plane position theta sits at the source-plane position
     * theta - alpha(theta) of the same lens (Eq. 1) */
    for (int c = 0; c < sys->ncomp; ++c) {
        if (ce[c].plane != ORA_PLANE_SOURCE_IMAGE) continue;
        double tx = ce[c].p[0], ty = ce[c].p[1], ax = 0.0, ay = 0.0;
        for (int l = 0; l < sys->ncomp; ++l) {
            if (ce[l].plane != ORA_PLANE_LENS) continue;
            double dax, day;
            ora_deflection_one(ce[l].type, ce[l].p, tx, ty, &dax, &day);
            ax += dax;
            ay += day;
        }
        ce[c].p[0] = tx - ax;
        ce[c].p[1] = ty - ay;
        ce[c].plane = ORA_PLANE_SOURCE;
    }
    return 1;
}

/* Deflection of one mass component at (x, y) (Eq. 1's alpha). */
void ora_deflection_one(int type, const double *p, double x, double y,
                        double *ax, double *ay)
{
    *ax = 0.0;
    *ay = 0.0;
    if (type == ORA_SIE) {
        double x0 = p[0], y0 = p[1], b = p[2], q = p[3], s = p[5];
        double c = cos(deg2rad(p[4])), sn = sin(deg2rad(p[4]));
        double dx = x - x0, dy = y - y0;
        /* into the lens frame: major axis on +x */
        double u = dx * c + dy * sn;
        double v = -dx * sn + dy * c;
        double e = sqrt((1.0 - q) * (1.0 + q));
        double psi = sqrt(q * q * (s * s + u * u) + v * v);
        if (psi + s == 0.0) return; /* exact centre of a coreless SIE: alpha = 0 */
        double zu = u / (psi + s), zv = v / (psi + q * q * s);
        double au, av;
        if (e < 1e-3) {
            /* atan(e z)/e and atanh(e z)/e to O(e^4) */
            double e2 = e * e;
            au = b * sqrt(q) * zu * (1.0 - e2 * zu * zu / 3.0 + e2 * e2 * zu * zu * zu * zu / 5.0);
            av = b * sqrt(q) * zv * (1.0 + e2 * zv * zv / 3.0 + e2 * e2 * zv * zv * zv * zv / 5.0);
        } else {
            au = b * sqrt(q) / e * atan(e * zu);
            av = b * sqrt(q) / e * atanh(e * zv);
        }
        /* back to the sky frame */
        *ax = au * c - av * sn;
        *ay = au * sn + av * c;
    } else if (type == ORA_SHEAR) {
        double dx = x - p[0], dy = y - p[1];
        double g1 = p[2] * cos(2.0 * deg2rad(p[3]));
        double g2 = p[2] * sin(2.0 * deg2rad(p[3]));
        *ax = g1 * dx + g2 * dy;
        *ay = g2 * dx - g1 * dy;
    } else if (type == ORA_POINTMASS) {
        double dx = x - p[0], dy = y - p[1];
        double r2 = dx * dx + dy * dy;
        if (r2 > 0.0) {
            *ax = p[2] * p[2] * dx / r2;
            *ay = p[2] * p[2] * dy / r2;
        }
    }
}

/* Surface brightness of one light component at (x, y) (Eqs. 22-23). */
static double brightness_one(const ora_comp_eval *e, double x, double y)
{
    if (e->type == ORA_SKY) return e->p[0]; /* flat sky (Sec. 5) */
    double dx = x - e->p[0], dy = y - e->p[1];
    double u = dx * e->cos_pa + dy * e->sin_pa;
    double v = -dx * e->sin_pa + dy * e->cos_pa;
    if (e->type == ORA_GAUSS) {
        double q = e->p[4], sig = e->p[2];
        double R2 = u * u * q + v * v / q;
        return e->I0 * exp(-R2 / (2.0 * sig * sig));
    }
    double q = (e->type == ORA_SERSIC) ? e->p[5] : e->p[4];
    double R = sqrt(u * u * q + v * v / q);
    return e->I0 * exp(-e->bn * pow(R / e->p[2], e->inv_n));
}

/* Eq. 2 with Eq. 1: total image-plane brightness at image position (x, y). */
static double image_brightness(const ora_system *sys, const ora_comp_eval *ce,
                               double x, double y)
{
    double I = 0.0, ax = 0.0, ay = 0.0;
    for (int c = 0; c < sys->ncomp; ++c)
        if (ce[c].plane == ORA_PLANE_FOREGROUND) I += brightness_one(&ce[c], x, y);
    for (int c = 0; c < sys->ncomp; ++c) {
        if (ce[c].plane != ORA_PLANE_LENS) continue;
        double dax, day;
        ora_deflection_one(ce[c].type, ce[c].p, x, y, &dax, &day);
        ax += dax;
        ay += day;
    }
    double yx = x - ax, yy = y - ay;
    for (int c = 0; c < sys->ncomp; ++c)
        if (ce[c].plane == ORA_PLANE_SOURCE) I += brightness_one(&ce[c], yx, yy);
    return I;
}

/* Eqs. 3 and 14: L_ij = sum_ab W_a W_b h^2 I(x_c + t_a h, y_c + t_b h). */
static void pixel_luminosities(const ora_system *sys, const ora_comp_eval *ce,
                               const double *t, const double *wt, int nn, double *L)
{
    double h = sys->h;
    for (int i = 0; i < sys->ny; ++i) {
        double yc = (i - 0.5 * (sys->ny - 1)) * h;
        for (int j = 0; j < sys->nx; ++j) {
            double xc = (j - 0.5 * (sys->nx - 1)) * h;
            double sum = 0.0;
            for (int b = 0; b < nn; ++b)
                for (int a = 0; a < nn; ++a)
                    sum += wt[a] * wt[b] * h * h *
                           image_brightness(sys, ce, xc + t[a] * h, yc + t[b] * h);
            L[i * sys->nx + j] = sum;
        }
    }
}

static int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

/* Eq. 15 with the PSF normalised to unit sum and clamp padding. */
static void psf_convolve(const ora_system *sys, const double *L, double *Ls)
{
    int nx = sys->nx, ny = sys->ny;
    if (!sys->psf) {
        memcpy(Ls, L, sizeof(double) * nx * ny);
        return;
    }
    int p = sys->psf_ny / 2, q = sys->psf_nx / 2;
    double norm = 0.0;
    for (int k = 0; k < sys->psf_nx * sys->psf_ny; ++k) norm += sys->psf[k];
    for (int i = 0; i < ny; ++i)
        for (int j = 0; j < nx; ++j) {
            double s = 0.0;
            for (int k = -p; k <= p; ++k)
                for (int l = -q; l <= q; ++l) {
                    /* F_{-k,-l}: array element (p - k, q - l) */
                    double F = sys->psf[(p - k) * sys->psf_nx + (q - l)] / norm;
                    s += F * L[clampi(i + k, 0, ny - 1) * nx + clampi(j + l, 0, nx - 1)];
                }
            Ls[i * nx + j] = s;
        }
}

/* Per-pixel integration error estimate of a Gauss-Kronrod system (Sec. 3.1,
 * the embedded-Gauss estimate): |L_K - L_G| with L_K the (2N+1)^2-point
 * Kronrod luminosity and L_G the N^2-point Gauss luminosity of the same
 * pixel, both unconvolved.  Returns 0, 1 outside the domain, -1 if the
 * system's rule is not Gauss-Kronrod. */
int ora_render_error(const ora_system *sys, const double *xi, double *err)
{
    ora_comp_eval ce[64];
    double tk[64], wk[64], tg[64], wg[64];
    if (sys->rule != ORA_RULE_GK || sys->ncomp > 64) return -1;
    int nk = ora_rule_nodes(ORA_RULE_GK, sys->order, tk, wk);
    int ng = ora_rule_nodes(ORA_RULE_GL, sys->order, tg, wg);
    if (nk < 1 || ng < 1) return -1;
    if (!resolve(sys, xi, ce)) return 1;
    int n = sys->nx * sys->ny;
    double *LK = (double *)malloc(sizeof(double) * n);
    double *LG = (double *)malloc(sizeof(double) * n);
    pixel_luminosities(sys, ce, tk, wk, nk, LK);
    pixel_luminosities(sys, ce, tg, wg, ng, LG);
    for (int i = 0; i < n; ++i) err[i] = fabs(LK[i] - LG[i]);
    free(LK);
    free(LG);
    return 0;
}

/* Weights w_i = extra_i / s_i^2 (Sec. 3.2, Sec. 3.3), zero where masked. */
int ora_weights(const ora_system *sys, double *w)
{
    int n = sys->nx * sys->ny;
    for (int i = 0; i < n; ++i) {
        if (sys->mask && sys->mask[i]) { w[i] = 0.0; continue; }
        double s2 = sys->variance ? sys->variance[i]
                                  : (sys->data[i] + sys->offset) / sys->gain;
        if (!(s2 > 0.0) || !isfinite(s2)) return -1;
        w[i] = (sys->extra_weight ? sys->extra_weight[i] : 1.0) / s2;
    }
    return 0;
}

/* Render L (convolved == 0) or L* (convolved != 0); returns 0 on success,
 * 1 if the point is outside the parameter domain (image left untouched). */
int ora_render(const ora_system *sys, const double *xi, int convolved, double *out)
{
    ora_comp_eval ce[64];
    double t[256], wt[256];
    if (sys->ncomp > 64) return -1;
    int nn = ora_rule_nodes(sys->rule, sys->order, t, wt);
    if (nn < 1) return -1;
    if (!resolve(sys, xi, ce)) return 1;
    int n = sys->nx * sys->ny;
    double *L = (double *)malloc(sizeof(double) * n);
    pixel_luminosities(sys, ce, t, wt, nn, L);
    if (convolved) psf_convolve(sys, L, out);
    else memcpy(out, L, sizeof(double) * n);
    free(L);
    return 0;
}

/* Eq. 17 summed with Neumaier compensation. */
static double loglike_from(const ora_system *sys, const double *Ls, const double *w)
{
    int n = sys->nx * sys->ny;
    double s = 0.0, c = 0.0;
    for (int i = 0; i < n; ++i) {
        if (w[i] == 0.0) continue;
        double r = sys->data[i] - Ls[i];
        double v = w[i] * r * r;
        double tsum = s + v;
        if (fabs(s) >= fabs(v)) c += (s - tsum) + v;
        else c += (v - tsum) + s;
        s = tsum;
    }
    return -0.5 * (s + c);
}

/* loglike for P parameter points xi[P][nparam]; -inf outside the domain. */
int ora_loglike_batch(const ora_system *sys, const double *xi, int P, double *out,
                      int nthreads)
{
    int n = sys->nx * sys->ny;
    double *w = (double *)malloc(sizeof(double) * n);
    if (ora_weights(sys, w) != 0) { free(w); return -1; }
    int bad = 0;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads > 0 ? nthreads : 1)
#endif
    for (int k = 0; k < P; ++k) {
        double *L = (double *)malloc(sizeof(double) * n);
        int rc = ora_render(sys, xi + (size_t)k * sys->nparam, 1, L);
        if (rc == 0) out[k] = loglike_from(sys, L, w);
        else if (rc == 1) out[k] = -INFINITY;
        else bad = 1;
        free(L);
    }
    (void)nthreads;
    free(w);
    return bad ? -1 : 0;
}

/* Sersic b_n, I_0 exposed for the tests. */
double ora_sersic_I0(double n, double r, double F)
{
    double bn = ora_sersic_bn(n);
    return F * pow(bn, 2.0 * n) / (2.0 * ORA_PI * n * r * r * tgamma(2.0 * n));
}

/* Convergence of the SIE with core (the reading stated above), for the
 * divergence and enclosed-mass checks in the tests. */
double ora_sie_kappa(const double *p, double x, double y)
{
    double q = p[3], s = p[5];
    double c = cos(deg2rad(p[4])), sn = sin(deg2rad(p[4]));
    double dx = x - p[0], dy = y - p[1];
    double u = dx * c + dy * sn, v = -dx * sn + dy * c;
    double psi = sqrt(q * q * (s * s + u * u) + v * v);
    return p[2] * sqrt(q) / (2.0 * psi);
}

/* Stand-alone PSF convolution and weights for the tests. */
void ora_psf_convolve(const ora_system *sys, const double *L, double *Ls)
{
    psf_convolve(sys, L, Ls);
}

double ora_loglike_image(const ora_system *sys, const double *Ls)
{
    int n = sys->nx * sys->ny;
    double *w = (double *)malloc(sizeof(double) * n);
    if (ora_weights(sys, w) != 0) { free(w); return NAN; }
    double v = loglike_from(sys, Ls, w);
    free(w);
    return v;
}
