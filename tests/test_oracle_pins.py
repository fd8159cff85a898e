"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: a library
routine (numpy/scipy), a closed form of lensing or of the Sersic law, an
invariant (divergence theorem, surface-brightness conservation), or brute
force on tiny inputs.  Together they are chosen so that a dropped term, a
wrong sign or index, or a transposed operand anywhere in the oracle fails at
least one of them.
"""
import math

import numpy as np
import pytest
import scipy.integrate as si
import scipy.signal as ss
import scipy.special as sp

from oracle import oracle as O
import workloads as W
from workloads import component, fixed, free


def make_spec(comps, nx=32, ny=32, h=0.05, rule=("gl", 3), psf=None, mask=None, n_params=0,
              zeropoint=0.0):
    return {"name": "t", "nx": nx, "ny": ny, "h": h, "rule": rule, "psf": psf, "mask": mask,
            "zeropoint": zeropoint, "components": comps, "n_params": n_params}


def pixel_centres(nx, ny, h):
    x = (np.arange(nx) - 0.5 * (nx - 1)) * h
    y = (np.arange(ny) - 0.5 * (ny - 1)) * h
    return np.meshgrid(x, y)


# --------------------------------------------------------------------------
# Quadrature rules (Sec. 3.1, Eq. 14; Sec. 4.5 rule list)

@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 7, 11, 15, 32, 64, 128])
def test_gauss_legendre_matches_numpy(n):
    x, w = O.gauss_legendre(n)
    X, Wt = np.polynomial.legendre.leggauss(n)
    assert np.allclose(x, X, rtol=0, atol=1e-14)
    assert np.allclose(w, Wt, rtol=0, atol=1e-13)


@pytest.mark.parametrize("n", [1, 2, 3, 5, 7])
def test_rule_exact_on_polynomials(n):
    # The N-point rule on the unit pixel integrates t^k exactly for k <= 2N-1.
    t, w = O.rule_nodes("gl", n)
    assert abs(w.sum() - 1.0) < 1e-15
    for k in range(2 * n):
        exact = 0.0 if k % 2 else 2 * 0.5 ** (k + 1) / (k + 1)
        assert abs((w * t ** k).sum() - exact) < 1e-15
    # and not for k = 2N
    k = 2 * n
    exact = 2 * 0.5 ** (k + 1) / (k + 1)
    assert abs((w * t ** k).sum() - exact) > 1e-12


def test_sub_and_point_rules():
    t, w = O.rule_nodes("point", 1)
    assert t.tolist() == [0.0] and w.tolist() == [1.0]
    t, w = O.rule_nodes("sub", 2)
    assert np.allclose(t, [-0.25, 0.25]) and np.allclose(w, [0.5, 0.5])
    t, w = O.rule_nodes("sub", 4)
    assert np.allclose(t, [-0.375, -0.125, 0.125, 0.375]) and np.allclose(w, 0.25)


# Gauss-Kronrod rules g3k7 / g5k11 / g7k15 (Sec. 3.1 default rule, Sec. 4.5)

# 15-point Kronrod extension of the 7-point Gauss rule as tabulated in
# QUADPACK (Piessens et al. 1983), the non-negative half: nodes, Kronrod
# weights, Gauss weights on the shared nodes.
G7K15_X = [0.991455371120812639, 0.949107912342758525, 0.864864423359769073,
           0.741531185599394440, 0.586087235467691130, 0.405845151377397167,
           0.207784955007898468, 0.0]
G7K15_WK = [0.022935322010529225, 0.063092092629978553, 0.104790010322250184,
            0.140653259715525919, 0.169004726639267903, 0.190350578064785410,
            0.204432940075298892, 0.209482141084727828]
G7K15_WG = [0.129484966168869693, 0.279705391489276668, 0.381830050505118945,
            0.417959183673469388]


def test_g7k15_matches_published_table():
    x, wk, wg = O.gauss_kronrod(7)
    assert np.allclose(x[7:][::-1], G7K15_X, rtol=0, atol=2e-15)
    assert np.allclose(x[:8], -np.array(G7K15_X), rtol=0, atol=2e-15)
    assert np.allclose(wk[7:][::-1], G7K15_WK, rtol=0, atol=2e-15)
    assert np.allclose(wg[7:][::-1][1::2], G7K15_WG, rtol=0, atol=2e-15)
    assert np.all(wg[7:][::-1][0::2] == 0.0)


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6, 7])
def test_kronrod_extension_properties(n):
    x, wk, wg = O.gauss_kronrod(n)
    # the embedded rule is the n-point Gauss-Legendre rule
    gx, gw = np.polynomial.legendre.leggauss(n)
    shared = wg != 0.0
    assert shared.sum() == n
    assert np.allclose(x[shared], gx, atol=1e-14) and np.allclose(wg[shared], gw, atol=1e-14)
    # added nodes interlace with the Gauss nodes (one on each side and one
    # between every pair), all weights positive
    assert np.all(np.diff(x) > 0) and np.all(wk > 0)
    assert shared[1::2].all() and not shared[0::2].any()
    # exact on x^k up to degree 3n+1 (3n+2 for odd n by symmetry) and not beyond
    deg = 3 * n + 1 + (n % 2)
    for k in range(deg + 1):
        exact = 0.0 if k % 2 else 2.0 / (k + 1)
        assert abs((wk * x ** k).sum() - exact) < 1e-14, k
    k = deg + 1 if (deg + 1) % 2 == 0 else deg + 2
    assert abs((wk * x ** k).sum() - 2.0 / (k + 1)) > 1e-10


def test_kronrod_smallest_case_is_three_point_gauss():
    # the Kronrod extension of the 1-point rule is the 3-point Gauss rule
    x, wk, _ = O.gauss_kronrod(1)
    assert np.allclose(x, [-math.sqrt(0.6), 0.0, math.sqrt(0.6)], atol=1e-15)
    assert np.allclose(wk, [5 / 9, 8 / 9, 5 / 9], atol=1e-15)
    t, w = O.rule_nodes("gk", 3)
    assert len(t) == 7 and abs(w.sum() - 1.0) < 1e-15 and np.all(np.abs(t) < 0.5)


def test_kronrod_error_estimate_tracks_gauss_error():
    # The per-pixel error estimate |L_K - L_G| measures the error of the
    # embedded Gauss rule: against a 64 x 64 Gauss-Legendre integral of a
    # lensed arc, |L_ref - L_G| agrees with it to a few per cent wherever
    # the error is not negligible, and the Kronrod luminosity itself is much
    # closer to the reference than the Gauss one.
    comps = [component("sie", "lens", [fixed(0.02), fixed(0.0), fixed(0.2), fixed(0.7), fixed(30),
                                       fixed(0.0)]),
             component("sersic", "source", [fixed(0.01), fixed(0.005), fixed(0.03), fixed(0),
                                            fixed(0.5), fixed(0.8), fixed(0)])]
    for n in (3, 5):
        spec = make_spec(comps, nx=16, ny=16, h=0.04, rule=("gk", n))
        err = O.OracleSystem(spec).render_error(np.zeros(0))
        LK = O.OracleSystem(spec).render(np.zeros(0), convolved=False)
        LG = O.OracleSystem(make_spec(comps, nx=16, ny=16, h=0.04, rule=("gl", n))).render(
            np.zeros(0), convolved=False)
        ref = O.OracleSystem(make_spec(comps, nx=16, ny=16, h=0.04, rule=("gl", 64))).render(
            np.zeros(0), convolved=False)
        assert np.array_equal(err, np.abs(LK - LG))
        true_g = np.abs(ref - LG)
        big = true_g > 1e-3 * true_g.max()
        assert big.sum() > 10
        assert np.allclose(err[big], true_g[big], rtol=0.05), np.abs(err[big] / true_g[big] - 1).max()
        assert np.abs(LK - ref).max() < 0.05 * true_g.max()


# --------------------------------------------------------------------------
# Sersic law (Sec. 4.1, Eqs. 22-23)

@pytest.mark.parametrize("a,x", [(1.0, 0.5), (2.0, 1.7), (8.0, 7.7), (16.0, 15.6), (0.2, 0.1),
                                 (3.3, 0.01), (1.0, 1.0)])
def test_incomplete_gamma_matches_scipy(a, x):
    assert abs(O.gammainc_lower(a, x) - sp.gammainc(a, x)) < 1e-14


@pytest.mark.parametrize("n", [0.3, 0.5, 1.0, 1.5, 2.0, 3.7, 4.0, 6.0, 8.0])
def test_sersic_bn_matches_scipy(n):
    assert abs(O.sersic_bn(n) - sp.gammaincinv(2 * n, 0.5)) < 1e-12 * max(1, n)


def test_sersic_bn_literature_values():
    # b_1 and b_4 (de Vaucouleurs) as tabulated in the literature
    assert abs(O.sersic_bn(1.0) - 1.678346990) < 1e-8
    assert abs(O.sersic_bn(4.0) - 7.669249443) < 1e-8
    # n = 1/2 is the Gaussian: P(1, b) = 1 - e^-b = 1/2
    assert abs(O.sersic_bn(0.5) - math.log(2.0)) < 1e-14


def test_sersic_half_light_radius():
    # The flux inside R = r_e is half the total (Sec. 4.1 defines r_S so).
    for n in (0.7, 1.0, 2.5, 4.0):
        r, F = 0.3, 2.0
        I0, bn = O.sersic_I0(n, r, F), O.sersic_bn(n)
        f = lambda R: 2 * math.pi * R * I0 * math.exp(-bn * (R / r) ** (1 / n))
        inner = si.quad(f, 0, r, epsabs=0, epsrel=1e-13, limit=200)[0]
        total = si.quad(f, 0, np.inf, epsabs=0, epsrel=1e-13, limit=200)[0]
        assert abs(total - F) < 1e-9 * F
        assert abs(inner - 0.5 * F) < 1e-9 * F


@pytest.mark.parametrize("n,q,pa,tol", [(0.5, 0.6, 30.0, 1e-10), (1.0, 0.4, 120.0, 5e-6),
                                        (1.0, 1.0, 0.0, 5e-6)])
def test_sersic_total_flux_unlensed(n, q, pa, tol):
    # Unlensed Sersic over a field wide enough that the tail is negligible
    # (n = 1 has a cusp at its centre, which bounds the rule to ~1e-6):
    # sum of pixel luminosities = F = 10^(-0.4 (mag - zp)).
    mag, zp = 1.3, 2.0
    F = 10 ** (-0.4 * (mag - zp))
    spec = make_spec([component("sersic", "foreground",
                                [fixed(0.07), fixed(-0.04), fixed(0.3), fixed(mag), fixed(n),
                                 fixed(q), fixed(pa)])],
                     nx=200, ny=200, h=0.05, rule=("gl", 6), zeropoint=zp)
    L = O.OracleSystem(spec).render(np.zeros(0), convolved=False)
    assert abs(L.sum() - F) < tol * F


def test_sersic_n4_flux_within_tail_bounds():
    # n = 4: the tail beyond the field is not negligible; for a round profile
    # the square field's flux lies between the closed-form fluxes inside the
    # inscribed and the circumscribed circle.
    n, r, F = 4.0, 0.1, 1.0
    spec = make_spec([component("devauc", "foreground",
                                [fixed(0.0), fixed(0.0), fixed(r), fixed(0.0), fixed(1.0),
                                 fixed(0.0)])],
                     nx=100, ny=100, h=0.04, rule=("gl", 8))
    L = O.OracleSystem(spec).render(np.zeros(0), convolved=False)
    bn = sp.gammaincinv(8.0, 0.5)
    half = 50 * 0.04
    inner = F * sp.gammainc(8.0, bn * (half / r) ** 0.25)
    outer = F * sp.gammainc(8.0, bn * (half * math.sqrt(2) / r) ** 0.25)
    assert inner - 1e-4 < L.sum() < outer + 1e-4


def test_gaussian_total_flux():
    F = 3.0
    spec = make_spec([component("gauss", "foreground",
                                [fixed(0.1), fixed(0.0), fixed(0.25), fixed(-2.5 * math.log10(F)),
                                 fixed(0.5), fixed(10.0)])],
                     nx=160, ny=160, h=0.05, rule=("gl", 4))
    L = O.OracleSystem(spec).render(np.zeros(0), convolved=False)
    assert abs(L.sum() - F) < 1e-9 * F


@pytest.mark.parametrize("ctype", ["sersic", "gauss"])
def test_position_angle_convention(ctype):
    # PA is counter-clockwise from +x to the major axis (Sec. 4): at PA=90
    # the light extends along +y, at PA=0 along +x, at PA=45 along x=y.
    def I_at(pa, x, y):
        if ctype == "sersic":
            p = [fixed(0), fixed(0), fixed(0.3), fixed(0), fixed(1.0), fixed(0.4), fixed(pa)]
        else:
            p = [fixed(0), fixed(0), fixed(0.3), fixed(0), fixed(0.4), fixed(pa)]
        spec = make_spec([component(ctype, "foreground", p)], nx=1, ny=1, h=1e-3,
                         rule=("point", 1))
        # shift the profile instead of the pixel: the single pixel sits at 0
        spec["components"][0]["params"][0] = fixed(-x)
        spec["components"][0]["params"][1] = fixed(-y)
        return O.OracleSystem(spec).render(np.zeros(0), convolved=False)[0, 0]

    assert I_at(90, 0, 0.3) > 2 * I_at(90, 0.3, 0)
    assert I_at(0, 0.3, 0) > 2 * I_at(0, 0, 0.3)
    d = 0.3 / math.sqrt(2)
    assert I_at(45, d, d) > 2 * I_at(45, d, -d)
    assert I_at(135, -d, d) > 2 * I_at(135, d, d)


def test_pixel_coordinate_convention():
    # column j runs along +x, row i along +y, centre of the image at 0
    def peak(x, y):
        spec = make_spec([component("gauss", "foreground",
                                    [fixed(x), fixed(y), fixed(0.05), fixed(0), fixed(1),
                                     fixed(0)])], nx=21, ny=21, h=0.05, rule=("gl", 2))
        L = O.OracleSystem(spec).render(np.zeros(0), convolved=False)
        return np.unravel_index(np.argmax(L), L.shape)

    assert peak(0.0, 0.0) == (10, 10)
    assert peak(0.25, 0.0) == (10, 15)
    assert peak(0.0, 0.25) == (15, 10)
    assert peak(-0.1, -0.2) == (6, 8)


# --------------------------------------------------------------------------
# Deflection fields (Sec. 2.1, Eq. 1)

def kappa_def(b, q, pa, s, x, y):
    """Convergence of an isothermal ellipsoid with core, major axis at PA
    (the definition the deflection must satisfy via div alpha = 2 kappa)."""
    c, sn = math.cos(math.radians(pa)), math.sin(math.radians(pa))
    u = x * c + y * sn
    v = -x * sn + y * c
    return b / (2 * math.sqrt(q * (s * s + u * u) + v * v / q))


@pytest.mark.parametrize("q,s,pa", [(0.3, 0.0, 17.0), (0.75, 0.0, 45.0), (0.75, 0.05, 45.0),
                                    (0.95, 0.02, 120.0), (0.9999, 0.0, 200.0), (1.0, 0.1, 0.0)])
def test_sie_divergence_and_curl(q, s, pa):
    rng = np.random.default_rng(7)
    b, x0, y0, eps = 1.2, 0.11, -0.07, 1e-5
    p = [x0, y0, b, q, pa, s]
    for _ in range(20):
        x, y = rng.uniform(-2, 2, 2)
        if math.hypot(x - x0, y - y0) < 0.1:
            continue
        axp, ayp = O.deflection("sie", p, x + eps, y)
        axm, aym = O.deflection("sie", p, x - eps, y)
        bxp, byp = O.deflection("sie", p, x, y + eps)
        bxm, bym = O.deflection("sie", p, x, y - eps)
        div = (axp - axm + byp - bym) / (2 * eps)
        curl = (ayp - aym - (bxp - bxm)) / (2 * eps)
        k = kappa_def(b, q, pa, s, x - x0, y - y0)
        assert abs(div - 2 * k) < 2e-6 * max(1, k)
        assert abs(curl) < 2e-6


@pytest.mark.parametrize("q,pa", [(0.4, 0.0), (0.75, 45.0), (0.93, 100.0)])
def test_sie_mean_convergence_inside_einstein_radius(q, pa):
    # s = 0: the ellipse of geometric-mean radius R = b (area pi b^2) holds
    # mean convergence 1, i.e. (1/2) * flux of alpha through it = pi b^2.
    b = 1.3624
    c, sn = math.cos(math.radians(pa)), math.sin(math.radians(pa))
    p = [0.0, 0.0, b, q, pa, 0.0]
    t = np.linspace(0, 2 * math.pi, 4001)[:-1]
    dt = t[1] - t[0]
    flux = 0.0
    for tt in t:
        u, v = b / math.sqrt(q) * math.cos(tt), b * math.sqrt(q) * math.sin(tt)
        # outward normal times dl in the lens frame: (dv/dt, -du/dt) dt
        nu, nv = b * math.sqrt(q) * math.cos(tt), b / math.sqrt(q) * math.sin(tt)
        x, y = u * c - v * sn, u * sn + v * c
        nx_, ny_ = nu * c - nv * sn, nu * sn + nv * c
        ax, ay = O.deflection("sie", p, x, y)
        flux += (ax * nx_ + ay * ny_) * dt
    mean_kappa = 0.5 * flux / (math.pi * b * b)
    assert abs(mean_kappa - 1.0) < 1e-10


def test_sis_einstein_ring():
    # q = 1, s = 0: |alpha| = b everywhere, radial; |x| = b maps to y = 0.
    b = 1.1
    for ang in np.linspace(0, 2 * math.pi, 13):
        for r in (0.3, b, 2.7):
            x, y = r * math.cos(ang), r * math.sin(ang)
            ax, ay = O.deflection("sie", [0, 0, b, 1.0, 33.0, 0.0], x, y)
            assert abs(math.hypot(ax, ay) - b) < 1e-14
            assert abs(ax * y - ay * x) < 1e-14
            if r == b:
                assert math.hypot(x - ax, y - ay) < 1e-14


def test_sie_round_limit_against_high_precision():
    # Near q = 1 the oracle switches from the closed form to the series in
    # e; both sides of the switch agree with the closed form evaluated in
    # 50-digit arithmetic, and q = 1 is the softened SIS alpha = b x/(psi+s).
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 50
    b, pa, s = 1.0, 20.0, 0.03
    c, sn = mpmath.cos(mpmath.radians(pa)), mpmath.sin(mpmath.radians(pa))
    for x, y in [(0.7, 0.2), (-0.1, 1.3), (0.5, -0.5)]:
        u = x * c + y * sn
        v = -x * sn + y * c
        for q in (1 - 4.9e-7, 1 - 5.1e-7, 1 - 1e-5, 0.999, 1.0):
            qm = mpmath.mpf(q)
            e = mpmath.sqrt((1 - qm) * (1 + qm))
            psi = mpmath.sqrt(qm * qm * (s * s + u * u) + v * v)
            if e == 0:
                au, av = b * u / (psi + s), b * v / (psi + s)
            else:
                au = b * mpmath.sqrt(qm) / e * mpmath.atan(e * u / (psi + s))
                av = b * mpmath.sqrt(qm) / e * mpmath.atanh(e * v / (psi + qm * qm * s))
            want = (float(au * c - av * sn), float(au * sn + av * c))
            got = O.deflection("sie", [0, 0, b, q, pa, s], x, y)
            assert abs(got[0] - want[0]) < 1e-14 and abs(got[1] - want[1]) < 1e-14, (q, got, want)


def test_sie_rotation_equivariance():
    p = [0.0, 0.0, 1.0, 0.6, 10.0, 0.02]
    th = math.radians(35.0)
    R = np.array([[math.cos(th), -math.sin(th)], [math.sin(th), math.cos(th)]])
    for x, y in [(0.5, 0.3), (-1.2, 0.4)]:
        a = np.array(O.deflection("sie", p, x, y))
        xr = R @ np.array([x, y])
        ar = np.array(O.deflection("sie", [0, 0, 1.0, 0.6, 45.0, 0.02], *xr))
        assert np.allclose(ar, R @ a, atol=1e-14)


def test_singular_centres_have_no_deflection():
    # reading: alpha = 0 exactly at a point mass and at the centre of a
    # coreless SIE (the direction is undefined there); a core removes the
    # singularity and alpha -> 0 continuously
    assert O.deflection("sie", [0.1, -0.2, 1.0, 0.7, 30.0, 0.0], 0.1, -0.2) == (0.0, 0.0)
    ax, ay = O.deflection("sie", [0.1, -0.2, 1.0, 0.7, 30.0, 0.05], 0.1 + 1e-9, -0.2)
    assert math.hypot(ax, ay) < 1e-7


def test_point_mass_closed_form():
    te = 0.3
    for x, y in [(0.1, 0.2), (-0.4, 0.05), (0.3, 0.0)]:
        ax, ay = O.deflection("pointmass", [0.05, -0.02, te], x, y)
        dx, dy = x - 0.05, y + 0.02
        r = math.hypot(dx, dy)
        assert abs(math.hypot(ax, ay) - te * te / r) < 1e-15
        assert abs(ax * dy - ay * dx) < 1e-15 and ax * dx > 0
    # ring at theta_E
    for ang in np.linspace(0, 2 * math.pi, 7):
        x, y = te * math.cos(ang), te * math.sin(ang)
        ax, ay = O.deflection("pointmass", [0, 0, te], x, y)
        assert math.hypot(x - ax, y - ay) < 1e-15
    # reading: no deflection exactly on the mass
    assert O.deflection("pointmass", [0.1, 0.1, te], 0.1, 0.1) == (0.0, 0.0)


def test_shear_jacobian():
    g, phi = 0.07, 25.0
    g1, g2 = g * math.cos(math.radians(2 * phi)), g * math.sin(math.radians(2 * phi))
    a0 = np.array(O.deflection("shear", [0.1, 0.2, g, phi], 0.1, 0.2))
    assert np.abs(a0).max() == 0.0
    ax, ay = O.deflection("shear", [0.1, 0.2, g, phi], 0.1 + 1.0, 0.2)
    assert abs(ax - g1) < 1e-15 and abs(ay - g2) < 1e-15
    ax, ay = O.deflection("shear", [0.1, 0.2, g, phi], 0.1, 0.2 + 1.0)
    assert abs(ax - g2) < 1e-15 and abs(ay + g1) < 1e-15


# --------------------------------------------------------------------------
# Full forward model (Eqs. 1-3, 14)

def test_shear_only_magnification():
    # kappa = 0, |gamma| = g: every source is magnified by 1 / (1 - g^2).
    g = 0.1
    F = 1.0
    spec = make_spec([component("shear", "lens", [fixed(0), fixed(0), fixed(g), fixed(20.0)]),
                      component("gauss", "source", [fixed(0.05), fixed(-0.03), fixed(0.12),
                                                    fixed(0.0), fixed(0.7), fixed(50.0)])],
                     nx=120, ny=120, h=0.05, rule=("gl", 4))
    L = O.OracleSystem(spec).render(np.zeros(0), convolved=False)
    assert abs(L.sum() - F / (1 - g * g)) < 1e-9


def test_surface_brightness_conservation():
    # A uniform source keeps its surface brightness through any lens: every
    # pixel gets I h^2 (here the source is a Gaussian so wide that it is flat
    # to 1e-9 over the field).
    sig = 3e4
    F = 2 * math.pi * sig * sig * 1e-3  # I0 = 1e-3 per arcsec^2
    spec = make_spec([
        component("sie", "lens", [fixed(0.1), fixed(0), fixed(1.2), fixed(0.6), fixed(30), fixed(0.0)]),
        component("shear", "lens", [fixed(0), fixed(0), fixed(0.08), fixed(70.0)]),
        component("pointmass", "lens", [fixed(-0.3), fixed(0.4), fixed(0.2)]),
        component("gauss", "source", [fixed(0), fixed(0), fixed(sig), fixed(-2.5 * math.log10(F)),
                                      fixed(1.0), fixed(0)])],
        nx=24, ny=24, h=0.1, rule=("gl", 3))
    L = O.OracleSystem(spec).render(np.zeros(0), convolved=False)
    assert np.abs(L / (1e-3 * 0.01) - 1).max() < 1e-8


@pytest.mark.parametrize("plane", ["foreground", "source"])
@pytest.mark.parametrize("rule", [("point", 1), ("sub", 4), ("gk", 3)])
def test_flat_sky(plane, rule):
    # Sec. 5's flat sky: a constant surface brightness S gives S h^2 in every
    # pixel whatever the rule (weights sum to one), the lens (surface
    # brightness is conserved) and the unit-sum PSF; it adds linearly to the
    # other components, and it may be negative.
    lens = [component("sie", "lens", [fixed(0.1), fixed(0), fixed(1.2), fixed(0.6), fixed(30),
                                      fixed(0.0)]),
            component("pointmass", "lens", [fixed(-0.3), fixed(0.4), fixed(0.2)])]
    src = component("sersic", "source", [fixed(0.05), fixed(0.02), fixed(0.2), fixed(0), fixed(1.5),
                                         fixed(0.7), fixed(20)])
    psf = W.gaussian_psf(5, 0.15, 0.1)
    for S in (0.37, -0.05):
        sky = component("sky", plane, [fixed(S)])
        L = O.OracleSystem(make_spec(lens + [sky], nx=20, ny=16, h=0.1, rule=rule, psf=psf)).render(
            np.zeros(0), convolved=True)
        assert np.abs(L - S * 0.01).max() <= 1e-14 * abs(S)
        a = O.OracleSystem(make_spec(lens + [src], nx=20, ny=16, h=0.1, rule=rule)).render(
            np.zeros(0), convolved=False)
        b = O.OracleSystem(make_spec(lens + [src, sky], nx=20, ny=16, h=0.1, rule=rule)).render(
            np.zeros(0), convolved=False)
        assert np.allclose(b - a, S * 0.01, rtol=0, atol=1e-14)


def test_image_plane_prior_places_source_behind_theta():
    # Sec. 5's image-plane prior: the source position parameters are an
    # image-plane position theta, and the source sits at y(theta).  With the
    # point rule a pixel whose centre is theta therefore sees the source's
    # central surface brightness I_0 exactly, for any lens.
    h = 0.05
    theta = (3 * h, -7 * h)   # a pixel centre of the 24 x 24 grid (offset by h/2)
    tx, ty = theta[0] + h / 2, theta[1] + h / 2
    lens = [component("sie", "lens", [fixed(0.03), fixed(-0.02), fixed(0.6), fixed(0.7), fixed(40),
                                      fixed(0.0)]),
            component("shear", "lens", [fixed(0), fixed(0), fixed(0.07), fixed(15.0)]),
            component("pointmass", "lens", [fixed(-0.25), fixed(0.1), fixed(0.1)])]
    mag, r, n = 1.0, 0.08, 1.3
    src = component("sersic", "source_image", [fixed(tx), fixed(ty), fixed(r), fixed(mag),
                                               fixed(n), fixed(0.6), fixed(30)])
    L = O.OracleSystem(make_spec(lens + [src], nx=24, ny=24, h=h, rule=("point", 1))).render(
        np.zeros(0), convolved=False)
    i = int(round(ty / h + 11.5))
    j = int(round(tx / h + 11.5))
    I0 = O.sersic_I0(n, r, 10 ** (-0.4 * mag))
    assert abs(L[i, j] / (h * h) - I0) < 1e-12 * I0
    assert L[i, j] == L.max()


def test_image_plane_prior_sis_closed_form():
    # For a singular isothermal sphere of Einstein radius b at the origin the
    # lens equation gives y = theta (1 - b/|theta|): an image-plane prior at
    # theta = (1.5, 0) is a source at (0.5, 0); and with no lens at all the
    # image-plane position is the source position.
    sis = component("sie", "lens", [fixed(0), fixed(0), fixed(1.0), fixed(1.0), fixed(0), fixed(0)])

    def img(plane, x, y, lens):
        src = component("sersic", plane, [fixed(x), fixed(y), fixed(0.1), fixed(0), fixed(1.0),
                                          fixed(0.8), fixed(10)])
        return O.OracleSystem(make_spec(lens + [src], nx=40, ny=40, h=0.1, rule=("gl", 3))).render(
            np.zeros(0), convolved=False)

    a = img("source_image", 1.5, 0.0, [sis])
    b = img("source", 0.5, 0.0, [sis])
    assert np.allclose(a, b, rtol=1e-12, atol=1e-15 * b.max())
    a = img("source_image", 0.3, -0.2, [])
    b = img("source", 0.3, -0.2, [])
    assert np.array_equal(a, b)


@pytest.mark.parametrize("lens", ["sis", "pointmass"])
def test_rendered_einstein_ring(lens):
    # A small source behind the lens centre is imaged into a ring of radius
    # theta_E; the flux-weighted mean radius of the image is theta_E.
    if lens == "sis":
        te = 1.0
        lc = component("sie", "lens", [fixed(0), fixed(0), fixed(te), fixed(1.0), fixed(0), fixed(0)])
    else:
        te = 0.8
        lc = component("pointmass", "lens", [fixed(0), fixed(0), fixed(te)])
    spec = make_spec([lc, component("gauss", "source", [fixed(0), fixed(0), fixed(0.01), fixed(0),
                                                        fixed(1), fixed(0)])],
                     nx=120, ny=120, h=0.025, rule=("gl", 5))
    L = O.OracleSystem(spec).render(np.zeros(0), convolved=False)
    xx, yy = pixel_centres(120, 120, 0.025)
    r = np.hypot(xx, yy)
    rmean = (L * r).sum() / L.sum()
    assert abs(rmean - te) < 2e-3
    # and nothing arrives far from the ring
    assert L[np.abs(r - te) > 0.2].sum() < 1e-6 * L.sum()


def test_quadrature_converges_brute_force():
    # 3x3 pixels around a lensed arc: the N x N Gauss-Legendre result
    # converges to the 64 x 64 brute-force integral as N grows.
    comps = [component("sie", "lens", [fixed(0.02), fixed(0.0), fixed(0.1), fixed(0.7), fixed(30),
                                       fixed(0.0)]),
             component("sersic", "source", [fixed(0.01), fixed(0.005), fixed(0.02), fixed(0),
                                            fixed(1.0), fixed(0.8), fixed(0)])]
    ref = O.OracleSystem(make_spec(comps, nx=3, ny=3, h=0.05, rule=("gl", 64))).render(
        np.zeros(0), convolved=False)
    errs = []
    for n in (1, 2, 3, 5, 7, 11):
        L = O.OracleSystem(make_spec(comps, nx=3, ny=3, h=0.05, rule=("gl", n))).render(
            np.zeros(0), convolved=False)
        errs.append(np.abs(L - ref).max() / np.abs(ref).max())
    assert errs[-1] < 1e-3 * errs[0]
    assert errs[-1] < 1e-4
    # brute force by scipy dblquad on one pixel: a smooth profile (n = 1/2)
    # with GL 7, and a cusped one (n = 1) with GL 64
    for n, order, tol in ((0.5, 7, 1e-9), (1.0, 64, 1e-5)):
        comps2 = [component("sersic", "foreground", [fixed(0.01), fixed(0.005), fixed(0.03),
                                                     fixed(0), fixed(n), fixed(0.8), fixed(0)])]
        L = O.OracleSystem(make_spec(comps2, nx=1, ny=1, h=0.05, rule=("gl", order))).render(
            np.zeros(0), convolved=False)[0, 0]
        bn = sp.gammaincinv(2 * n, 0.5)
        I0 = bn ** (2 * n) / (2 * math.pi * n * 0.03 ** 2 * math.gamma(2 * n))

        def I(y, x):
            u, v = x - 0.01, y - 0.005
            return I0 * math.exp(-bn * (math.sqrt(u * u * 0.8 + v * v / 0.8) / 0.03) ** (1 / n))

        exact = si.dblquad(I, -0.025, 0.025, -0.025, 0.025, epsabs=0, epsrel=1e-12)[0]
        assert abs(L - exact) < tol * exact, (n, L, exact)


# --------------------------------------------------------------------------
# PSF convolution (Sec. 3.1, Eq. 15) and likelihood (Sec. 3.2, Eq. 17)

def test_psf_matches_scipy_with_edge_padding():
    rng = np.random.default_rng(3)
    L = rng.random((13, 17))
    F = rng.random((5, 7))  # p = 2 rows, q = 3 columns, not symmetric
    spec = make_spec([], nx=17, ny=13, psf=F)
    got = O.OracleSystem(spec).convolve(L)
    want = ss.convolve2d(np.pad(L, ((2, 2), (3, 3)), mode="edge"), F / F.sum(), mode="valid")
    assert np.abs(got - want).max() < 1e-14


def test_psf_identities():
    rng = np.random.default_rng(4)
    L = rng.random((9, 11))
    delta = np.zeros((7, 5))
    delta[3, 2] = 5.0  # normalised automatically
    got = O.OracleSystem(make_spec([], nx=11, ny=9, psf=delta)).convolve(L)
    assert np.abs(got - L).max() < 1e-15
    const = np.full((9, 11), 2.5)
    got = O.OracleSystem(make_spec([], nx=11, ny=9, psf=rng.random((7, 7)))).convolve(const)
    assert np.abs(got - 2.5).max() < 1e-14
    # a shifted delta moves the image: F_{k,l} = delta at (k, l) = (1, 0)
    # gives L*_ij = L_{i-1, j} (true convolution), clamped at the border
    sh = np.zeros((3, 3))
    sh[2, 1] = 1.0
    got = O.OracleSystem(make_spec([], nx=11, ny=9, psf=sh)).convolve(L)
    assert np.array_equal(got[1:], L[:-1]) and np.array_equal(got[0], L[0])


def test_loglike_closed_forms():
    rng = np.random.default_rng(5)
    ny, nx = 10, 12
    Ls = rng.random((ny, nx))
    var = rng.uniform(0.5, 2.0, (ny, nx))
    mask = (rng.random((ny, nx)) < 0.3).astype(np.uint8)
    extra = rng.uniform(0.5, 1.5, (ny, nx))
    spec = make_spec([], nx=nx, ny=ny, mask=mask)
    # d = L*: loglike 0
    o = O.OracleSystem(spec, {"data": Ls, "variance": var})
    assert o.loglike_of_image(Ls) == 0.0
    # constant offset c: -1/2 c^2 sum(w), masked pixels excluded
    c = 0.3
    o = O.OracleSystem(spec, {"data": Ls + c, "variance": var}, extra_weight=extra)
    w = extra / var * (mask == 0)
    assert abs(o.loglike_of_image(Ls) - (-0.5 * c * c * w.sum())) < 1e-13
    # masked pixels contribute nothing even if wildly off
    d = Ls + c
    d[mask != 0] += 1e6
    o = O.OracleSystem(spec, {"data": d, "variance": var}, extra_weight=extra)
    assert abs(o.loglike_of_image(Ls) - (-0.5 * c * c * w.sum())) < 1e-13


def test_variance_from_gain_and_offset():
    # Sec. 3.3: s^2 = (d + b) / g, w = extra / s^2
    rng = np.random.default_rng(6)
    d = rng.uniform(0.1, 3.0, (6, 7))
    g, b = 250.0, 0.4
    extra = rng.uniform(0.5, 2, (6, 7))
    o = O.OracleSystem(make_spec([], nx=7, ny=6), {"data": d, "gain": g, "offset": b},
                       extra_weight=extra)
    assert np.allclose(o.weights(), extra * g / (d + b), rtol=1e-15)
    bad = d.copy()
    bad[2, 3] = -b - 1.0
    with pytest.raises(RuntimeError):
        O.OracleSystem(make_spec([], nx=7, ny=6), {"data": bad, "gain": g, "offset": b}).weights()


def test_invalid_points_are_minus_inf():
    spec = W.c1_small()
    obs = O.mock_observation(spec)
    o = O.OracleSystem(spec, obs)
    t = np.array(spec["truth"])
    bad = np.tile(t, (5, 1))
    bad[0, 3] = 1.2    # SIE q > 1
    bad[1, 3] = 0.0    # SIE q = 0
    bad[2, 9] = -0.1   # source r < 0
    bad[3, 10] = 0.0   # n = 0
    bad[4, 2] = -1.0   # b < 0
    ll = o.loglike(np.vstack([bad, t]))
    assert np.all(np.isneginf(ll[:5])) and np.isfinite(ll[5])


def test_mock_truth_chi2_is_noise_level():
    # At the truth of the C1 mock (Gaussian noise sigma = 0.01 and matching
    # variance), chi^2 / N is 1 within its sampling spread sqrt(2/N).
    spec = W.c1_small()
    o = O.OracleSystem(spec, O.mock_observation(spec))
    ll = o.loglike(np.array(spec["truth"]))[0]
    N = 64 * 64
    assert abs(-2 * ll / N - 1) < 5 * math.sqrt(2 / N)
