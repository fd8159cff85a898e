"""Seeded synthetic inputs for the ray-tracing likelihood.

This module draws inputs only: model layouts, truth parameters, prior boxes,
parameter points, PSF arrays, masks and noise.  It holds none of the forward
model's or the likelihood's arithmetic, so the CUDA library and the FP64
oracle can both consume it.  The mock observation itself is the noiseless
image of whichever implementation is under test plus the noise drawn here
(``add_noise``).

The shapes and value ranges follow the paper's HST-like mocks (Sec. 4: 0.05
arcsec pixels, SIE lens with r_L = 1.3624", q_L = 0.75, PA 45 deg; de
Vaucouleurs foreground of r_H = 2", q_H in [0.6, 0.9], PA_H in [25, 65] deg,
16.5 mag; Sersic sources with n, r_S, q_S, PA_S drawn uniformly, 23 mag,
placed inside a disc around the caustic) scaled to the workload sizes below.
Where the paper's data (Glamer mocks, TinyTim PSF, HST images) are not
available, these seeded stand-ins take their place.

Component parameter order (the same on both sides):
    sie        x, y, b, q, pa_deg, s
    shear      x, y, gamma, phi_deg
    pointmass  x, y, theta_E
    sersic     x, y, r_e, mag, n, q, pa_deg
    devauc     x, y, r_e, mag, q, pa_deg
    gauss      x, y, sigma, mag, q, pa_deg
    sky        surface brightness per arcsec^2 (flat sky)
Planes: "lens" (mass), "foreground" (light at the image position), "source"
(light at the traced position), "source_image" (a source whose x, y are an
image-plane position: the image-plane prior).
"""
from __future__ import annotations

import math

import numpy as np

NPAR = {"sie": 6, "shear": 4, "pointmass": 3, "sersic": 7, "devauc": 6, "gauss": 6, "sky": 1}
MASS_TYPES = ("sie", "shear", "pointmass")


def free(k):
    return ("free", int(k))


def fixed(v):
    return ("fixed", float(v))


def component(ctype, plane, params):
    assert len(params) == NPAR[ctype], (ctype, len(params))
    if ctype in MASS_TYPES:
        assert plane == "lens"
    elif ctype == "sky":
        assert plane in ("foreground", "source")
    else:
        assert plane in ("foreground", "source", "source_image")
    return {"type": ctype, "plane": plane, "params": list(params)}


def gaussian_psf(size, fwhm, h, halo_frac=0.0, halo_fwhm=None):
    """Unnormalised (size x size) PSF array: a Gaussian core of the given FWHM
    (arcsec), optionally plus a broader Gaussian halo carrying halo_frac of
    the light.  Sampled at pixel centres; the consumer normalises it."""
    assert size % 2 == 1
    r = (np.arange(size) - size // 2) * h
    xx, yy = np.meshgrid(r, r)
    rr = xx * xx + yy * yy

    def g(f):
        s = f / 2.3548200450309493
        a = np.exp(-rr / (2 * s * s))
        return a / a.sum()

    psf = (1.0 - halo_frac) * g(fwhm)
    if halo_frac > 0:
        psf = psf + halo_frac * g(halo_fwhm)
    return psf


def annular_mask(nx, ny, h, r_in, r_out):
    """uint8 mask, nonzero = excluded: keeps r_in <= r <= r_out (arcsec)."""
    x = (np.arange(nx) - 0.5 * (nx - 1)) * h
    y = (np.arange(ny) - 0.5 * (ny - 1)) * h
    xx, yy = np.meshgrid(x, y)
    r = np.hypot(xx, yy)
    return (~((r >= r_in) & (r <= r_out))).astype(np.uint8)


def draw_points(spec, P, seed):
    """P parameter points drawn uniformly from the spec's prior box."""
    rng = np.random.default_rng(seed)
    lo = np.asarray(spec["prior_lo"], float)
    hi = np.asarray(spec["prior_hi"], float)
    return lo + (hi - lo) * rng.random((P, len(lo)))


def add_noise(spec, noiseless, seed):
    """Observation d = noiseless image + the spec's noise model.

    Returns a dict with ``data`` and either ``variance`` or ``gain``/``offset``
    (the latter for the Poisson model, whose variance the consumer estimates
    from the data as the paper's Sec. 3.3 prescribes)."""
    rng = np.random.default_rng(seed)
    noise = spec["noise"]
    img = np.asarray(noiseless, float)
    if noise["kind"] == "gaussian":
        sigma = noise["sigma"] if "sigma" in noise else noise["sigma_frac"] * float(img.max())
        d = img + sigma * rng.standard_normal(img.shape)
        return {"data": d, "variance": np.full(img.shape, sigma * sigma)}
    if noise["kind"] == "poisson":
        # Sky offset b and read noise as fractions of the peak pixel, gain
        # chosen so the peak pixel has the requested signal-to-noise.
        Lmax = float(img.max())
        b = noise["sky_frac"] * Lmax
        sr = noise["read_frac"] * Lmax
        snr = noise["snr"]
        g = snr * snr * (Lmax + b) / (Lmax * Lmax - snr * snr * sr * sr)
        counts = rng.poisson(np.clip(g * (img + b), 0, None))
        d = counts / g - b + sr * rng.standard_normal(img.shape)
        return {"data": d, "gain": g, "offset": b}
    raise ValueError(noise["kind"])


# ---------------------------------------------------------------------------
# Workloads

def c1_small(seed=1001):
    """One 64x64 image at 0.05"/px; SIE (b=1", q=0.8, PA 30 deg, core 0.01")
    plus external shear (gamma=0.05); Sersic source (n=1, r_e=0.2", q=0.7)
    offset 0.1" along +x; no lens light; 5x5 Gauss-Legendre rays per pixel;
    7x7 Gaussian PSF of FWHM 0.1"; Gaussian noise sigma = 0.01; 13 free
    parameters with uniform box priors."""
    comps = [
        component("sie", "lens", [free(0), free(1), free(2), free(3), free(4), fixed(0.01)]),
        component("shear", "lens", [free(0), free(1), free(5), free(6)]),
        component("sersic", "source", [free(7), free(8), free(9), fixed(0.0), free(10),
                                       free(11), free(12)]),
    ]
    names = ["x_L", "y_L", "b_L", "q_L", "pa_L", "gamma", "phi",
             "x_S", "y_S", "r_S", "n_S", "q_S", "pa_S"]
    lo = [-0.05, -0.05, 0.8, 0.5, 0.0, 0.0, 0.0, -0.3, -0.3, 0.1, 0.5, 0.3, 0.0]
    hi = [0.05, 0.05, 1.2, 0.99, 180.0, 0.1, 180.0, 0.3, 0.3, 0.4, 4.0, 1.0, 180.0]
    truth = [0.0, 0.0, 1.0, 0.8, 30.0, 0.05, 0.0, 0.1, 0.0, 0.2, 1.0, 0.7, 0.0]
    return {
        "name": "c1_64x64_gl5_psf7",
        "nx": 64, "ny": 64, "h": 0.05,
        "rule": ("gl", 5),
        "psf": gaussian_psf(7, 0.1, 0.05),
        "mask": None,
        "zeropoint": 0.0,
        "components": comps,
        "n_params": 13, "param_names": names,
        "prior_lo": lo, "prior_hi": hi, "truth": truth,
        "noise": {"kind": "gaussian", "sigma": 0.01},
        "seed": seed,
    }


def c2_hst(seed=1002):
    """HST-like single system: 200x200 at 0.05"; SIE (b=1.3624", q=0.75, PA
    45 deg, core 0.01") + external shear; de Vaucouleurs lens light (r_H=2",
    16.5 mag, q_H and PA_H drawn in [0.6, 0.9] and [25, 65] deg, co-centred,
    fixed); Sersic source (23 mag, n in [0.5, 4]) inside a disc of radius
    0.5 b; 21x21 PSF (0.9 Gaussian FWHM 0.1" + 0.1 halo FWHM 0.5"); annular
    mask 0.5"-3"; Poisson + read noise with the peak pixel at SNR ~ 50;
    11 free parameters (SIE b, q, PA; shear gamma, phi; source x, y, r, n,
    q, PA).  The quadrature is 5x5 Gauss-Legendre."""
    rng = np.random.default_rng(seed)
    qH = rng.uniform(0.6, 0.9)
    paH = rng.uniform(25.0, 65.0)
    rad = 0.5 * 1.3624 * math.sqrt(rng.random())
    ang = rng.uniform(0, 2 * math.pi)
    xs, ys = rad * math.cos(ang), rad * math.sin(ang)
    comps = [
        component("sie", "lens", [fixed(0.0), fixed(0.0), free(0), free(1), free(2), fixed(0.01)]),
        component("shear", "lens", [fixed(0.0), fixed(0.0), free(3), free(4)]),
        component("devauc", "foreground", [fixed(0.0), fixed(0.0), fixed(2.0), fixed(16.5),
                                           fixed(qH), fixed(paH)]),
        component("sersic", "source", [free(5), free(6), free(7), fixed(23.0), free(8),
                                       free(9), free(10)]),
    ]
    names = ["b_L", "q_L", "pa_L", "gamma", "phi", "x_S", "y_S", "r_S", "n_S", "q_S", "pa_S"]
    lo = [1.2, 0.5, 0.0, 0.0, 0.0, -0.7, -0.7, 0.1, 0.5, 0.1, 0.0]
    hi = [1.5, 0.99, 180.0, 0.1, 180.0, 0.7, 0.7, 0.4, 4.0, 1.0, 180.0]
    truth = [1.3624, 0.75, 45.0, 0.03, 20.0, xs, ys,
             rng.uniform(0.1, 0.4), rng.uniform(0.5, 4.0), rng.uniform(0.1, 1.0),
             rng.uniform(0.0, 180.0)]
    return {
        "name": "c2_200x200_gl5_psf21_annulus",
        "nx": 200, "ny": 200, "h": 0.05,
        "rule": ("gl", 5),
        "psf": gaussian_psf(21, 0.1, 0.05, halo_frac=0.1, halo_fwhm=0.5),
        "mask": annular_mask(200, 200, 0.05, 0.5, 3.0),
        "zeropoint": 23.0,
        "components": comps,
        "n_params": 11, "param_names": names,
        "prior_lo": lo, "prior_hi": hi, "truth": truth,
        "noise": {"kind": "poisson", "snr": 50.0, "sky_frac": 0.05, "read_frac": 0.002},
        "seed": seed,
    }


def c3_system(k, seed=1003):
    """System k of the batched uneven workload: nx, ny uniform integers in
    [48, 320] at 0.05"; Gauss-Legendre order uniform in 3..7; odd PSF size
    uniform in 7..31 with a Gaussian FWHM in [0.08, 0.2]"; SIE (b in
    [0.5, 1.5], q in [0.5, 0.99]) + shear (gamma <= 0.1), plus a point mass
    (theta_E in [0.05, 0.3]", within 1") with probability 1/2; Sersic source.
    Free: SIE x, y, b, q, PA; shear gamma, phi; [point mass x, y, theta_E];
    source x, y, r, n, q, PA (13 or 16 parameters)."""
    rng = np.random.default_rng([seed, k])
    nx = int(rng.integers(48, 321))
    ny = int(rng.integers(48, 321))
    order = int(rng.integers(3, 8))
    psf_size = int(rng.choice(np.arange(7, 32, 2)))
    fwhm = float(rng.uniform(0.08, 0.2))
    has_pm = bool(rng.random() < 0.5)
    b = float(rng.uniform(0.5, 1.5))
    comps = [
        component("sie", "lens", [free(0), free(1), free(2), free(3), free(4), fixed(0.01)]),
        component("shear", "lens", [free(0), free(1), free(5), free(6)]),
    ]
    names = ["x_L", "y_L", "b_L", "q_L", "pa_L", "gamma", "phi"]
    lo = [-0.05, -0.05, 0.5, 0.5, 0.0, 0.0, 0.0]
    hi = [0.05, 0.05, 1.5, 0.99, 180.0, 0.1, 180.0]
    truth = [0.0, 0.0, b, float(rng.uniform(0.5, 0.99)), float(rng.uniform(0, 180)),
             float(rng.uniform(0, 0.1)), float(rng.uniform(0, 180))]
    k0 = 7
    if has_pm:
        comps.append(component("pointmass", "lens", [free(k0), free(k0 + 1), free(k0 + 2)]))
        names += ["x_P", "y_P", "thetaE_P"]
        lo += [-1.0, -1.0, 0.05]
        hi += [1.0, 1.0, 0.3]
        r = float(rng.uniform(0.3, 1.0))
        a = float(rng.uniform(0, 2 * math.pi))
        truth += [r * math.cos(a), r * math.sin(a), float(rng.uniform(0.05, 0.3))]
        k0 += 3
    comps.append(component("sersic", "source", [free(k0), free(k0 + 1), free(k0 + 2), fixed(0.0),
                                                free(k0 + 3), free(k0 + 4), free(k0 + 5)]))
    names += ["x_S", "y_S", "r_S", "n_S", "q_S", "pa_S"]
    lo += [-0.5 * b, -0.5 * b, 0.1, 0.5, 0.3, 0.0]
    hi += [0.5 * b, 0.5 * b, 0.4, 4.0, 1.0, 180.0]
    rad = 0.5 * b * math.sqrt(rng.random())
    ang = rng.uniform(0, 2 * math.pi)
    truth += [rad * math.cos(ang), rad * math.sin(ang), float(rng.uniform(0.1, 0.4)),
              float(rng.uniform(0.5, 4.0)), float(rng.uniform(0.3, 1.0)),
              float(rng.uniform(0, 180))]
    return {
        "name": f"c3_sys{k}_{nx}x{ny}_gl{order}_psf{psf_size}",
        "nx": nx, "ny": ny, "h": 0.05,
        "rule": ("gl", order),
        "psf": gaussian_psf(psf_size, fwhm, 0.05),
        "mask": None,
        "zeropoint": 0.0,
        "components": comps,
        "n_params": len(names), "param_names": names,
        "prior_lo": lo, "prior_hi": hi, "truth": truth,
        "noise": {"kind": "gaussian", "sigma_frac": 0.02},
        "seed": seed * 1000 + k,
    }


def c3_batch(n_systems=256, seed=1003):
    return [c3_system(k, seed) for k in range(n_systems)]


def c4_euclid(seed=1004):
    """Euclid-like 400x400 at 0.1"; 15x15 Gaussian PSF (FWHM 0.18"); SIE +
    shear, Sersic lens light and two Sersic sources; 18 free parameters: SIE
    x, y, b, q, PA (5), shear gamma, phi (2), lens light r, n, q, PA (4,
    centre tied to the SIE, magnitude fixed), source A x, y, r, n, q (5),
    source B x, y (2).  Poisson noise at peak SNR ~ 50; 5x5
    Gauss-Legendre."""
    rng = np.random.default_rng(seed)
    comps = [
        component("sie", "lens", [free(0), free(1), free(2), free(3), free(4), fixed(0.01)]),
        component("shear", "lens", [free(0), free(1), free(5), free(6)]),
        component("sersic", "foreground", [free(0), free(1), free(7), fixed(18.0), free(8),
                                           free(9), free(10)]),
        component("sersic", "source", [free(11), free(12), free(13), fixed(22.5), free(14),
                                       free(15), fixed(30.0)]),
        component("sersic", "source", [free(16), free(17), fixed(0.1), fixed(24.0), fixed(1.0),
                                       fixed(0.8), fixed(100.0)]),
    ]
    names = ["x_L", "y_L", "b_L", "q_L", "pa_L", "gamma", "phi",
             "r_H", "n_H", "q_H", "pa_H",
             "x_A", "y_A", "r_A", "n_A", "q_A", "x_B", "y_B"]
    lo = [-0.1, -0.1, 1.0, 0.5, 0.0, 0.0, 0.0, 0.5, 2.0, 0.5, 0.0,
          -0.5, -0.5, 0.1, 0.5, 0.3, -0.5, -0.5]
    hi = [0.1, 0.1, 1.6, 0.99, 180.0, 0.1, 180.0, 2.5, 6.0, 1.0, 180.0,
          0.5, 0.5, 0.5, 4.0, 1.0, 0.5, 0.5]
    truth = [0.0, 0.0, 1.3, 0.75, 45.0, 0.04, 30.0, 1.5, 4.0, 0.8, 40.0,
             0.08, 0.05, 0.25, 1.5, 0.6, -0.2, 0.1]
    return {
        "name": "c4_400x400_h0.1_gl5_psf15",
        "nx": 400, "ny": 400, "h": 0.1,
        "rule": ("gl", 5),
        "psf": gaussian_psf(15, 0.18, 0.1),
        "mask": None,
        "zeropoint": 25.0,
        "components": comps,
        "n_params": 18, "param_names": names,
        "prior_lo": lo, "prior_hi": hi, "truth": truth,
        "noise": {"kind": "poisson", "snr": 50.0, "sky_frac": 0.05, "read_frac": 0.002},
        "seed": seed,
    }


def j0808_like(seed=1006, image_prior=False):
    """Multi-component lens in the style of the paper's J0808+4706 model
    (Sec. 5: two SIEs for a lens galaxy and its companion, two Sersic
    components for the main lens light, one for the companion, two Sersic
    sources) plus the flat sky of the paper's base model; 35 free
    parameters.  160x160 at 0.05" (HST ACS-like), 15x15 Gaussian PSF (FWHM
    0.1"), the paper's default g3k7 rule, Poisson noise at peak SNR ~ 50.

    Free parameters: sky S (1); main SIE x, y, b, q, PA (5); companion SIE
    x, y, b, q, PA (5); main light A r, mag, n, q, PA and main light B r,
    mag, q, PA (n = 1), both centred on the main SIE (9); companion light r,
    mag, n, centred on the companion SIE with its q and PA (3); source 1 x,
    y, r, mag, n, q, PA (7); source 2 x, y, r, mag, q (5).

    image_prior=True gives source 1's position as an image-plane position
    (the image-plane prior of Sec. 5): its truth and prior box are then on
    the image plane, near the arc."""
    comps = [
        component("sky", "foreground", [free(0)]),
        component("sie", "lens", [free(1), free(2), free(3), free(4), free(5), fixed(0.01)]),
        component("sie", "lens", [free(6), free(7), free(8), free(9), free(10), fixed(0.01)]),
        component("sersic", "foreground", [free(1), free(2), free(11), free(12), free(13),
                                           free(14), free(15)]),
        component("sersic", "foreground", [free(1), free(2), free(16), free(17), fixed(1.0),
                                           free(18), free(19)]),
        component("sersic", "foreground", [free(6), free(7), free(20), free(21), free(22),
                                           free(9), free(10)]),
        component("sersic", "source_image" if image_prior else "source",
                  [free(23), free(24), free(25), free(26), free(27), free(28), free(29)]),
        component("sersic", "source", [free(30), free(31), free(32), free(33), fixed(1.0),
                                       free(34), fixed(0.0)]),
    ]
    names = ["sky", "x_L", "y_L", "b_L", "q_L", "pa_L", "x_C", "y_C", "b_C", "q_C", "pa_C",
             "r_HA", "mag_HA", "n_HA", "q_HA", "pa_HA", "r_HB", "mag_HB", "q_HB", "pa_HB",
             "r_HC", "mag_HC", "n_HC",
             "x_1", "y_1", "r_1", "mag_1", "n_1", "q_1", "pa_1", "x_2", "y_2", "r_2", "mag_2",
             "q_2"]
    truth = [0.02, 0.0, 0.0, 1.2, 0.8, 40.0, 1.3, -0.9, 0.35, 0.9, 110.0,
             0.9, 17.5, 4.0, 0.8, 40.0, 0.3, 18.5, 0.7, 50.0,
             0.3, 19.5, 2.5,
             0.1, 0.05, 0.15, 22.0, 1.5, 0.6, 70.0, -0.15, 0.12, 0.1, 23.0, 0.7]
    lo = [-0.1, -0.1, -0.1, 0.9, 0.5, 0.0, 1.1, -1.1, 0.1, 0.5, 0.0,
          0.5, 16.5, 2.0, 0.5, 0.0, 0.1, 17.5, 0.4, 0.0,
          0.1, 18.5, 1.0,
          -0.4, -0.4, 0.05, 21.0, 0.5, 0.3, 0.0, -0.4, -0.4, 0.05, 22.0, 0.3]
    hi = [0.1, 0.1, 0.1, 1.5, 0.99, 180.0, 1.5, -0.7, 0.6, 0.99, 180.0,
          1.5, 18.5, 6.0, 0.99, 180.0, 0.6, 19.5, 0.99, 180.0,
          0.6, 20.5, 4.0,
          0.4, 0.4, 0.3, 23.0, 4.0, 0.99, 180.0, 0.4, 0.4, 0.3, 24.0, 0.99]
    name = "j0808like_160x160_h0.05_g3k7_psf15"
    if image_prior:
        truth[23], truth[24] = 0.75, 0.95
        lo[23], hi[23], lo[24], hi[24] = 0.45, 1.05, 0.65, 1.25
        name += "_imgprior"
    return {
        "name": name,
        "nx": 160, "ny": 160, "h": 0.05,
        "rule": ("gk", 3),
        "psf": gaussian_psf(15, 0.1, 0.05),
        "mask": None,
        "zeropoint": 25.0,
        "components": comps,
        "n_params": 35, "param_names": names,
        "prior_lo": lo, "prior_hi": hi, "truth": truth,
        "noise": {"kind": "poisson", "snr": 50.0, "sky_frac": 0.05, "read_frac": 0.002},
        "seed": seed,
    }


def rules_mock(k, seed=1007, snr=1000.0):
    """Mock k of the integration-rule comparison (the paper's Sec. 4.5, which
    repeats the exact-model test of Sec. 4.1 with each rule): 120 x 120 at
    0.05" (a 6" HST-like field), a singular isothermal ellipsoid at the
    centre (r_L = 1.3624", q_L = 0.75, PA 45 deg), a co-centred de
    Vaucouleurs foreground (r_H = 2", 16.5 mag, q_H in [0.6, 0.9], PA_H in
    [25, 65] deg) and a Sersic source (23 mag, n in [0.5, 8], r_S in [0.1,
    0.4]", q_S in [0.1, 1], PA_S in [0, 180) deg) placed uniformly in a disc
    of radius 0.5 r_L around the lens centre.  18 free parameters (5 + 6 +
    7), broad uniform priors.  21x21 PSF (Gaussian core plus halo) and
    Poisson + read noise; the peak pixel (the lens galaxy's centre) has SNR
    1000 by default, which leaves the arcs of the 6.5 mag fainter source at
    SNR ~ 10-100 per pixel, as in deep HST exposures.  The rule is set by the
    caller; the mock itself is rendered with a much finer one."""
    rng = np.random.default_rng([seed, k])
    comps = [
        component("sie", "lens", [free(0), free(1), free(2), free(3), free(4), fixed(0.0)]),
        component("devauc", "foreground", [free(5), free(6), free(7), free(8), free(9),
                                           free(10)]),
        component("sersic", "source", [free(11), free(12), free(13), free(14), free(15),
                                       free(16), free(17)]),
    ]
    names = ["x_L", "y_L", "r_L", "q_L", "pa_L", "x_H", "y_H", "r_H", "mag_H", "q_H", "pa_H",
             "x_S", "y_S", "r_S", "mag_S", "n_S", "q_S", "pa_S"]
    b = 1.3624
    rad = 0.5 * b * math.sqrt(rng.uniform())
    ang = rng.uniform(0, 2 * math.pi)
    truth = [0.0, 0.0, b, 0.75, 45.0,
             0.0, 0.0, 2.0, 16.5, float(rng.uniform(0.6, 0.9)), float(rng.uniform(25, 65)),
             rad * math.cos(ang), rad * math.sin(ang), float(rng.uniform(0.1, 0.4)), 23.0,
             float(rng.uniform(0.5, 8.0)), float(rng.uniform(0.1, 1.0)), float(rng.uniform(0, 180))]
    lo = [-0.3, -0.3, 1.0, 0.4, 0.0, -0.3, -0.3, 1.0, 15.5, 0.3, 0.0,
          -1.0, -1.0, 0.05, 21.0, 0.3, 0.05, 0.0]
    hi = [0.3, 0.3, 2.0, 1.0, 180.0, 0.3, 0.3, 4.0, 17.5, 1.0, 180.0,
          1.0, 1.0, 0.6, 25.0, 10.0, 1.0, 180.0]
    return {
        "name": f"rules_mock{k}_120x120_h0.05",
        "nx": 120, "ny": 120, "h": 0.05,
        "rule": ("gl", 16),
        "psf": gaussian_psf(21, 0.1, 0.05, halo_frac=0.1, halo_fwhm=0.5),
        "mask": None,
        "zeropoint": 23.0,
        "components": comps,
        "n_params": 18, "param_names": names,
        "prior_lo": lo, "prior_hi": hi, "truth": truth,
        "noise": {"kind": "poisson", "snr": float(snr), "sky_frac": 0.05, "read_frac": 0.0002},
        "seed": seed + k,
    }


def shrink(spec, nx, ny):
    """The same model on a smaller nx x ny field (mask recut to size), for
    quick parity cases."""
    s = dict(spec)
    s["nx"], s["ny"] = nx, ny
    if spec.get("mask") is not None:
        m = spec["mask"]
        cy, cx = m.shape[0] // 2, m.shape[1] // 2
        s["mask"] = m[cy - ny // 2: cy - ny // 2 + ny, cx - nx // 2: cx - nx // 2 + nx].copy()
    s["name"] = f"{spec['name']}_cut{nx}x{ny}"
    return s
