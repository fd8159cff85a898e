"""Python front end of the plain FP64 CPU oracle (``lensed_oracle.c``).

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the CPU
baseline leg of the benchmark are the only callers.  The CUDA library never
imports this module, and this module imports nothing from the CUDA library.

``build()`` compiles the C file with gcc (plain -O2, IEEE semantics, OpenMP
over parameter points).  Inputs are the workload specs of the seeded input
module: a dict with nx, ny, h, rule, psf, mask, components, ...
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lensed_oracle.c")
_OUT = os.path.join(_HERE, "_build", "liblensed_oracle.so")

TYPES = {"sie": 1, "shear": 2, "pointmass": 3, "sersic": 4, "devauc": 5, "gauss": 6, "sky": 7}
PLANES = {"lens": 0, "foreground": 1, "source": 2, "source_image": 3}
RULES = {"point": 0, "sub": 1, "gl": 2, "gk": 3}
MAXPAR = 8


class Component(C.Structure):
    _fields_ = [("type", C.c_int), ("plane", C.c_int),
                ("free_index", C.c_int * MAXPAR), ("value", C.c_double * MAXPAR)]


class System(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("h", C.c_double),
                ("data", C.c_void_p), ("variance", C.c_void_p),
                ("gain", C.c_double), ("offset", C.c_double),
                ("extra_weight", C.c_void_p), ("mask", C.c_void_p),
                ("psf", C.c_void_p), ("psf_nx", C.c_int), ("psf_ny", C.c_int),
                ("rule", C.c_int), ("order", C.c_int), ("zeropoint", C.c_double),
                ("ncomp", C.c_int), ("comp", C.c_void_p), ("nparam", C.c_int)]


def build(force=False):
    """Compile the oracle shared library (gcc, -O2, OpenMP)."""
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    if not force and os.path.exists(_OUT) and os.path.getmtime(_OUT) >= os.path.getmtime(_SRC):
        return _OUT
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-shared", "-fPIC", _SRC, "-o", _OUT + ".tmp",
           "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(_OUT + ".tmp", _OUT)
    return _OUT


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_OUT)
        dp = C.POINTER(C.c_double)
        L.ora_gauss_legendre.argtypes = [C.c_int, dp, dp]
        L.ora_rule_nodes.argtypes = [C.c_int, C.c_int, dp, dp]
        L.ora_gauss_kronrod.argtypes = [C.c_int, dp, dp, dp]
        L.ora_render_error.argtypes = [C.c_void_p, dp, dp]
        L.ora_gammainc_lower.argtypes = [C.c_double, C.c_double]
        L.ora_gammainc_lower.restype = C.c_double
        L.ora_sersic_bn.argtypes = [C.c_double]
        L.ora_sersic_bn.restype = C.c_double
        L.ora_sersic_I0.argtypes = [C.c_double, C.c_double, C.c_double]
        L.ora_sersic_I0.restype = C.c_double
        L.ora_deflection_one.argtypes = [C.c_int, dp, C.c_double, C.c_double, dp, dp]
        L.ora_sie_kappa.argtypes = [dp, C.c_double, C.c_double]
        L.ora_sie_kappa.restype = C.c_double
        L.ora_render.argtypes = [C.c_void_p, dp, C.c_int, dp]
        L.ora_loglike_batch.argtypes = [C.c_void_p, dp, C.c_int, dp, C.c_int]
        L.ora_psf_convolve.argtypes = [C.c_void_p, dp, dp]
        L.ora_loglike_image.argtypes = [C.c_void_p, dp]
        L.ora_loglike_image.restype = C.c_double
        L.ora_weights.argtypes = [C.c_void_p, dp]
        _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


class OracleSystem:
    """One imaging system marshalled for the C oracle.  ``obs`` is the
    observation dict from ``add_noise`` (data + variance or gain/offset);
    without it the system can only render."""

    def __init__(self, spec, obs=None, extra_weight=None):
        self.spec = spec
        nx, ny = spec["nx"], spec["ny"]
        self._keep = []

        def arr(a, dtype=np.float64):
            if a is None:
                return None
            a = np.ascontiguousarray(np.asarray(a, dtype=dtype).reshape(-1))
            self._keep.append(a)
            return a

        comps = spec["components"]
        self.comp = (Component * len(comps))()
        for c, cd in enumerate(comps):
            self.comp[c].type = TYPES[cd["type"]]
            self.comp[c].plane = PLANES[cd["plane"]]
            for k in range(MAXPAR):
                self.comp[c].free_index[k] = -1
                self.comp[c].value[k] = 0.0
            for k, (kind, v) in enumerate(cd["params"]):
                if kind == "free":
                    self.comp[c].free_index[k] = int(v)
                else:
                    self.comp[c].value[k] = float(v)
        s = System()
        s.nx, s.ny, s.h = nx, ny, spec["h"]
        obs = obs or {}
        self.data = arr(obs.get("data"))
        self.variance = arr(obs.get("variance"))
        self.extra = arr(extra_weight)
        self.mask = arr(spec.get("mask"), np.uint8)
        self.psf = arr(spec.get("psf"))
        s.data = self.data.ctypes.data if self.data is not None else None
        s.variance = self.variance.ctypes.data if self.variance is not None else None
        s.gain = float(obs.get("gain", 1.0))
        s.offset = float(obs.get("offset", 0.0))
        s.extra_weight = self.extra.ctypes.data if self.extra is not None else None
        s.mask = self.mask.ctypes.data if self.mask is not None else None
        if self.psf is not None:
            ps = np.asarray(spec["psf"]).shape
            s.psf = self.psf.ctypes.data
            s.psf_ny, s.psf_nx = ps
        else:
            s.psf = None
            s.psf_nx = s.psf_ny = 0
        rule, order = spec["rule"]
        s.rule, s.order = RULES[rule], int(order)
        s.zeropoint = float(spec.get("zeropoint", 0.0))
        s.ncomp = len(comps)
        s.comp = C.cast(self.comp, C.c_void_p)
        s.nparam = int(spec["n_params"])
        self.sys = s

    def render(self, xi, convolved=True):
        xi = np.ascontiguousarray(xi, dtype=np.float64)
        out = np.zeros(self.spec["ny"] * self.spec["nx"])
        rc = lib().ora_render(C.byref(self.sys), _dp(xi), int(bool(convolved)), _dp(out))
        if rc < 0:
            raise RuntimeError("oracle render failed")
        if rc == 1:
            return None
        return out.reshape(self.spec["ny"], self.spec["nx"])

    def render_error(self, xi):
        """Per-pixel Gauss-Kronrod error estimate |L_K - L_G| (unconvolved)."""
        xi = np.ascontiguousarray(xi, dtype=np.float64)
        out = np.zeros(self.spec["ny"] * self.spec["nx"])
        rc = lib().ora_render_error(C.byref(self.sys), _dp(xi), _dp(out))
        if rc < 0:
            raise RuntimeError("oracle error map failed (rule not Gauss-Kronrod?)")
        if rc == 1:
            return None
        return out.reshape(self.spec["ny"], self.spec["nx"])

    def loglike(self, xis, nthreads=None):
        xis = np.ascontiguousarray(np.atleast_2d(xis), dtype=np.float64)
        assert xis.shape[1] == self.spec["n_params"]
        out = np.zeros(xis.shape[0])
        nt = nthreads if nthreads else (os.cpu_count() or 1)
        rc = lib().ora_loglike_batch(C.byref(self.sys), _dp(xis), xis.shape[0], _dp(out), nt)
        if rc != 0:
            raise RuntimeError("oracle loglike failed")
        return out

    def weights(self):
        w = np.zeros(self.spec["ny"] * self.spec["nx"])
        if lib().ora_weights(C.byref(self.sys), _dp(w)) != 0:
            raise RuntimeError("non-positive or non-finite variance")
        return w.reshape(self.spec["ny"], self.spec["nx"])

    def convolve(self, L):
        L = np.ascontiguousarray(L, dtype=np.float64).reshape(-1)
        out = np.zeros_like(L)
        lib().ora_psf_convolve(C.byref(self.sys), _dp(L), _dp(out))
        return out.reshape(self.spec["ny"], self.spec["nx"])

    def loglike_of_image(self, Ls):
        Ls = np.ascontiguousarray(Ls, dtype=np.float64).reshape(-1)
        return lib().ora_loglike_image(C.byref(self.sys), _dp(Ls))


def mock_observation(spec, seed=None):
    """Observation rendered by the oracle at the spec's truth plus noise."""
    import workloads
    img = OracleSystem(spec).render(np.asarray(spec["truth"], float), convolved=True)
    return workloads.add_noise(spec, img, spec["seed"] if seed is None else seed)


# --- stand-alone routines for the pins -------------------------------------

def gauss_legendre(n):
    x = np.zeros(n)
    w = np.zeros(n)
    if lib().ora_gauss_legendre(n, _dp(x), _dp(w)) != 0:
        raise RuntimeError("gauss_legendre failed")
    return x, w


def gauss_kronrod(n):
    """(2n+1)-point Kronrod extension of the n-point Gauss rule on [-1, 1]:
    nodes ascending, Kronrod weights, embedded Gauss weights (zero on the
    added nodes)."""
    x, wk, wg = np.zeros(2 * n + 1), np.zeros(2 * n + 1), np.zeros(2 * n + 1)
    if lib().ora_gauss_kronrod(n, _dp(x), _dp(wk), _dp(wg)) != 0:
        raise RuntimeError("gauss_kronrod failed")
    return x, wk, wg


def rule_nodes(rule, order):
    t = np.zeros(256)
    w = np.zeros(256)
    n = lib().ora_rule_nodes(RULES[rule], order, _dp(t), _dp(w))
    if n < 1:
        raise RuntimeError("rule failed")
    return t[:n].copy(), w[:n].copy()


def gammainc_lower(a, x):
    return lib().ora_gammainc_lower(a, x)


def sersic_bn(n):
    return lib().ora_sersic_bn(n)


def sersic_I0(n, r, F):
    return lib().ora_sersic_I0(n, r, F)


def deflection(ctype, p, x, y):
    p = np.zeros(MAXPAR) + np.pad(np.asarray(p, float), (0, MAXPAR - len(p)))
    ax = C.c_double()
    ay = C.c_double()
    lib().ora_deflection_one(TYPES[ctype], _dp(p), float(x), float(y), C.byref(ax), C.byref(ay))
    return ax.value, ay.value


def sie_kappa(p, x, y):
    p = np.pad(np.asarray(p, float), (0, MAXPAR - len(p)))
    return lib().ora_sie_kappa(_dp(p), float(x), float(y))
