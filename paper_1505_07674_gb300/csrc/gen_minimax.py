"""Write lensed_minimax.cuh: the polynomial cores of the FP32 SIE's atan and atanh.

The SIE deflection (Sec. 2.1, Eqs. 1-3) needs atan(N/D) and atanh(N/D) per ray.
The FP32 ray kernel evaluates them as

    atan(t)  = t + t^3 Qa(t^2),   0 <= t <= 1  (t = min(|N|, D) / max(|N|, D),
                                                 pi/2 - atan(1/t) beyond 1)
    atanh(z) = z + z^3 Qh(z^2),   |z| <= 1/2   (0.5 ln((D + N) / (D - N)) beyond)

with Qa of degree 7 and Qh of degree 5.  The coefficients are minimax in the
relative error of the whole function, fitted here by Lawson's iteratively
reweighted least squares (C. L. Lawson, 1961): repeated weighted least-squares
fits whose weights grow where the error is largest converge to the
equioscillating (Chebyshev) fit.  Run from the repository root:

    python paper_1505_07674_gb300/csrc/gen_minimax.py
"""
from __future__ import annotations

import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
HEADER = os.path.join(HERE, "lensed_minimax.cuh")

# (name, f(u) = F(sqrt u) / sqrt u, u range, degree of Q)
FITS = (
    ("kAtanQ", lambda u: np.arctan(np.sqrt(u)) / np.sqrt(u), 1.0, 7),
    ("kAtanhQ", lambda u: np.arctanh(np.sqrt(u)) / np.sqrt(u), 0.25, 5),
)
# the device function that evaluates each Q
FUNCS = {"kAtanQ": "minimax_atan_q", "kAtanhQ": "minimax_atanh_q"}


def lawson_fit(f, hi, deg, nodes=6000, iters=60):
    """Q with F(t) ~ t + t^3 Q(t^2) minimax in relative error over u = t^2 in (0, hi].

    The relative error of t (1 + u Q(u)) against F(t) = t f(u) is
    u (Q(u) - (f(u) - 1) / u) / f(u): a weighted fit of (f - 1) / u.
    """
    u = np.maximum((1.0 - np.cos(np.linspace(0.0, np.pi, nodes))) * hi / 2.0, 1e-12)
    fu = f(u)
    y = (fu - 1.0) / u
    scale = u / fu
    V = np.vander(u, deg + 1, increasing=True)
    w = np.full(nodes, 1.0 / nodes)
    for _ in range(iters):
        sw = np.sqrt(w) * scale
        c, *_ = np.linalg.lstsq(V * sw[:, None], y * sw, rcond=None)
        err = np.abs(V @ c - y) * scale
        w = w * (err / err.max()) + 1e-15
        w /= w.sum()
    return c, float(err.max())


def coefficients():
    """{name: float32 coefficients (constant term first)}."""
    return {name: np.float32(lawson_fit(f, hi, deg)[0]) for name, f, hi, deg in FITS}


def eval_f32(coef, t):
    """t + t^3 Q(t^2) in float32, Horner in fused multiply-adds as the kernel does."""
    t = np.asarray(t, np.float32)
    u = (t * t).astype(np.float32)
    r = np.full(t.shape, coef[-1], np.float32)
    for c in coef[-2::-1]:
        r = (r.astype(np.float64) * u + np.float64(c)).astype(np.float32)
    tu = (t * u).astype(np.float32)
    return (tu.astype(np.float64) * r + t).astype(np.float32)


def render(coefs):
    out = [
        "// Generated by gen_minimax.py (Lawson minimax fits; do not edit).",
        "// atan(t) = t + t^3 Qa(t^2) on [0, 1]; atanh(z) = z + z^3 Qh(z^2) on [0, 1/2].",
        "// Each function evaluates Q(u) by Horner's rule in fused multiply-adds, for",
        "// one ray (V = float) or a pair of rays (V = float2, packed instructions).",
        "#pragma once",
        "",
        '#include "lensed_vec2.cuh"',
        "",
        "namespace lensed {",
    ]
    for name, c in coefs.items():
        out.append("template <class V>")
        out.append(f"__device__ __forceinline__ V {FUNCS[name]}(V u)")
        out.append("{")
        out.append(f"    V q = vsplat<V>({float(c[-1]):.9e}f);")
        for v in c[-2::-1]:
            out.append(f"    q = vfma(q, u, vsplat<V>({float(v):.9e}f));")
        out.append("    return q;")
        out.append("}")
    out += ["}  // namespace lensed", ""]
    return "\n".join(out)


def parse(path=HEADER):
    """Coefficients as written in the header (constant term first)."""
    coefs, name, cur = {}, None, []
    inv = {v: k for k, v in FUNCS.items()}

    def number(text):
        return float(text.strip().rstrip(";").rstrip(")").rstrip(")").rstrip("f"))

    for line in open(path):
        line = line.strip()
        if line.startswith("__device__"):
            name, cur = inv[line.split("(")[0].split()[-1]], []
        elif line.startswith("V q = vsplat<V>("):
            cur.append(number(line.split("vsplat<V>(")[1]))
        elif line.startswith("q = vfma("):
            cur.append(number(line.split("vsplat<V>(")[1]))
        elif line.startswith("return q;") and name:
            coefs[name] = np.array(cur[::-1], np.float32)
    return coefs


if __name__ == "__main__":
    with open(HEADER, "w") as fh:
        fh.write(render(coefficients()))
    print("wrote", HEADER)
