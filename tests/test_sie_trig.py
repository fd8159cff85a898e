"""The FP32 SIE's atan / atanh polynomial cores (Sec. 2.1, Eqs. 2-3).

The kernel's lensed_minimax.cuh holds minimax coefficients written by
csrc/gen_minimax.py.  These CPU tests pin them to the functions they stand
for: evaluated in float32 exactly as the kernel's Horner scheme does, they
stay within about one unit in the last place of numpy's FP64 arctan and
arctanh over their whole ranges, and the generator reproduces the committed
header.
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, os.path.join(ROOT, "paper_1505_07674_gb300", "csrc"))
import gen_minimax as G  # noqa: E402


def _ulps(got, ref):
    return np.abs(got.astype(np.float64) - ref) / np.spacing(np.abs(ref).astype(np.float32))


def test_atan_core_within_one_ulp_on_unit_interval():
    c = G.parse()["kAtanQ"]
    t = np.linspace(0.0, 1.0, 500_001, dtype=np.float32)[1:]
    assert _ulps(G.eval_f32(c, t), np.arctan(t.astype(np.float64))).max() <= 1.05


def test_atanh_core_within_one_ulp_to_one_half():
    c = G.parse()["kAtanhQ"]
    z = np.linspace(0.0, 0.5, 500_001, dtype=np.float32)[1:]
    assert _ulps(G.eval_f32(c, z), np.arctanh(z.astype(np.float64))).max() <= 1.0


def test_cores_reduce_to_the_taylor_series_at_small_arguments():
    # atan(t) = t - t^3/3 + ..., atanh(z) = z + z^3/3 + ...: the constant
    # term of Q is -1/3 and +1/3 to a few float32 ulp
    c = G.parse()
    assert abs(c["kAtanQ"][0] + 1.0 / 3.0) < 1e-5
    assert abs(c["kAtanhQ"][0] - 1.0 / 3.0) < 1e-6
    assert abs(c["kAtanhQ"][1] - 1.0 / 5.0) < 1e-3


def test_generator_reproduces_the_header():
    got = G.coefficients()
    ref = G.parse()
    assert set(got) == set(ref)
    for name in ref:
        a, b = got[name].astype(np.float64), ref[name].astype(np.float64)
        assert a.shape == b.shape
        # the same fit up to the least-squares solver's last bits
        assert np.all(np.abs(a - b) <= 4 * np.spacing(np.abs(b).astype(np.float32))), name


def test_half_pi_and_half_ln2_pairs():
    src = open(os.path.join(ROOT, "paper_1505_07674_gb300", "csrc", "lensed_sie_trig.cuh")).read()

    def const(name):
        tail = src.split(name + " = ")[1]
        return np.float32(float(tail.split("f")[0]))

    hp = np.float64(const("kHalfPiHi")) + np.float64(const("kHalfPiLo"))
    hl = np.float64(const("kHalfLn2Hi")) + np.float64(const("kHalfLn2Lo"))
    # each pair is exact to the rounding of its residual to float32
    assert abs(hp - np.pi / 2) <= np.spacing(np.float32(abs(const("kHalfPiLo"))))
    assert abs(hl - np.log(2.0) / 2) <= np.spacing(np.float32(abs(const("kHalfLn2Lo"))))
    assert const("kHalfPiHi") == np.float32(np.pi / 2)
    assert const("kHalfLn2Hi") == np.float32(np.log(2.0) / 2)


def test_header_is_its_own_rendering():
    # the committed header is exactly what the generator writes for the
    # coefficients it holds (templated over one ray or a pair of rays)
    path = os.path.join(ROOT, "paper_1505_07674_gb300", "csrc", "lensed_minimax.cuh")
    assert open(path).read() == G.render(G.parse())
