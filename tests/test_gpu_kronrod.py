"""Gauss-Kronrod rules on the GPU (g3k7 -- the paper's default --, g5k11,
g7k15; Sec. 3.1 and the rule list of Sec. 4.5) against the oracle: the
rendered images, the per-pixel embedded-Gauss error estimate and the
likelihood, through the C ABI.

The error map is |L_K - L_G| of two luminosities that each carry the image
tolerance (1e-5 |L| + 1e-5 max|L|), so it is compared at twice that
tolerance, scaled by the Kronrod image.
"""
import numpy as np
import pytest

from oracle import oracle as O
import workloads as W
from test_gpu_parity import assert_image_close, assert_loglike_close

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def built():
    import paper_1505_07674_gb300 as pkg
    pkg.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def lensed():
    from paper_1505_07674_gb300 import lensed as LZ
    return LZ


def gk_case(n):
    spec = W.c1_small()
    spec["rule"] = ("gk", n)
    obs = O.mock_observation(spec)
    return spec, obs, O.OracleSystem(spec, obs)


@pytest.mark.parametrize("n", [3, 5, 7])
@pytest.mark.parametrize("precision", ["fp32", "mixed", "mixed_ff", "fp64"])
def test_kronrod_render_and_error_map(n, precision):
    spec, obs, osys = gk_case(n)
    m = lensed().Model(spec, obs, precision=precision)
    pts = np.vstack([spec["truth"], W.draw_points(spec, 3, 21 + n)])
    for xi in pts:
        LK = osys.render(xi, convolved=False)
        assert_image_close(m.render(0, xi, convolved=False).cpu().numpy(), LK,
                           what=(n, precision, "L"))
        assert_image_close(m.render(0, xi, convolved=True).cpu().numpy(),
                           osys.render(xi, convolved=True), what=(n, precision, "L*"))
        e_gpu = m.render_error(0, xi).cpu().numpy().astype(float)
        e_ora = osys.render_error(xi)
        tol = 2 * (1e-5 * np.abs(LK) + 1e-5 * np.abs(LK).max())
        d = np.abs(e_gpu - e_ora)
        k = np.unravel_index(np.argmax(d - tol), d.shape)
        assert np.all(d <= tol), (n, precision, k, e_gpu[k], e_ora[k], tol[k])
        assert np.all(e_gpu >= 0)


# g3k7 has 7 nodes per row (MIXED_FF's queued re-trace), g5k11 and g7k15 have
# 11 and 15 (its in-place re-trace)
@pytest.mark.parametrize("n", [3, 5, 7])
@pytest.mark.parametrize("precision", ["fp32", "mixed", "mixed_ff", "fp64"])
def test_kronrod_loglike(n, precision):
    spec, obs, osys = gk_case(n)
    m = lensed().Model(spec, obs, precision=precision)
    pts = np.vstack([spec["truth"], W.draw_points(spec, 63, 31 + n)])
    g = m.loglike_batch(pts).cpu().numpy()[0]
    assert_loglike_close(g, osys.loglike(pts), 64 * 64, precision)
    assert np.array_equal(g, m.loglike_plain(pts).cpu().numpy()[0])


def test_error_map_needs_a_kronrod_rule():
    spec = W.c1_small()
    obs = O.mock_observation(spec)
    m = lensed().Model(spec, obs, precision="fp32")
    from paper_1505_07674_gb300._native import LensedError
    with pytest.raises(LensedError):
        m.render_error(0, spec["truth"])


def test_error_map_of_invalid_point_is_nan():
    spec, obs, osys = gk_case(3)
    m = lensed().Model(spec, obs, precision="mixed")
    xi = np.array(spec["truth"], float)
    xi[3] = 1.5  # axis ratio outside (0, 1]
    assert osys.render_error(xi) is None
    assert torch.isnan(m.render_error(0, xi)).all()
