"""The library's integration rules (host side of the C ABI, no device needed)
against the oracle's independent construction and the published 15-point
Gauss-Kronrod table (Sec. 3.1 default rule; rule list of Sec. 4.5)."""
import numpy as np
import pytest

from oracle import oracle as O
from test_oracle_pins import G7K15_WK, G7K15_X


@pytest.fixture(scope="module")
def LZ():
    import paper_1505_07674_gb300 as pkg
    pkg.build()
    from paper_1505_07674_gb300 import lensed
    return lensed


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6, 7])
def test_kronrod_nodes_match_oracle(LZ, n):
    t, w, wg = LZ.rule_nodes("gk", n)
    x, wk, wgo = O.gauss_kronrod(n)
    assert len(t) == 2 * n + 1
    assert np.allclose(t, 0.5 * x, rtol=0, atol=2e-15)
    assert np.allclose(w, 0.5 * wk, rtol=0, atol=2e-15)
    assert np.allclose(wg, 0.5 * wgo, rtol=0, atol=2e-15)
    assert np.array_equal(wg == 0, wgo == 0)
    assert abs(w.sum() - 1) < 1e-15 and abs(wg.sum() - 1) < 1e-15


def test_g7k15_library_matches_published_table(LZ):
    t, w, _ = LZ.rule_nodes("gk", 7)
    assert np.allclose(2 * t[7:][::-1], G7K15_X, rtol=0, atol=5e-15)
    assert np.allclose(2 * w[7:][::-1], G7K15_WK, rtol=0, atol=5e-15)


@pytest.mark.parametrize("rule,order", [("gl", 1), ("gl", 5), ("gl", 16), ("sub", 4), ("point", 1)])
def test_other_rules_match_oracle(LZ, rule, order):
    t, w, wg = LZ.rule_nodes(rule, order)
    to, wo = O.rule_nodes(rule, order)
    assert np.allclose(t, to, rtol=0, atol=1e-15) and np.allclose(w, wo, rtol=0, atol=1e-15)
    assert np.all(wg == 0)


@pytest.mark.parametrize("rule,order", [("gk", 0), ("gk", 8), ("gl", 17), ("sub", 0)])
def test_rule_out_of_range_is_rejected(LZ, rule, order):
    from paper_1505_07674_gb300._native import LensedError
    with pytest.raises(LensedError):
        LZ.rule_nodes(rule, order)
