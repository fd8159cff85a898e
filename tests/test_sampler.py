"""The nested-sampling driver against evidences known in closed form (CPU).

A Gaussian likelihood L = exp(-|u - mu|^2 / (2 s^2)) on the unit cube with a
uniform prior has Z = (2 pi s^2)^(d/2) (the Gaussian lies well inside the
cube) and posterior mean mu; the driver's log Z must land within a few of
its own error bars, and a pre-screen that only drops candidates below the
threshold must not change the answer."""
import math

import numpy as np
import pytest

from paper_1505_07674_gb300.sampler import nested_sampling


def gauss(mu, s):
    def f(U):
        d = U - mu
        return -0.5 * (d * d).sum(1) / (s * s)
    return f


@pytest.mark.parametrize("d,s,n_live", [(2, 0.05, 300), (5, 0.08, 400)])
def test_gaussian_evidence_and_mean(d, s, n_live):
    mu = np.full(d, 0.45)
    res = nested_sampling(gauss(mu, s), d, n_live, seed=1, dlogz=0.05)
    exact = 0.5 * d * math.log(2 * math.pi * s * s)
    assert abs(res["logz"] - exact) < 4 * res["logz_err"] + 0.05, (res["logz"], exact, res["logz_err"])
    assert np.allclose(res.posterior_mean(), mu, atol=4 * s / math.sqrt(n_live) + 0.01)
    # information of a Gaussian posterior under a unit-cube prior
    H = -0.5 * d * (math.log(2 * math.pi * s * s) + 1)
    assert abs(res["information"] - H) < 0.15 * H
    assert 0.1 < res["accept"] < 0.9


def test_prescreen_is_exact_and_saves_evaluations():
    mu, s, d = np.full(3, 0.6), 0.07, 3
    f = gauss(mu, s)
    plain = nested_sampling(f, d, 200, seed=3, dlogz=0.05)
    # an exact pre-screen (it rejects exactly the proposals the likelihood
    # rejects): the walks make the same moves, with fewer exact evaluations
    exact = nested_sampling(f, d, 200, seed=3, dlogz=0.05, prescreen=lambda U, thr: f(U) > thr)
    assert exact["logz"] == plain["logz"]
    assert exact["n_evals"] < plain["n_evals"] and exact["n_prescreened"] > 0
    # a looser pre-screen (region containing the contour) is still exact in
    # distribution: the evidence stays within its error
    loose = nested_sampling(f, d, 200, seed=4, dlogz=0.05,
                            prescreen=lambda U, thr: f(U) > thr - 2.0)
    truth = 0.5 * d * math.log(2 * math.pi * s * s)
    assert abs(loose["logz"] - truth) < 4 * loose["logz_err"] + 0.05
    assert loose["n_evals"] < plain["n_evals"]


def test_bimodal_evidence():
    # two separated Gaussians of equal mass: Z doubles (log Z + log 2)
    d, s = 2, 0.04
    a, b = np.array([0.25, 0.25]), np.array([0.75, 0.7])

    def f(U):
        la = -0.5 * ((U - a) ** 2).sum(1) / s ** 2
        lb = -0.5 * ((U - b) ** 2).sum(1) / s ** 2
        return np.logaddexp(la, lb)

    res = nested_sampling(f, d, 500, seed=5, dlogz=0.05)
    exact = 0.5 * d * math.log(2 * math.pi * s * s) + math.log(2.0)
    assert abs(res["logz"] - exact) < 4 * res["logz_err"] + 0.05
