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


class _NumpyEllipsoid:
    """A host-only bounded sampler for the hook: rejection from the live
    points' enlarged bounding ellipsoid (the GPU sampler's rule, here drawn
    with numpy), optionally with an exact pre-screen."""

    def __init__(self, f, d, enlarge=1.25, screen=False, seed=0):
        self.f, self.d, self.enlarge, self.screen = f, d, enlarge, screen
        self.rng = np.random.default_rng(seed)
        self.calls = self.exact = 0

    def __call__(self, live_u, live_l, lstar, k):
        self.calls += 1
        d = self.d
        c = live_u.mean(0)
        W = np.linalg.cholesky(np.cov(live_u.T) + 1e-12 * np.eye(d))
        z = np.linalg.solve(W, (live_u - c).T)
        L = W * math.sqrt((z * z).sum(0).max()) * self.enlarge
        acc_u, acc_l, n_exact, n_scr = [], [], 0, 0
        while len(acc_u) < k:
            g = self.rng.standard_normal((4096, d))
            r = self.rng.random(4096) ** (1.0 / d) / np.linalg.norm(g, axis=1)
            u = c + (g * r[:, None]) @ L.T
            u = u[np.all((u > 0) & (u < 1), axis=1)]
            ll = self.f(u)
            good = np.nonzero(ll > lstar)[0][:k - len(acc_u)]
            # candidates up to the last one needed count as evaluated
            used = good[-1] + 1 if len(good) == k - len(acc_u) else len(u)
            if self.screen:  # a perfect screen: only contour points are evaluated
                n_scr += int((ll[:used] <= lstar).sum())
                n_exact += int((ll[:used] > lstar).sum())
            else:
                n_exact += used
            acc_u.extend(u[good])
            acc_l.extend(ll[good])
        self.exact += n_exact
        return np.asarray(acc_u), np.asarray(acc_l), n_exact, n_scr


@pytest.mark.parametrize("screen", [False, True])
def test_bounded_hook_gives_the_closed_form_evidence(screen):
    # independent draws from a bounding ellipsoid replace the walks; the
    # Gaussian contours are ellipsoids, so the evidence must be unbiased, and
    # an exact screen can only lower the exact evaluations
    d, s = 4, 0.06
    mu = np.full(d, 0.5)
    f = gauss(mu, s)
    b = _NumpyEllipsoid(f, d, screen=screen, seed=4)
    res = nested_sampling(f, d, 300, seed=2, dlogz=0.05, bounded=b)
    exact = 0.5 * d * math.log(2 * math.pi * s * s)
    assert b.calls > 10
    assert abs(res["logz"] - exact) < 4 * res["logz_err"] + 0.05, (res["logz"], exact)
    assert np.allclose(res.posterior_mean(), mu, atol=4 * s / math.sqrt(300) + 0.01)
    walk = nested_sampling(f, d, 300, seed=2, dlogz=0.05)
    # rejection from a tight ellipsoid costs far fewer evaluations than the
    # 20-step walks
    assert res["n_evals"] < 0.5 * walk["n_evals"]
    if screen:
        assert res["n_prescreened"] > 0


def test_bounded_hook_partial_rounds_fall_back_to_walks():
    # a bounded sampler that offers only part of each round's replacements
    d, s = 3, 0.07
    mu = np.full(d, 0.4)
    f = gauss(mu, s)
    inner = _NumpyEllipsoid(f, d, seed=5)

    def half(live_u, live_l, lstar, k):
        u, l, e, n = inner(live_u, live_l, lstar, k // 2)
        return u, l, e, n

    res = nested_sampling(f, d, 200, seed=3, dlogz=0.05, bounded=half)
    exact = 0.5 * d * math.log(2 * math.pi * s * s)
    assert abs(res["logz"] - exact) < 4 * res["logz_err"] + 0.05
    assert 0.1 < res["accept"] < 0.9  # the walks ran for the other half
