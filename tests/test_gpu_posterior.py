"""Nested sampling driven by the batched GPU likelihood, with and without
the surrogate pre-screen, on the 64x64 workload (few live points, so it runs
in seconds).  The posterior must recover the truth; a pre-screen whose cut
every live point passes must reproduce the plain run exactly, skipping only
exact evaluations; the online pre-screen must skip a measurable share of
them, and wrongly almost never (an audit on the plain run's own walk)."""
import math

import numpy as np
import pytest

from oracle import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def built():
    import paper_1505_07674_gb300 as pkg
    pkg.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.fixture(scope="module")
def setup():
    from paper_1505_07674_gb300 import lensed as LZ
    spec = W.c1_small()
    obs = O.mock_observation(spec)
    return spec, LZ.Model(spec, obs, precision="mixed")


def test_posterior_recovers_truth(setup):
    from paper_1505_07674_gb300.posterior import GpuLikelihood
    from paper_1505_07674_gb300.sampler import nested_sampling
    spec, m = setup
    like = GpuLikelihood(m, spec)
    res = nested_sampling(like, like.ndim, 200, seed=3, dlogz=0.2)
    post = like.to_params(res.posterior_mean())
    sd = res.posterior_sd() * (like.hi - like.lo)
    truth = np.asarray(spec["truth"])
    names = spec["param_names"]
    for k in ("b_L", "q_L", "x_S", "r_S"):
        i = names.index(k)
        assert abs(post[i] - truth[i]) < 5 * sd[i] + 1e-3, (k, post[i], truth[i], sd[i])
    assert np.isfinite(res["logz"]) and res["logz_err"] > 0


def test_surrogate_trained_once_is_calibrated_and_changes_nothing(setup):
    # A network trained once on the exact evaluations of an earlier run
    # (another seed), its cut calibrated on every round's live points: with
    # the same seed as the plain run it must take exactly the plain run's
    # decisions, skipping only exact evaluations.  (Trained once over the
    # whole likelihood range, its held-out scatter near the late contours is
    # too large for the calibrated cut to screen much: the online network is
    # the one that saves evaluations.)
    from paper_1505_07674_gb300.posterior import GpuLikelihood, SurrogateScreen
    from paper_1505_07674_gb300.sampler import nested_sampling
    spec, m = setup
    rec = GpuLikelihood(m, spec, record=True)
    nested_sampling(rec, rec.ndim, 200, seed=5, dlogz=0.2)
    U, L = np.concatenate(rec.U), np.concatenate(rec.L)
    screen = SurrogateScreen(rec.ndim, 256, 4096).fit(U, L, epochs=30, batch=4096)
    a = nested_sampling(GpuLikelihood(m, spec), rec.ndim, 200, seed=7, dlogz=0.2)
    b = nested_sampling(GpuLikelihood(m, spec), rec.ndim, 200, seed=7, dlogz=0.2,
                        prescreen=screen, on_round=screen.on_round)
    assert screen.n_screen > 0
    assert b["n_evals"] + b["n_prescreened"] == a["n_evals"]
    assert b["logz"] == a["logz"] and b["n_iter"] == a["n_iter"]


def test_online_surrogate_saves_exact_evaluations_and_changes_nothing_else(setup):
    # The online network screens the walk proposals.  Its cut is calibrated
    # so that every live point passes it, plus a margin of held-out scatters;
    # a proposal it rejects is then outside the contour, where the exact
    # likelihood would have rejected it too.  So with the same seed the
    # screened run takes exactly the plain run's decisions: the same
    # iterations, samples and evidence, bit for bit, with exactly the
    # screened proposals' exact evaluations saved.  A single proposal inside
    # the contour that the screen wrongly rejected would change the walk and
    # break the equality.  (A margin of 8 scatters here; the production
    # margin of 5 is audited below.)
    from paper_1505_07674_gb300.posterior import GpuLikelihood, OnlineSurrogate
    from paper_1505_07674_gb300.sampler import nested_sampling
    spec, m = setup
    a = nested_sampling(GpuLikelihood(m, spec), 13, 200, seed=9, dlogz=0.2)
    rec = GpuLikelihood(m, spec, record=True)
    online = OnlineSurrogate(rec, 13, retrain_every=4, window=60_000, min_pairs=8_000,
                             batch=4096, forward_batch=65536, steps=400, margin_sigmas=8.0)
    b = nested_sampling(rec, 13, 200, seed=9, dlogz=0.2, prescreen=online,
                        on_round=online.on_round)
    assert any(f[3] for f in online.fits), online.fits
    assert b["n_prescreened"] > 0
    assert b["n_evals"] + b["n_prescreened"] == a["n_evals"], (a["n_evals"], b["n_evals"],
                                                               b["n_prescreened"])
    assert b["n_evals"] < a["n_evals"]
    assert b["n_iter"] == a["n_iter"] and b["logz"] == a["logz"]
    assert np.array_equal(b["samples"], a["samples"])


def test_online_surrogate_audit_at_the_production_margin(setup):
    # At the production margin (5 scatters) the screen is audited on the
    # plain run's own walk: every proposal is still evaluated exactly and
    # decides the walk, and the run counts the proposals the screen would
    # have skipped and those of them that lie inside the contour.  It must
    # skip at least 1 % of the exact evaluations, wrongly at most 1 in 200
    # of the proposals it drops; the screened run itself reaches the plain
    # run's evidence within its error.
    from paper_1505_07674_gb300.posterior import GpuLikelihood, OnlineSurrogate
    from paper_1505_07674_gb300.sampler import nested_sampling
    spec, m = setup
    a = nested_sampling(GpuLikelihood(m, spec), 13, 200, seed=9, dlogz=0.2)
    out = {}
    for audit in (True, False):
        rec = GpuLikelihood(m, spec, record=True)
        online = OnlineSurrogate(rec, 13, retrain_every=4, window=60_000, min_pairs=8_000,
                                 batch=4096, forward_batch=65536, steps=400)
        out[audit] = nested_sampling(rec, 13, 200, seed=9, dlogz=0.2, prescreen=online,
                                     on_round=online.on_round, audit_prescreen=audit)
    r = out[True]
    assert r["n_evals"] == a["n_evals"] and r["logz"] == a["logz"]  # the plain run itself
    assert r["n_prescreened"] >= 0.01 * a["n_evals"], (r["n_prescreened"], a["n_evals"])
    assert r["n_screen_false"] <= 0.005 * r["n_prescreened"], (r["n_screen_false"],
                                                                r["n_prescreened"])
    b = out[False]
    assert abs(a["logz"] - b["logz"]) < 4 * math.hypot(a["logz_err"], b["logz_err"]), (a["logz"], b["logz"])
