"""Host nested-sampling driver for the batched likelihood.

Nested sampling (Skilling 2004, 2006) as the paper uses it through MultiNest
(Sec. 3.2): the evidence Z = integral of L(xi) P(xi) dxi (Eq. 13) is
accumulated over a shrinking sequence of likelihood contours while live
points are replaced by prior draws constrained to lie above the current
threshold.  The posterior (Eq. 12) is carried by the dead points with weights
w_i L_i / Z.

Parameters live in the unit hypercube (uniform box priors, as in the paper's
tests, Sec. 4.1).  Each round removes the k lowest of the N live points at
once: the j-th of them (j = 0..k-1) sits at expected log prior volume
log X - sum_{i<=j} 1/(N - i) (order statistics of N uniform volumes), which
sets its weight.  The k replacements come from k constrained random walks run
in lockstep -- each starts at a surviving live point and takes `walks`
Metropolis steps under the constraint L > L* (L* the highest removed
likelihood), with Gaussian steps shaped by the live points' covariance and a
scale adapted towards a 40 % acceptance -- so every step of all k walks is
one batched likelihood evaluation.

With a pre-screen (the surrogate network: prescreen(U, L*) says which
points it predicts above the threshold, with a safety margin) each walk step
is a two-stage (delayed-acceptance, Christen & Fox 2005) Metropolis step: a
proposal the pre-screen places outside is rejected without an exact
evaluation; one it lets through is evaluated exactly and accepted iff
L > L*.  For the uniform target on the contour this chain samples exactly the
part of the contour inside the pre-screen's region -- the whole contour when
the margin-enlarged region contains it -- and every accepted point is decided
by the exact likelihood; the saving is the exact evaluations of the rejected
proposals the pre-screen catches.
"""
from __future__ import annotations

import math
import time

import numpy as np


class Result(dict):
    """logz, logz_err, information, n_evals, n_iter, samples (dead + live, in
    the unit cube), logl, logwt (normalised log posterior weights), wall_s,
    n_prescreened (walk proposals the pre-screen rejected without an exact
    evaluation), accept (mean walk acceptance)."""

    def posterior_mean(self):
        w = np.exp(self["logwt"] - self["logwt"].max())
        return (self["samples"] * w[:, None]).sum(0) / w.sum()

    def posterior_sd(self):
        w = np.exp(self["logwt"] - self["logwt"].max())
        m = self.posterior_mean()
        return np.sqrt(((self["samples"] - m) ** 2 * w[:, None]).sum(0) / w.sum())


def nested_sampling(loglike, ndim, n_live, seed=0, dlogz=0.1, k_frac=0.25, walks=20,
                    prescreen=None, max_evals=None, callback=None, on_round=None,
                    bounded=None, accept_target=0.4, screened_accept_target=None,
                    audit_prescreen=False):
    """Run nested sampling.

    loglike(U) -> logL for a float64 array U [B, ndim] in the unit cube (one
    batched evaluation).  prescreen(U, threshold) -> boolean mask of the
    proposals worth an exact evaluation (or None); a pre-screen whose
    attribute `active` is False is skipped for that round.  on_round(live_u,
    live_l, threshold) is called before each round's replacements.
    bounded(live_u, live_l, threshold, k) -> (U [m], logL [m], exact
    evaluations, proposals screened out) or None: independent draws from the
    prior inside the contour L > threshold (m <= k of them) made some other
    way (e.g. rejection from a bounding region); the walks replace the rest.
    The walks' step scale adapts towards an acceptance of accept_target, or
    of screened_accept_target in rounds where a pre-screen is active: a
    proposal the screen rejects costs no exact evaluation, so larger steps
    (more rejections, farther moves) are cheap there.  With audit_prescreen
    the screen's verdicts are only recorded: every proposal is still
    evaluated exactly and decided by the exact value (the plain run), and
    n_prescreened / n_screen_false count the proposals the screen would
    have dropped and those of them that lie inside the contour.  Stops when
    the live points can add at most dlogz to log Z (or after max_evals
    evaluations)."""
    rng = np.random.default_rng(seed)
    t0 = time.perf_counter()
    N = n_live
    k = max(1, min(N - 1, int(round(k_frac * N))))
    live_u = rng.random((N, ndim))
    live_l = np.asarray(loglike(live_u), dtype=np.float64)
    n_evals, n_screened, n_prop, n_acc = N, 0, 0, 0
    n_false = 0
    dead_u, dead_l, dead_logw = [], [], []
    logz, info, logx = -np.inf, 0.0, 0.0
    scale = 1.0
    it = 0

    def add(logw, l):
        nonlocal logz, info
        lwt = logw + l
        new = np.logaddexp(logz, lwt)
        info = (math.exp(lwt - new) * l +
                (math.exp(logz - new) * (info + logz) if np.isfinite(logz) else 0.0) - new)
        logz = new

    while True:
        lmax = live_l.max()
        if np.isfinite(logz) and np.logaddexp(logz, lmax + logx) - logz < dlogz:
            break
        if max_evals is not None and n_evals >= max_evals:
            break
        order = np.argsort(live_l, kind="stable")
        gone, kept = order[:k], order[k:]
        lstar = live_l[gone[-1]]
        # the k removed points, lowest first, at their order-statistic volumes
        for j, i in enumerate(gone):
            step = -1.0 / (N - j)
            logw = logx + math.log1p(-math.exp(step))
            add(logw, live_l[i])
            dead_u.append(live_u[i].copy())
            dead_l.append(live_l[i])
            dead_logw.append(logw)
            logx += step
            it += 1
        if on_round is not None:
            on_round(live_u[kept], live_l[kept], lstar)
        # independent draws inside the contour, where a bounded sampler
        # offers them; constrained random walks for the rest
        n_b = 0
        if bounded is not None:
            got = bounded(live_u, live_l, lstar, k)
            if got is not None:
                bu, bl, be, bs = got
                n_b = len(bu)
                live_u[gone[:n_b]] = bu
                live_l[gone[:n_b]] = bl
                n_evals += be
                n_screened += bs
        if n_b == k:
            if callback:
                callback(it, n_evals, logz, lstar)
            continue
        gone = gone[n_b:]
        kw = len(gone)
        # kw constrained random walks from surviving points
        cov = np.cov(live_u[kept].T) + 1e-12 * np.eye(ndim)
        chol = np.linalg.cholesky(cov)
        screen = prescreen if (prescreen is not None and
                               getattr(prescreen, "active", True)) else None
        start = kept[rng.integers(0, len(kept), size=kw)]
        cu, cl = live_u[start].copy(), live_l[start].copy()
        for _ in range(walks):
            prop = cu + scale * rng.standard_normal((kw, ndim)) @ chol.T
            ok = np.all((prop > 0.0) & (prop < 1.0), axis=1)
            dropped = None
            if screen is not None and ok.any():
                idx = np.nonzero(ok)[0]
                keep = np.asarray(screen(prop[idx], lstar), dtype=bool)
                n_screened += int((~keep).sum())
                if audit_prescreen:
                    dropped = np.zeros(kw, dtype=bool)
                    dropped[idx[~keep]] = True
                else:
                    ok[idx[~keep]] = False
            acc = np.zeros(kw, dtype=bool)
            if ok.any():
                idx = np.nonzero(ok)[0]
                pl = np.asarray(loglike(prop[idx]), dtype=np.float64)
                n_evals += len(idx)
                good = pl > lstar
                if dropped is not None:
                    n_false += int((good & dropped[idx]).sum())
                acc[idx[good]] = True
                cu[idx[good]] = prop[idx[good]]
                cl[idx[good]] = pl[good]
            frac = acc.mean()
            n_prop += kw
            n_acc += int(acc.sum())
            target = (screened_accept_target if (screen is not None and
                                                 screened_accept_target is not None)
                      else accept_target)
            scale = min(max(scale * math.exp(frac - target), 1e-4), 10.0)
        live_u[gone] = cu
        live_l[gone] = cl
        if callback:
            callback(it, n_evals, logz, lstar)
    # the remaining live points share the final volume equally
    logw_live = logx - math.log(N)
    for i in range(N):
        add(logw_live, live_l[i])
    samples = np.vstack([np.asarray(dead_u).reshape(-1, ndim), live_u])
    logl = np.concatenate([np.asarray(dead_l), live_l])
    logw = np.concatenate([np.asarray(dead_logw), np.full(N, logw_live)])
    return Result(logz=float(logz), logz_err=float(math.sqrt(max(info, 0.0) / N)),
                  information=float(info), n_evals=int(n_evals), n_iter=it, samples=samples,
                  logl=logl, logwt=logw + logl - logz, wall_s=time.perf_counter() - t0,
                  n_prescreened=n_screened, n_screen_false=n_false,
                  accept=n_acc / max(n_prop, 1))
