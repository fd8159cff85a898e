"""Host nested-sampling driver for the batched likelihood.

Nested sampling (Skilling 2004, 2006) as the paper uses it through MultiNest
(Sec. 3.2): the evidence Z = integral of L(xi) P(xi) dxi (Eq. 13) is
accumulated over a shrinking sequence of likelihood contours while N live
points are replaced one at a time by prior draws constrained to lie above the
current worst likelihood.  The posterior (Eq. 12) is carried by the dead
points with weights w_i L_i / Z.

Parameters live in the unit hypercube (uniform box priors, as in the paper's
tests, Sec. 4.1).  Replacement points come from one bounding ellipsoid of the
live points (enlarged in volume), drawn in large batches so each batch is a
single batched GPU evaluation; a batch drawn for one threshold stays a valid
uniform proposal for every later (higher) threshold, so its candidates are
consumed in order while the threshold rises.  An optional pre-screen (the
surrogate network) may drop candidates before the exact evaluation; every
accepted point is judged by the exact likelihood.
"""
from __future__ import annotations

import heapq
import math
import time

import numpy as np


class Result(dict):
    """logz, logz_err, information, n_evals, n_iter, samples (dead + live, in
    the unit cube), logl, log weights (normalised), wall_s, and
    n_prescreened (candidates the pre-screen dropped)."""

    def posterior_mean(self):
        w = np.exp(self["logwt"] - self["logwt"].max())
        return (self["samples"] * w[:, None]).sum(0) / w.sum()


def _ellipsoid(points, enlarge):
    """Centre and Cholesky factor of the smallest scaled covariance ellipsoid
    enclosing the points, enlarged in volume by `enlarge`."""
    n, d = points.shape
    mean = points.mean(0)
    cov = np.cov(points.T) + 1e-12 * np.eye(d)
    inv = np.linalg.inv(cov)
    delta = points - mean
    r2 = np.einsum("ij,jk,ik->i", delta, inv, delta).max()
    scale = r2 * enlarge ** (2.0 / d)
    return mean, np.linalg.cholesky(cov * scale)


def _sample_ellipsoid(mean, chol, n, rng):
    d = mean.size
    z = rng.standard_normal((n, d))
    z /= np.linalg.norm(z, axis=1, keepdims=True)
    z *= rng.random((n, 1)) ** (1.0 / d)
    return mean + z @ chol.T


def nested_sampling(loglike, ndim, n_live, seed=0, dlogz=0.1, enlarge=2.0, batch_min=1024,
                    batch_max=65536, refit_frac=0.1, prescreen=None, max_evals=None,
                    callback=None):
    """Run nested sampling.

    loglike(U) -> logL for a float64 array U [B, ndim] in the unit cube (one
    batched evaluation).  prescreen(U, threshold) -> boolean mask of the
    candidates worth an exact evaluation (or None).  Stops when the live
    points can add at most dlogz to log Z."""
    rng = np.random.default_rng(seed)
    t0 = time.perf_counter()
    live_u = rng.random((n_live, ndim))
    live_l = np.asarray(loglike(live_u), dtype=np.float64)
    n_evals = n_live
    n_screened = 0
    heap = [(float(l), i) for i, l in enumerate(live_l)]
    heapq.heapify(heap)
    dead_u, dead_l, dead_logw = [], [], []
    logz, info, logx = -np.inf, 0.0, 0.0
    shrink = -1.0 / n_live
    eff = 1.0
    it = 0
    while True:
        # stop when the live points cannot move log Z by dlogz any more
        lmax = live_l.max()
        if np.isfinite(logz) and np.logaddexp(logz, lmax + logx) - logz < dlogz:
            break
        if max_evals is not None and n_evals >= max_evals:
            break
        mean, chol = _ellipsoid(live_u, enlarge)
        need = max(1, int(refit_frac * n_live))
        B = int(np.clip(1.5 * need / max(eff, 1e-4), batch_min, batch_max))
        cand = _sample_ellipsoid(mean, chol, B, rng)
        cand = cand[np.all((cand > 0.0) & (cand < 1.0), axis=1)]
        if prescreen is not None and len(cand):
            keep = np.asarray(prescreen(cand, heap[0][0]), dtype=bool)
            n_screened += int((~keep).sum())
            cand = cand[keep]
        if len(cand) == 0:
            eff = max(eff * 0.5, 1e-4)
            continue
        cand_l = np.asarray(loglike(cand), dtype=np.float64)
        n_evals += len(cand)
        # candidates above the current threshold, consumed in draw order
        accepted = 0
        for c in np.nonzero(cand_l > heap[0][0])[0]:
            lc = cand_l[c]
            if lc <= heap[0][0]:
                continue
            lw, iw = heap[0]
            # dead point: weight X_{i-1} - X_i with X_i = exp(-i / N)
            logw = logx + math.log1p(-math.exp(shrink))
            lwt = logw + lw
            new_logz = np.logaddexp(logz, lwt)
            info = (math.exp(lwt - new_logz) * lw + (math.exp(logz - new_logz) * (info + logz)
                                                    if np.isfinite(logz) else 0.0) - new_logz)
            logz = new_logz
            dead_u.append(live_u[iw].copy())
            dead_l.append(lw)
            dead_logw.append(logw)
            logx += shrink
            it += 1
            live_u[iw] = cand[c]
            live_l[iw] = lc
            heapq.heapreplace(heap, (float(lc), iw))
            accepted += 1
        eff = max(accepted / len(cand), 1e-4) if accepted else max(eff * 0.5, 1e-4)
        if callback:
            callback(it, n_evals, logz, heap[0][0])
    # the remaining live points share the final volume equally
    logw_live = logx - math.log(n_live)
    for i in range(n_live):
        lwt = logw_live + live_l[i]
        new_logz = np.logaddexp(logz, lwt)
        info = (math.exp(lwt - new_logz) * live_l[i] + math.exp(logz - new_logz) * (info + logz)
                - new_logz)
        logz = new_logz
    samples = np.vstack([np.asarray(dead_u).reshape(-1, ndim), live_u])
    logl = np.concatenate([np.asarray(dead_l), live_l])
    logw = np.concatenate([np.asarray(dead_logw), np.full(n_live, logw_live)])
    logwt = logw + logl - logz
    return Result(logz=float(logz), logz_err=float(math.sqrt(max(info, 0.0) / n_live)),
                  information=float(info), n_evals=int(n_evals), n_iter=it, samples=samples,
                  logl=logl, logwt=logwt, wall_s=time.perf_counter() - t0,
                  n_prescreened=n_screened)
