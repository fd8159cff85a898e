"""Posterior runs: nested sampling driven by the batched GPU likelihood, with
the optional surrogate pre-screen.

``GpuLikelihood`` maps unit-cube points to the model's parameters (uniform
box priors) and evaluates them with one ``lensed_loglike_batch`` call per
batch; batch sizes are rounded up to a multiple of 128 (padding repeats the
first point) so the library's CUDA-graph cache sees a handful of shapes.

``SurrogateScreen`` trains the BF16 network once on (parameters, logL) pairs
from earlier exact evaluations and drops, before the exact evaluation,
candidates it predicts to lie far below the current threshold.
``OnlineSurrogate`` retrains it during the run, every few rounds, on the most
recent exact evaluations with the inputs whitened by the live points'
covariance, so the network models the likelihood locally (near the current
contour, where it is close to quadratic) to a few per cent.  The regression target is
y = log(1 + L_ref - logL) (L_ref the best logL in the training data), which
spreads the region near the top of the likelihood and compresses the far
tails; a candidate is kept when its prediction is within `margin` (a multiple
of the held-out residual scatter) of the threshold's y.  The exact likelihood
decides every candidate that passes.
"""
from __future__ import annotations

import math
import time

import numpy as np
import torch

from .lensed import Model
from .surrogate import Surrogate


def periodic_axes(spec):
    """Unit-cube axes whose parameter is an orientation with a 180-degree
    period over a [0, 180) prior (position angles, the shear angle): the
    likelihood repeats across the ends of their range."""
    names = spec.get("param_names") or []
    return [k for k, n in enumerate(names)
            if (n.startswith("pa") or n == "phi")
            and spec["prior_lo"][k] == 0.0 and spec["prior_hi"][k] == 180.0]


class GpuLikelihood:
    def __init__(self, model: Model, spec, record=False, pad_to=128):
        self.m = model
        self.lo = np.asarray(spec["prior_lo"], float)
        self.hi = np.asarray(spec["prior_hi"], float)
        self.ndim = len(self.lo)
        self.periodic = periodic_axes(spec)
        self.pad_to = pad_to
        self.cap = 0
        self.record = record
        self.U, self.L = [], []
        self.n_calls = 0
        self.seconds = 0.0

    def to_params(self, U):
        return self.lo + (self.hi - self.lo) * U

    def __call__(self, U):
        t0 = time.perf_counter()
        U = np.asarray(U, float)
        B = len(U)
        P = -(-B // self.pad_to) * self.pad_to
        if P > self.cap:
            self.params = torch.zeros((1, P, self.m.n_params_max), dtype=torch.float64,
                                      device="cuda")
            self.out = {}
            self.cap = P
        theta = self.to_params(U)
        host = np.empty((P, self.m.n_params_max))
        host[:B, :self.ndim] = theta
        host[B:, :self.ndim] = theta[0]
        p = self.params[:, :P]
        p[0].copy_(torch.from_numpy(host))
        if P not in self.out:
            self.out[P] = torch.empty((1, P), dtype=torch.float64, device="cuda")
        ll = self.m.loglike_batch(p, out=self.out[P])[0, :B].cpu().numpy()
        self.n_calls += 1
        self.seconds += time.perf_counter() - t0
        if self.record:
            self.U.append(U.copy())
            self.L.append(ll.copy())
        return ll


class SurrogateScreen:
    """Surrogate pre-screen for nested sampling (see the module docstring)."""

    def __init__(self, ndim, hidden=256, max_batch=8192):
        self.net = Surrogate(ndim, hidden, max_batch)
        self.ndim = ndim
        self.margin = None
        self.train_s = 0.0
        self.n_screen = 0
        self.screen_s = 0.0

    def _x(self, U):
        return (np.asarray(U, np.float32) - 0.5) * math.sqrt(12.0)

    def fit(self, U, L, epochs=20, batch=8192, lr=2e-3, seed=0, margin_sigmas=4.0,
            holdout=0.05):
        t0 = time.perf_counter()
        ok = np.isfinite(L)
        U, L = U[ok], L[ok]
        self.L_ref = float(L.max())
        y = np.log1p(self.L_ref - L)
        self.y_mean, self.y_std = float(y.mean()), float(y.std() + 1e-12)
        ys = (y - self.y_mean) / self.y_std
        rng = np.random.default_rng(seed)
        idx = rng.permutation(len(U))
        n_hold = max(1024, int(holdout * len(U)))
        hold, train = idx[:n_hold], idx[n_hold:]
        theta = _init_params(self.ndim, self.net.hidden, seed)
        self.net.set_params(theta)
        X = torch.as_tensor(self._x(U[train]), device="cuda")
        T = torch.as_tensor(ys[train].astype(np.float32), device="cuda")
        n = len(train)
        steps = max(1, epochs * n // batch)
        g = torch.Generator(device="cuda").manual_seed(seed)
        for s in range(steps):
            j = torch.randint(0, n, (batch,), device="cuda", generator=g)
            cur = lr * 0.5 * (1 + math.cos(math.pi * s / steps)) + 1e-5
            self.net.train_step(X[j], T[j], cur)
        torch.cuda.synchronize()
        pred = self.predict_y(U[hold])
        resid = pred - y[hold]
        self.val_rms = float(np.sqrt(np.mean(resid ** 2)))
        self.margin = margin_sigmas * self.val_rms
        self.train_s = time.perf_counter() - t0
        self.n_train = n
        return self

    def predict_y(self, U):
        out = self.net.forward(self._x(U)).cpu().numpy().astype(np.float64)
        return out * self.y_std + self.y_mean

    def on_round(self, live_u, live_l, threshold):
        """Calibration (pass as the sampler's on_round): the cut is raised to
        the highest prediction among the current live points, which all lie
        inside the contour (see OnlineSurrogate._calibrate)."""
        self.live_y_max = float(self.predict_y(live_u).max())

    def __call__(self, U, threshold):
        t0 = time.perf_counter()
        y_thr = math.log1p(max(self.L_ref - threshold, 0.0))
        cut = max(y_thr, getattr(self, "live_y_max", y_thr)) + self.margin
        keep = self.predict_y(U) < cut
        self.n_screen += len(U)
        self.screen_s += time.perf_counter() - t0
        return keep


def _init_params(n_in, H, seed):
    """He-style initial weights, zero biases (flat order of the C ABI)."""
    rng = np.random.default_rng(seed)
    parts = [rng.standard_normal((H, n_in)) * math.sqrt(2.0 / n_in), np.zeros(H),
             rng.standard_normal((H, H)) * math.sqrt(2.0 / H), np.zeros(H),
             rng.standard_normal((H, H)) * math.sqrt(2.0 / H), np.zeros(H),
             rng.standard_normal(H) * math.sqrt(1.0 / H), np.zeros(1)]
    return np.concatenate([p.ravel() for p in parts]).astype(np.float32)


class OnlineSurrogate:
    """Surrogate retrained during a nested-sampling run (see the module
    docstring).  Pass it as the sampler's `prescreen` and its `on_round` as
    the sampler's `on_round`; it reads the exact evaluations the recording
    likelihood keeps.  Inactive (the sampler then runs exact walks) until the
    first fit and whenever the held-out scatter exceeds `max_rms`."""

    def __init__(self, recorder: GpuLikelihood, ndim, hidden=256, retrain_every=12,
                 window=150_000, min_pairs=20_000, steps=400, batch=8192, lr=1e-3,
                 margin_sigmas=5.0, max_rms=0.3, seed=0, forward_batch=None):
        self.rec = recorder
        self.ndim = ndim
        # forward calls run in slices of the network's largest batch
        self.net = Surrogate(ndim, hidden, max(batch, forward_batch or batch))
        self.net.set_params(_init_params(ndim, hidden, seed))
        self.retrain_every, self.window, self.min_pairs = retrain_every, window, min_pairs
        self.steps, self.batch, self.lr = steps, batch, lr
        self.margin_sigmas, self.max_rms = margin_sigmas, max_rms
        self.rng = np.random.default_rng(seed)
        self.round = 0
        self.active = False
        self.fits = []
        self.train_s = 0.0
        self.screen_s = 0.0
        self.n_screen = 0

    def _x(self, U):
        return np.asarray(np.linalg.solve(self.W, (np.asarray(U) - self.c).T).T, np.float32)

    def on_round(self, live_u, live_l, threshold):
        self.round += 1
        if self.round % self.retrain_every != 1 and self.retrain_every > 1:
            self._calibrate(live_u)
            return
        # the most recent exact evaluations, at least `window` of them
        n, calls = 0, 0
        for u in reversed(self.rec.U):
            n += len(u)
            calls += 1
            if n >= self.window:
                break
        if n < self.min_pairs:
            return
        t0 = time.perf_counter()
        U = np.concatenate(self.rec.U[-calls:])
        L = np.concatenate(self.rec.L[-calls:])
        U, L = U[-self.window:], L[-self.window:]
        ok = np.isfinite(L)
        U, L = U[ok], L[ok]
        self.c = live_u.mean(0)
        self.W = np.linalg.cholesky(np.cov(live_u.T) + 1e-12 * np.eye(self.ndim))
        self.L_ref = float(max(live_l.max(), L.max()))
        y = np.log1p(self.L_ref - L)
        self.y_mean, self.y_std = float(y.mean()), float(y.std() + 1e-12)
        X = self._x(U)
        idx = self.rng.permutation(len(U))
        n_hold = max(2048, len(U) // 20)
        hold, train = idx[:n_hold], idx[n_hold:]
        Xd = torch.as_tensor(X[train], device="cuda")
        Td = torch.as_tensor(((y[train] - self.y_mean) / self.y_std).astype(np.float32),
                             device="cuda")
        n = len(train)
        g = torch.Generator(device="cuda").manual_seed(int(self.round))
        for s in range(self.steps):
            j = torch.randint(0, n, (self.batch,), device="cuda", generator=g)
            self.net.train_step(Xd[j], Td[j], self.lr * (0.5 * (1 + math.cos(math.pi * s / self.steps))) + 1e-5)
        pred = self.net.forward(X[hold]).cpu().numpy().astype(np.float64) * self.y_std + self.y_mean
        # scatter of the prediction near the current threshold
        y_thr = math.log1p(max(self.L_ref - threshold, 0.0))
        near = np.abs(y[hold] - y_thr) < 1.0
        resid = (pred - y[hold])[near] if near.sum() > 100 else (pred - y[hold])
        self.rms = float(np.sqrt(np.mean(resid ** 2)))
        self.margin = self.margin_sigmas * self.rms
        self.active = self.rms < self.max_rms
        self.train_s += time.perf_counter() - t0
        self.fits.append((self.round, len(U), self.rms, self.active))
        self._calibrate(live_u)

    def _calibrate(self, live_u):
        """The screen must let through every current live point (all lie
        inside the contour): its cut is raised to the highest prediction
        among them, so that the region it excludes holds (statistically)
        less than about 1/N of the contour, and every walk starts from a
        point the screen passes -- the condition under which rejecting a
        screened proposal without an exact evaluation leaves the walk's
        uniform target unchanged."""
        if not hasattr(self, "W"):
            return
        t0 = time.perf_counter()
        pred = self.net.forward(self._x(live_u)).cpu().numpy().astype(np.float64)
        self.live_y_max = float(pred.max() * self.y_std + self.y_mean)
        self.screen_s += time.perf_counter() - t0

    def cut_y(self, threshold, margin):
        """Largest predicted y = log(1 + L_ref - logL) a proposal may have to
        pass the screen at this threshold."""
        y_thr = math.log1p(max(self.L_ref - threshold, 0.0))
        return max(y_thr, getattr(self, "live_y_max", y_thr)) + margin

    def __call__(self, U, threshold):
        t0 = time.perf_counter()
        pred = self.net.forward(self._x(U)).cpu().numpy().astype(np.float64)
        keep = pred * self.y_std + self.y_mean < self.cut_y(threshold, self.margin)
        self.n_screen += len(U)
        self.screen_s += time.perf_counter() - t0
        return keep


class EllipsoidSampler:
    """Replacement draws for nested sampling by rejection from an enlarged
    bounding ellipsoid of the live points, with the surrogate network as a
    pre-screen (the `bounded` hook of sampler.nested_sampling).

    Each round: the ellipsoid is the live points' covariance scaled to their
    largest Mahalanobis radius times `enlarge`; batches of `batch` candidates
    are drawn uniformly inside it on the GPU (lensed_mlp_screen_ellipsoid);
    those outside the unit cube and, when the screen is active, those the
    network places clearly below the threshold (beyond the surrogate's
    margin) are dropped on the GPU; the survivors are evaluated exactly in
    candidate order and accepted iff L > L*, until the round's k
    replacements are found.  Accepted points are independent uniform draws of
    the part of the contour inside the ellipsoid and the screen's region --
    all of it when both contain the contour.  `audit` screened-out candidates
    per round (in-cube, chosen at random) are also evaluated exactly: any of
    them above the threshold is a screen error, counted in `missed` and
    answered by widening the margin.  Without a screen (screen=None) every
    in-cube candidate is evaluated exactly: the same sampler without the
    network.

    A round falls back to the random walks (returns None, or the points
    found so far) when the exact evaluations per accepted point exceed
    `walks` (the walk's cost per replacement), or after `max_batches`
    batches; after a fallback the ellipsoid is tried again `retry` rounds
    later."""

    def __init__(self, like: GpuLikelihood, ndim, screen=None, enlarge=1.25, batch=65536,
                 seed=0, walks=20, max_batches=256, audit=16, audit_batch=4096, retry=4,
                 margin_sigmas=4.0, periodic=None, max_margin=0.35):
        from .surrogate import ProposalScreen
        self.like, self.ndim, self.screen = like, ndim, screen
        self.periodic = list(like.periodic if periodic is None else periodic)
        self.enlarge, self.batch, self.seed = enlarge, batch, seed
        self.walks, self.max_batches, self.audit, self.retry = walks, max_batches, audit, retry
        self.audit_batch = min(audit_batch, batch)
        # exact-evaluation chunk sizes (a few shapes, so the likelihood's
        # graph cache keeps them all)
        self.ladder = [128, 256, 512, 1024, 2048, 4096]
        self.margin_sigmas, self.max_margin = margin_sigmas, max_margin
        self.log = []  # (round, screened, accepted, exact evaluations, candidates)
        self.ps = ProposalScreen(ndim, batch)
        self.counter = 0
        self.skip = 0
        self.rng = np.random.default_rng(seed + 1)
        self.rounds = self.rounds_used = 0
        self.n_exact = self.n_accept = self.n_candidates = 0
        self.n_audit = self.missed = self.n_screened = 0
        self.margin_boost = 1.0
        self.last_rate = 0.25
        self.draw_s = 0.0   # drawing and screening candidates
        self.round_s = 0.0  # whole rounds, exact evaluations included

    def _ellipsoid(self, live_u):
        """Center, scaled Cholesky factor and periodic-axis shift of the
        bounding ellipsoid: on each periodic axis the live points' widest
        circular gap is moved to the ends of the range first."""
        shift = np.zeros(self.ndim)
        for j in self.periodic:
            v = np.sort(live_u[:, j])
            gaps = np.diff(np.concatenate([v, [v[0] + 1.0]]))
            g = int(np.argmax(gaps))
            shift[j] = (v[g] + 0.5 * gaps[g]) % 1.0
        v = (live_u - shift) % 1.0
        c = v.mean(0)
        cov = np.cov(v.T) + 1e-12 * np.eye(self.ndim)
        W = np.linalg.cholesky(cov)
        z = np.linalg.solve(W, (v - c).T)
        r = math.sqrt(float((z * z).sum(0).max()))
        return c, W * (r * self.enlarge), shift

    def _screen_args(self, lstar):
        s = self.screen
        if s is None or not getattr(s, "active", False):
            return None, 0.0
        margin = self.margin_sigmas * s.rms * self.margin_boost
        cut = (s.cut_y(lstar, margin) - s.y_mean) / s.y_std
        return s.net, cut

    def __call__(self, live_u, live_l, lstar, k):
        self.rounds += 1
        if self.skip > 0:
            self.skip -= 1
            return None
        if self.screen is not None and not getattr(self.screen, "active", False):
            return None  # the walks run until the network is trained
        if self.screen is not None and self.margin_sigmas * self.screen.rms > self.max_margin:
            # too loose a screen: the region it lets through is many times
            # the contour's volume in this dimension, and the walks are cheaper
            return None
        t0 = time.perf_counter()
        c, L, shift = self._ellipsoid(live_u)
        self.ps.set_ellipsoid(c, L, shift)
        net, cut = self._screen_args(lstar)
        if net is not None:
            self.ps.set_whitening(self.screen.c, np.linalg.inv(self.screen.W))
        acc_u, acc_l = [], []
        n_exact = n_screened = 0
        rate = self.last_rate  # accepted per exact evaluation
        audit = np.zeros((0, self.ndim))
        if net is not None and self.audit:
            # a small batch of its own, drawn both ways: some of its
            # screened-out in-cube candidates are evaluated exactly with the
            # round's first chunk
            first = self.counter
            self.counter += self.audit_batch
            U_k, idx_k = self.ps.draw(self.seed, first, net, cut, n=self.audit_batch)
            U_in, idx_in = self.ps.draw(self.seed, first, n=self.audit_batch)
            out = U_in[~np.isin(idx_in, idx_k)]
            if len(out):
                audit = out[self.rng.choice(len(out), size=min(self.audit, len(out)),
                                            replace=False)]
            in_frac = len(U_in) / self.audit_batch
        else:
            in_frac = 1.0

        def too_costly():
            return n_exact >= 512 and n_exact > self.walks * max(len(acc_u), 1)

        def evaluate(chunk):
            nonlocal audit, n_exact
            a = len(audit)
            ll = self.like(np.concatenate([audit, chunk]) if a else chunk)
            n_exact += a + len(chunk)
            if a:
                self._audited(ll[:a], lstar)
                audit = audit[:0]
            return ll[a:]

        b = 0
        for b in range(self.max_batches):
            first = self.counter
            self.counter += self.batch
            t1 = time.perf_counter()
            U, idx = self.ps.draw(self.seed, first, net, cut)
            self.draw_s += time.perf_counter() - t1
            self.n_candidates += self.batch
            if net is not None:
                n_screened += max(0, int(round(self.batch * in_frac)) - len(U))
            pos = 0
            while pos < len(U) and len(acc_u) < k and not too_costly():
                need = k - len(acc_u)
                want = 1.2 * need / max(rate, 0.02)
                n = next((x for x in self.ladder if x >= want), self.ladder[-1])
                chunk = U[pos:pos + n]
                pos += len(chunk)
                ll = evaluate(chunk)
                good = np.nonzero(ll > lstar)[0][:need]
                acc_u.extend(chunk[good])
                acc_l.extend(ll[good])
                rate = max(len(acc_u), 1) / n_exact
            if len(acc_u) >= k or too_costly():
                break
        if len(audit):
            evaluate(np.zeros((0, self.ndim)))
        self.last_rate = rate
        self.round_s += time.perf_counter() - t0
        self.log.append((self.rounds, net is not None, len(acc_u), n_exact,
                         (b + 1) * self.batch))
        self.n_exact += n_exact
        self.n_accept += len(acc_u)
        self.n_screened += n_screened
        if len(acc_u) < k:
            self.skip = self.retry
        if not acc_u and n_exact == 0:
            return None
        self.rounds_used += 1
        return (np.asarray(acc_u).reshape(-1, self.ndim), np.asarray(acc_l), n_exact,
                n_screened)

    def _audited(self, ll, lstar):
        """Exact values of audited screened-out candidates: any above the
        threshold is a screen error, answered by a wider margin."""
        self.n_audit += len(ll)
        miss = int((ll > lstar).sum())
        if miss:
            self.missed += miss
            self.margin_boost *= 1.5
