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


class GpuLikelihood:
    def __init__(self, model: Model, spec, record=False, pad_to=128):
        self.m = model
        self.lo = np.asarray(spec["prior_lo"], float)
        self.hi = np.asarray(spec["prior_hi"], float)
        self.ndim = len(self.lo)
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

    def __call__(self, U, threshold):
        t0 = time.perf_counter()
        y_thr = math.log1p(max(self.L_ref - threshold, 0.0))
        keep = self.predict_y(U) < y_thr + self.margin
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
                 window=150_000, min_pairs=20_000, steps=120, batch=8192, lr=1e-3,
                 margin_sigmas=3.0, max_rms=0.3, seed=0):
        self.rec = recorder
        self.ndim = ndim
        self.net = Surrogate(ndim, hidden, batch)
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

    def __call__(self, U, threshold):
        t0 = time.perf_counter()
        y_thr = math.log1p(max(self.L_ref - threshold, 0.0))
        pred = self.net.forward(self._x(U)).cpu().numpy().astype(np.float64)
        keep = pred * self.y_std + self.y_mean < y_thr + self.margin
        self.n_screen += len(U)
        self.screen_s += time.perf_counter() - t0
        return keep
