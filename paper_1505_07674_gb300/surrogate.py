"""Python front end of the surrogate network (argument marshalling only; the
network's forward, backward and Adam steps run in the CUDA library)."""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import _native as N


def _stream(stream):
    return C.c_void_p((stream or torch.cuda.current_stream()).cuda_stream)


class Surrogate:
    """MLP n_in -> H -> H -> H -> 1 with SiLU, BF16 tensor-core GEMMs."""

    def __init__(self, n_in, hidden=256, max_batch=8192):
        h = C.c_void_p()
        N.check_mlp(N.lib().lensed_mlp_create(n_in, hidden, max_batch, C.byref(h)))
        self._h = h
        self.n_in, self.hidden, self.max_batch = n_in, hidden, max_batch
        self.n_params = int(N.lib().lensed_mlp_param_count(h))
        self._loss = torch.zeros(1, dtype=torch.float32, device="cuda")

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            N.lib().lensed_mlp_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, theta):
        a = np.ascontiguousarray(theta, dtype=np.float32)
        assert a.size == self.n_params
        N.check_mlp(N.lib().lensed_mlp_set_params(self._h, C.c_void_p(a.ctypes.data)))

    def get_params(self):
        a = np.empty(self.n_params, dtype=np.float32)
        N.check_mlp(N.lib().lensed_mlp_get_params(self._h, C.c_void_p(a.ctypes.data)))
        return a

    @staticmethod
    def _dev(x):
        return torch.as_tensor(x, dtype=torch.float32).to("cuda").contiguous()

    def forward(self, X, out=None, stream=None):
        X = self._dev(X)
        B = X.shape[0]
        if out is None:
            out = torch.empty(B, dtype=torch.float32, device="cuda")
        N.check_mlp(N.lib().lensed_mlp_forward(self._h, C.c_void_p(X.data_ptr()), B,
                                               C.c_void_p(out.data_ptr()), _stream(stream)))
        self._keep = X
        return out

    def gradient(self, X, t, stream=None):
        X, t = self._dev(X), self._dev(t)
        g = torch.empty(self.n_params, dtype=torch.float32, device="cuda")
        N.check_mlp(N.lib().lensed_mlp_gradient(self._h, C.c_void_p(X.data_ptr()),
                                                C.c_void_p(t.data_ptr()), X.shape[0],
                                                C.c_void_p(g.data_ptr()),
                                                C.c_void_p(self._loss.data_ptr()),
                                                _stream(stream)))
        self._keep = (X, t)
        return self._loss.clone(), g

    def train_step(self, X, t, lr, stream=None):
        """One Adam step; returns the (device) loss before the step."""
        X, t = self._dev(X), self._dev(t)
        N.check_mlp(N.lib().lensed_mlp_train_step(self._h, C.c_void_p(X.data_ptr()),
                                                  C.c_void_p(t.data_ptr()), X.shape[0],
                                                  C.c_float(lr),
                                                  C.c_void_p(self._loss.data_ptr()),
                                                  _stream(stream)))
        self._keep = (X, t)
        return self._loss


class ProposalScreen:
    """Device buffers and marshalling for lensed_mlp_screen_ellipsoid: draws
    n candidates uniformly inside an ellipsoid of the unit cube (the
    library's counter-based generator), keeps those inside the cube and, with
    a network, those whose output is below the cut; returns the survivors in
    candidate order."""

    def __init__(self, ndim, n):
        self.d, self.n = ndim, n
        dev = dict(dtype=torch.float32, device="cuda")
        self.center = torch.zeros(ndim, **dev)
        self.chol = torch.zeros((ndim, ndim), **dev)
        self.shift = torch.zeros(ndim, **dev)
        self.xc = torch.zeros(ndim, **dev)
        self.xw = torch.zeros((ndim, ndim), **dev)
        self.u = torch.empty((n, ndim), dtype=torch.float64, device="cuda")
        self.idx = torch.empty(n, dtype=torch.int32, device="cuda")
        self.cnt = torch.zeros(1, dtype=torch.int32, device="cuda")

    def set_ellipsoid(self, center, chol, shift=None):
        """The ellipsoid in coordinates whose periodic axes are shifted by
        `shift` (zeros: none)."""
        self.center.copy_(torch.as_tensor(center, dtype=torch.float32))
        self.chol.copy_(torch.as_tensor(chol, dtype=torch.float32))
        self.shift.copy_(torch.as_tensor(np.zeros(self.d) if shift is None else shift,
                                         dtype=torch.float32))

    def set_whitening(self, x_center, x_whiten):
        self.xc.copy_(torch.as_tensor(x_center, dtype=torch.float32))
        self.xw.copy_(torch.as_tensor(x_whiten, dtype=torch.float32))

    def draw(self, seed, first, net=None, y_cut=0.0, n=None, stream=None):
        """(points [m][d] float64, candidate numbers [m]) of the survivors of
        candidates first .. first + n - 1 (n <= the batch size given at
        construction), ordered by candidate number."""
        n = self.n if n is None else n
        assert 0 <= n <= self.n
        h = net._h if net is not None else C.c_void_p()
        N.check_mlp(N.lib().lensed_mlp_screen_ellipsoid(
            h, self.d, n, C.c_ulonglong(seed), C.c_ulonglong(first),
            C.c_void_p(self.center.data_ptr()), C.c_void_p(self.chol.data_ptr()),
            C.c_void_p(self.shift.data_ptr()), C.c_void_p(self.xc.data_ptr()), C.c_void_p(self.xw.data_ptr()), C.c_float(y_cut),
            C.c_void_p(self.u.data_ptr()), C.c_void_p(self.idx.data_ptr()),
            C.c_void_p(self.cnt.data_ptr()), _stream(stream)))
        m = int(self.cnt.item())
        idx = self.idx[:m].cpu().numpy()
        u = self.u[:m].cpu().numpy()
        order = np.argsort(idx, kind="stable")
        return u[order], idx[order].astype(np.int64)
