"""Python front end of the CUDA likelihood library (argument marshalling only).

A model is built from one or more system specs (the dict layout of the
``workloads`` package: nx, ny, h, rule, psf, mask, zeropoint, components,
n_params) plus one observation per system (``data`` and either
``variance`` or ``gain``/``offset``).  Device memory and streams come from
PyTorch; every computation runs in the library's kernels.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import _native as N

_TYPES = {"sie": N.SIE, "shear": N.SHEAR, "pointmass": N.POINTMASS, "sersic": N.SERSIC,
          "devauc": N.DEVAUC, "gauss": N.GAUSS, "sky": N.SKY}
_PLANES = {"lens": N.PLANE_LENS, "foreground": N.PLANE_FOREGROUND, "source": N.PLANE_SOURCE,
           "source_image": N.PLANE_SOURCE_IMAGE}
_RULES = {"point": N.RULE_POINT, "sub": N.RULE_SUB, "gl": N.RULE_GL, "gk": N.RULE_GK}
_PREC = {"fp32": N.PREC_FP32, "mixed": N.PREC_MIXED, "fp64": N.PREC_FP64,
         "mixed_ff": N.PREC_MIXED_FF}


def _stream_handle(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


class Model:
    def __init__(self, specs, observations, precision="mixed_ff", extra_weights=None):
        if isinstance(specs, dict):
            specs = [specs]
            observations = [observations]
            extra_weights = [extra_weights]
        if extra_weights is None:
            extra_weights = [None] * len(specs)
        assert len(specs) == len(observations) == len(extra_weights)
        self.specs = specs
        self.precision = precision
        self._keep = []
        descs = (N.SystemDesc * len(specs))()
        comps_keep = []

        def arr(a, dtype=np.float64):
            if a is None:
                return None
            a = np.ascontiguousarray(np.asarray(a, dtype=dtype).reshape(-1))
            self._keep.append(a)
            return a.ctypes.data

        for s, (spec, obs, ex) in enumerate(zip(specs, observations, extra_weights)):
            d = descs[s]
            d.nx, d.ny, d.pixel_scale = spec["nx"], spec["ny"], spec["h"]
            d.data = arr(obs["data"])
            d.variance = arr(obs.get("variance"))
            d.gain = float(obs.get("gain", 0.0))
            d.offset = float(obs.get("offset", 0.0))
            d.extra_weight = arr(ex)
            d.mask = arr(spec.get("mask"), np.uint8)
            if spec.get("psf") is not None:
                psf = np.asarray(spec["psf"])
                d.psf = arr(psf)
                d.psf_ny, d.psf_nx = psf.shape
            rule, order = spec["rule"]
            d.rule, d.rule_order = _RULES[rule], int(order)
            d.zeropoint = float(spec.get("zeropoint", 0.0))
            cs = spec["components"]
            ca = (N.Component * len(cs))()
            for c, cd in enumerate(cs):
                ca[c].type = _TYPES[cd["type"]]
                ca[c].plane = _PLANES[cd["plane"]]
                for k in range(N.MAX_COMPONENT_PARAMS):
                    ca[c].free_index[k] = -1
                    ca[c].value[k] = 0.0
                for k, (kind, v) in enumerate(cd["params"]):
                    if kind == "free":
                        ca[c].free_index[k] = int(v)
                    else:
                        ca[c].value[k] = float(v)
            comps_keep.append(ca)
            d.n_components = len(cs)
            d.components = C.cast(ca, C.c_void_p)
            d.n_params = int(spec["n_params"])
        handle = C.c_void_p()
        N.check(N.lib().lensed_create_model(C.cast(descs, C.c_void_p), len(specs),
                                            _PREC[precision], C.byref(handle)))
        self._h = handle
        self._keep = []  # the library copied everything
        info = N.ModelInfo()
        N.check(N.lib().lensed_model_info_get(self._h, C.byref(info)))
        self.n_systems = info.n_systems
        self.n_params_max = info.n_params_max
        self.total_pixels = info.total_pixels
        self.rays_per_eval_all = info.rays_per_eval_all
        self.rays_per_eval_traced = info.rays_per_eval_traced
        self.psf_taps_per_eval = info.psf_taps_per_eval
        self.flops_per_ray = info.flops_per_ray
        self.transcendentals_per_ray = info.transcendentals_per_ray

    # -- lifetime
    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            N.lib().lensed_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- helpers
    def pack_params(self, params):
        """[P, n] (one system) or [n_sys, P, n] -> contiguous float64 CUDA
        tensor [n_sys, P, n_params_max] (zero padded)."""
        t = torch.as_tensor(params, dtype=torch.float64)
        if t.dim() == 2:
            t = t.unsqueeze(0)
        assert t.dim() == 3 and t.shape[0] == self.n_systems, t.shape
        if t.shape[2] < self.n_params_max:
            t = torch.nn.functional.pad(t, (0, self.n_params_max - t.shape[2]))
        return t.to("cuda").contiguous()

    # -- evaluation
    def render(self, system, params, convolved=True, out=None, stream=None):
        spec = self.specs[system]
        p = torch.as_tensor(params, dtype=torch.float64).to("cuda").contiguous()
        if out is None:
            out = torch.empty((spec["ny"], spec["nx"]), dtype=torch.float32, device="cuda")
        flags = N.RENDER_CONVOLVED if convolved else N.RENDER_UNCONVOLVED
        N.check(N.lib().lensed_render(self._h, system, C.c_void_p(p.data_ptr()), flags,
                                      C.c_void_p(out.data_ptr()), _stream_handle(stream)))
        self._last = p
        return out

    def render_error(self, system, params, out=None, stream=None):
        """Per-pixel Gauss-Kronrod error estimate |L_K - L_G| (unconvolved) of
        a system whose rule is ("gk", N)."""
        spec = self.specs[system]
        p = torch.as_tensor(params, dtype=torch.float64).to("cuda").contiguous()
        if out is None:
            out = torch.empty((spec["ny"], spec["nx"]), dtype=torch.float32, device="cuda")
        N.check(N.lib().lensed_render_error(self._h, system, C.c_void_p(p.data_ptr()),
                                            C.c_void_p(out.data_ptr()), _stream_handle(stream)))
        self._last = p
        return out

    def _loglike(self, fn, params, out, stream):
        if not (isinstance(params, torch.Tensor) and params.is_cuda and params.dtype == torch.float64
                and params.dim() == 3 and params.shape[2] == self.n_params_max
                and params.is_contiguous()):
            params = self.pack_params(params)
        P = params.shape[1]
        if out is None:
            out = torch.empty((self.n_systems, P), dtype=torch.float64, device="cuda")
        N.check(fn(self._h, C.c_void_p(params.data_ptr()), P, C.c_void_p(out.data_ptr()),
                   _stream_handle(stream)))
        self._last = params
        return out

    def loglike_batch(self, params, out=None, stream=None):
        return self._loglike(N.lib().lensed_loglike_batch, params, out, stream)

    def loglike_batch_noalloc(self, params, out=None, stream=None):
        """loglike_batch without any device allocation by the library (its
        scratch is a fixed array inside the library; see include/lensed.h).
        params and out must already be device tensors to allocate nothing
        on this side either."""
        return self._loglike(N.lib().lensed_loglike_batch_noalloc, params, out, stream)

    def loglike_plain(self, params, out=None, stream=None):
        return self._loglike(N.lib().lensed_loglike_plain, params, out, stream)

    def loglike_batch_host(self, params_host, out_host=None, stream=None):
        """params_host: float64 array [n_sys, P, n_params_max] in host memory
        (pinned for speed); returns / fills out_host [n_sys, P]."""
        if isinstance(params_host, torch.Tensor):
            assert params_host.device.type == "cpu" and params_host.dtype == torch.float64
            assert params_host.is_contiguous()
            P = params_host.shape[1]
            if out_host is None:
                out_host = torch.empty((self.n_systems, P), dtype=torch.float64)
            pptr, optr = params_host.data_ptr(), out_host.data_ptr()
        else:
            params_host = np.ascontiguousarray(params_host, dtype=np.float64)
            P = params_host.shape[1]
            if out_host is None:
                out_host = np.empty((self.n_systems, P))
            pptr, optr = params_host.ctypes.data, out_host.ctypes.data
        N.check(N.lib().lensed_loglike_batch_host(self._h, C.c_void_p(pptr), P, C.c_void_p(optr),
                                                  _stream_handle(stream)))
        return out_host

    def autotune(self, params, stream=None):
        params = self.pack_params(params) if not isinstance(params, torch.Tensor) else params
        N.check(N.lib().lensed_autotune(self._h, C.c_void_p(params.data_ptr()), params.shape[1],
                                        _stream_handle(stream)))
        return self.tuned_config()

    def batch_plan(self, P):
        """(kernel launches, points per scratch chunk) of one batched call."""
        n, c = C.c_int(), C.c_int()
        N.check(N.lib().lensed_batch_plan(self._h, P, C.byref(n), C.byref(c)))
        return n.value, c.value

    def profile_batch(self, params, out=None, stream=None):
        """One batched pass without the graph, timed per stage with CUDA
        events: returns ({stage: ms}, trace launches, loglike tensor)."""
        if not (isinstance(params, torch.Tensor) and params.is_cuda):
            params = self.pack_params(params)
        P = params.shape[1]
        if out is None:
            out = torch.empty((self.n_systems, P), dtype=torch.float64, device="cuda")
        ms = (C.c_double * 4)()
        nt = C.c_int()
        N.check(N.lib().lensed_profile_batch(self._h, C.c_void_p(params.data_ptr()), P,
                                             C.c_void_p(out.data_ptr()), _stream_handle(stream),
                                             ms, C.byref(nt)))
        names = ("prologue", "trace", "psf_chi2", "finalize")
        return {k: ms[i] for i, k in enumerate(names)}, nt.value, out

    def set_config(self, index):
        """Pin launch configuration `index` (-1: default); returns how many
        there are."""
        n = N.lib().lensed_set_config(self._h, int(index))
        N.check(min(n, 0))
        return n

    def set_chunk_points(self, points):
        """At most `points` points per scratch chunk of the batched schedule
        (0: as many as the scratch holds); never changes a result."""
        N.check(N.lib().lensed_set_chunk_points(self._h, int(points)))

    def tuned_config(self):
        buf = C.create_string_buffer(256)
        idx = N.lib().lensed_tuned_config(self._h, buf, 256)
        return idx, buf.value.decode()


def rule_nodes(rule, order):
    """The library's 1-D rule on the unit pixel for ("point"|"sub"|"gl"|"gk",
    order): offsets t, weights w and, for "gk", the embedded Gauss weights
    (zero on the Kronrod-only nodes; all zero for other rules).  Host only."""
    t = np.zeros(N.MAX_RULE_ORDER)
    w = np.zeros(N.MAX_RULE_ORDER)
    wg = np.zeros(N.MAX_RULE_ORDER)
    n = N.lib().lensed_rule_nodes(_RULES[rule], int(order), t.ctypes.data, w.ctypes.data,
                                  wg.ctypes.data)
    N.check(min(n, 0))
    return t[:n].copy(), w[:n].copy(), wg[:n].copy()



def measure_alu_peaks(stream=None):
    """(FP32 FMA TFLOP/s, MUFU ex2 Tops/s) measured on the current GPU."""
    a, b = C.c_double(), C.c_double()
    N.check(N.lib().lensed_measure_alu_peaks(C.byref(a), C.byref(b), _stream_handle(stream)))
    return a.value, b.value
