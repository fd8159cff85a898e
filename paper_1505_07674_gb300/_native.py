"""ctypes declarations of the C ABI in include/lensed.h.

Argument marshalling only: every step of the likelihood runs in the CUDA
library.  Loading fails loudly if the library has not been built.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_native", "liblensed_gb300.so")

LENSED_OK = 0
STATUS = {0: "LENSED_OK", -1: "LENSED_E_ARG", -2: "LENSED_E_NOMEM", -3: "LENSED_E_CUDA",
          -4: "LENSED_E_NONFINITE", -5: "LENSED_E_TIMEOUT", -6: "LENSED_E_UNSUPPORTED"}

SIE, SHEAR, POINTMASS, SERSIC, DEVAUC, GAUSS, SKY = 1, 2, 3, 4, 5, 6, 7
PLANE_LENS, PLANE_FOREGROUND, PLANE_SOURCE, PLANE_SOURCE_IMAGE = 0, 1, 2, 3
RULE_POINT, RULE_SUB, RULE_GL, RULE_GK = 0, 1, 2, 3
PREC_FP32, PREC_MIXED, PREC_FP64, PREC_MIXED_FF = 0, 1, 2, 3
RENDER_UNCONVOLVED, RENDER_CONVOLVED = 0, 1
MAX_COMPONENT_PARAMS = 8
MAX_RULE_ORDER = 16
MAX_KRONROD_ORDER = 7

# the C entry points, by name (the ABI symbol list the tests check)
EXPORTS = ("lensed_create_model", "lensed_destroy", "lensed_model_info_get", "lensed_render",
           "lensed_render_error", "lensed_rule_nodes", "lensed_set_config", "lensed_set_chunk_points",
           "lensed_measure_alu_peaks", "lensed_eval_sie_trig",
           "lensed_loglike_batch", "lensed_loglike_plain", "lensed_loglike_batch_host",
           "lensed_autotune", "lensed_tuned_config", "lensed_last_error", "lensed_batch_plan",
           "lensed_profile_batch", "lensed_loglike_batch_noalloc",
           "lensed_mlp_create", "lensed_mlp_destroy", "lensed_mlp_param_count",
           "lensed_mlp_set_params", "lensed_mlp_get_params", "lensed_mlp_forward",
           "lensed_mlp_gradient", "lensed_mlp_train_step", "lensed_mlp_last_error",
           "lensed_debug_fail_alloc", "lensed_debug_ff_queue_cap", "lensed_mlp_debug_spin_limit",
           "lensed_mlp_screen_ellipsoid")


class Component(C.Structure):
    _fields_ = [("type", C.c_int), ("plane", C.c_int),
                ("free_index", C.c_int * MAX_COMPONENT_PARAMS),
                ("value", C.c_double * MAX_COMPONENT_PARAMS)]


class SystemDesc(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("pixel_scale", C.c_double),
                ("data", C.c_void_p), ("variance", C.c_void_p),
                ("gain", C.c_double), ("offset", C.c_double),
                ("extra_weight", C.c_void_p), ("mask", C.c_void_p),
                ("psf", C.c_void_p), ("psf_nx", C.c_int), ("psf_ny", C.c_int),
                ("rule", C.c_int), ("rule_order", C.c_int), ("zeropoint", C.c_double),
                ("n_components", C.c_int), ("components", C.c_void_p), ("n_params", C.c_int)]


class ModelInfo(C.Structure):
    _fields_ = [("n_systems", C.c_int), ("n_params_max", C.c_int), ("precision", C.c_int),
                ("total_pixels", C.c_longlong), ("rays_per_eval_all", C.c_longlong),
                ("rays_per_eval_traced", C.c_longlong), ("psf_taps_per_eval", C.c_longlong),
                ("flops_per_ray", C.c_double), ("transcendentals_per_ray", C.c_double)]


class LensedError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


_lib = None


def lib():
    """The loaded library (raises if it is missing: there is no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"CUDA library not built: {LIB_PATH} is missing "
                               "(run __graft_entry__.build())")
        L = C.CDLL(LIB_PATH)
        vp, dp = C.c_void_p, C.POINTER(C.c_double)
        L.lensed_create_model.argtypes = [vp, C.c_int, C.c_int, C.POINTER(vp)]
        L.lensed_destroy.argtypes = [vp]
        L.lensed_destroy.restype = None
        L.lensed_model_info_get.argtypes = [vp, C.POINTER(ModelInfo)]
        L.lensed_render.argtypes = [vp, C.c_int, vp, C.c_int, vp, vp]
        L.lensed_render_error.argtypes = [vp, C.c_int, vp, vp, vp]
        L.lensed_rule_nodes.argtypes = [C.c_int, C.c_int, vp, vp, vp]
        L.lensed_set_config.argtypes = [vp, C.c_int]
        L.lensed_set_chunk_points.argtypes = [vp, C.c_int]
        L.lensed_measure_alu_peaks.argtypes = [C.POINTER(C.c_double), C.POINTER(C.c_double), vp]
        L.lensed_eval_sie_trig.argtypes = [vp, vp, C.c_longlong, vp, vp]
        for name in ("lensed_loglike_batch", "lensed_loglike_plain", "lensed_loglike_batch_host",
                     "lensed_loglike_batch_noalloc"):
            getattr(L, name).argtypes = [vp, vp, C.c_int, vp, vp]
        L.lensed_autotune.argtypes = [vp, vp, C.c_int, vp]
        L.lensed_tuned_config.argtypes = [vp, C.c_char_p, C.c_int]
        L.lensed_batch_plan.argtypes = [vp, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int)]
        L.lensed_profile_batch.argtypes = [vp, vp, C.c_int, vp, vp, dp, C.POINTER(C.c_int)]
        L.lensed_mlp_create.argtypes = [C.c_int, C.c_int, C.c_int, C.POINTER(vp)]
        L.lensed_mlp_destroy.argtypes = [vp]
        L.lensed_mlp_destroy.restype = None
        L.lensed_mlp_param_count.argtypes = [vp]
        L.lensed_mlp_param_count.restype = C.c_longlong
        L.lensed_mlp_set_params.argtypes = [vp, vp]
        L.lensed_mlp_get_params.argtypes = [vp, vp]
        L.lensed_mlp_forward.argtypes = [vp, vp, C.c_int, vp, vp]
        L.lensed_mlp_gradient.argtypes = [vp, vp, vp, C.c_int, vp, vp, vp]
        L.lensed_mlp_train_step.argtypes = [vp, vp, vp, C.c_int, C.c_float, vp, vp]
        L.lensed_mlp_screen_ellipsoid.argtypes = [vp, C.c_int, C.c_int, C.c_ulonglong,
                                                  C.c_ulonglong, vp, vp, vp, vp, vp, C.c_float,
                                                  vp, vp, vp, vp]
        L.lensed_debug_fail_alloc.argtypes = [C.c_longlong]
        L.lensed_debug_fail_alloc.restype = C.c_longlong
        L.lensed_debug_ff_queue_cap.argtypes = [vp, C.c_longlong]
        L.lensed_mlp_debug_spin_limit.argtypes = [vp, C.c_int]
        L.lensed_mlp_last_error.restype = C.c_char_p
        L.lensed_mlp_last_error.argtypes = []
        L.lensed_last_error.restype = C.c_char_p
        L.lensed_last_error.argtypes = []
        _lib = L
    return _lib


def check(rc):
    if rc != LENSED_OK:
        raise LensedError(rc, lib().lensed_last_error().decode())
    return rc


def check_mlp(rc):
    if rc != LENSED_OK:
        raise LensedError(rc, lib().lensed_mlp_last_error().decode())
    return rc
