"""C ABI checks that need no GPU: the library builds and loads, exports every
entry point include/lensed.h declares, and rejects malformed descriptors
with a status code before it touches the device."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import paper_1505_07674_gb300 as pkg
from paper_1505_07674_gb300 import _native as N

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    pkg.build()
    return N.lib()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "lensed.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lensed_[a-z_0-9]+)\s*\(", src)))


def test_header_declarations_match_binding():
    assert declared_functions() == sorted(N.EXPORTS)


def test_library_exports_every_declared_symbol(L):
    for name in declared_functions():
        assert hasattr(L, name), name


def test_struct_layout_matches_header():
    # sizes the C compiler gives the structs of lensed.h, via a tiny probe
    import subprocess
    import tempfile
    src = r'''
#include <stdio.h>
#include <stddef.h>
#include "lensed.h"
int main(void){
 printf("%zu %zu %zu %zu %zu\n", sizeof(lensed_component), sizeof(lensed_system_desc),
        offsetof(lensed_system_desc, n_params), sizeof(lensed_model_info),
        offsetof(lensed_system_desc, components));
 return 0;}
'''
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "probe.c")
        open(c, "w").write(src)
        exe = os.path.join(d, "probe")
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()
    got = [C.sizeof(N.Component), C.sizeof(N.SystemDesc), N.SystemDesc.n_params.offset,
           C.sizeof(N.ModelInfo), N.SystemDesc.components.offset]
    assert [int(x) for x in out] == got


def test_enum_values_match_header():
    # every constant the binding passes through the ABI, against the header's
    import subprocess
    import tempfile
    names = {"LENSED_SIE": N.SIE, "LENSED_SHEAR": N.SHEAR, "LENSED_POINTMASS": N.POINTMASS,
             "LENSED_SERSIC": N.SERSIC, "LENSED_DEVAUC": N.DEVAUC, "LENSED_GAUSS": N.GAUSS,
             "LENSED_SKY": N.SKY, "LENSED_PLANE_LENS": N.PLANE_LENS,
             "LENSED_PLANE_FOREGROUND": N.PLANE_FOREGROUND,
             "LENSED_PLANE_SOURCE": N.PLANE_SOURCE,
             "LENSED_PLANE_SOURCE_IMAGE": N.PLANE_SOURCE_IMAGE,
             "LENSED_RULE_POINT": N.RULE_POINT, "LENSED_RULE_SUB": N.RULE_SUB,
             "LENSED_RULE_GL": N.RULE_GL, "LENSED_RULE_GK": N.RULE_GK,
             "LENSED_PREC_FP32": N.PREC_FP32, "LENSED_PREC_MIXED": N.PREC_MIXED,
             "LENSED_PREC_FP64": N.PREC_FP64, "LENSED_PREC_MIXED_FF": N.PREC_MIXED_FF,
             "LENSED_RENDER_UNCONVOLVED": N.RENDER_UNCONVOLVED,
             "LENSED_RENDER_CONVOLVED": N.RENDER_CONVOLVED,
             "LENSED_MAX_COMPONENT_PARAMS": N.MAX_COMPONENT_PARAMS,
             "LENSED_MAX_RULE_ORDER": N.MAX_RULE_ORDER,
             "LENSED_MAX_KRONROD_ORDER": N.MAX_KRONROD_ORDER}
    src = '#include <stdio.h>\n#include "lensed.h"\nint main(void){\n'
    src += "".join(f' printf("%d\\n", (int)({k}));\n' for k in names) + " return 0;}\n"
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "enums.c")
        open(c, "w").write(src)
        exe = os.path.join(d, "enums")
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()
    assert [int(x) for x in out] == list(names.values())


def _desc(nx=8, ny=8, psf=(3, 3), comps=None, n_params=2, data=None, variance=True, gain=0.0):
    keep = []
    d = N.SystemDesc()
    d.nx, d.ny, d.pixel_scale = nx, ny, 0.05
    a = np.ones(max(nx * ny, 1)) if data is None else np.asarray(data, float)
    keep.append(a)
    d.data = a.ctypes.data
    if variance:
        v = np.ones(max(nx * ny, 1))
        keep.append(v)
        d.variance = v.ctypes.data
    d.gain = gain
    if psf:
        f = np.ones(psf[0] * psf[1])
        keep.append(f)
        d.psf = f.ctypes.data
        d.psf_ny, d.psf_nx = psf
    d.rule, d.rule_order = N.RULE_GL, 3
    if comps is None:
        comps = [(N.SIE, N.PLANE_LENS, [0, 1, -1, -1, -1, -1]),
                 (N.SERSIC, N.PLANE_SOURCE, [-1] * 7)]
    ca = (N.Component * max(len(comps), 1))()
    for c, (t, pl, fi) in enumerate(comps):
        ca[c].type, ca[c].plane = t, pl
        for k in range(8):
            ca[c].free_index[k] = fi[k] if k < len(fi) else -1
            ca[c].value[k] = 0.5
    keep.append(ca)
    d.n_components = len(comps)
    d.components = C.cast(ca, C.c_void_p)
    d.n_params = n_params
    return d, keep


def _create(L, d, prec=N.PREC_MIXED):
    h = C.c_void_p()
    rc = L.lensed_create_model(C.byref(d), 1, prec, C.byref(h))
    return rc, L.lensed_last_error().decode()


@pytest.mark.parametrize("case,code", [
    ("even_psf", -1), ("zero_size", -1), ("no_components", -1),
    ("free_index_too_big", -1), ("mass_on_source_plane", -1), ("unknown_type", -1),
    ("nan_data", -4), ("zero_variance", -4), ("no_variance_no_gain", -1), ("bad_precision", -1),
    ("psf_too_big", -6), ("rule_order_zero", -1), ("nan_psf", -4),
])
def test_create_rejects_malformed(L, case, code):
    kw = {}
    if case == "even_psf":
        kw["psf"] = (3, 4)
    elif case == "zero_size":
        kw["nx"] = 0
    elif case == "no_components":
        kw["comps"] = []
    elif case == "free_index_too_big":
        kw["comps"] = [(N.SIE, N.PLANE_LENS, [5, -1, -1, -1, -1, -1])]
    elif case == "mass_on_source_plane":
        kw["comps"] = [(N.SIE, N.PLANE_SOURCE, [-1] * 6)]
    elif case == "unknown_type":
        kw["comps"] = [(42, N.PLANE_LENS, [-1] * 6)]
    elif case == "nan_data":
        dd = np.ones(64)
        dd[7] = np.nan
        kw["data"] = dd
    elif case == "zero_variance":
        kw["variance"] = False
        kw["gain"] = 1.0
        kw["data"] = np.zeros(64)  # (d + 0) / g = 0
    elif case == "no_variance_no_gain":
        kw["variance"] = False
    elif case == "psf_too_big":
        kw["psf"] = (33, 33)
    d, keep = _desc(**kw)
    if case == "rule_order_zero":
        d.rule_order = 0
    if case == "nan_psf":
        f = np.ones(9)
        f[4] = np.inf
        keep.append(f)
        d.psf = f.ctypes.data
    prec = 7 if case == "bad_precision" else N.PREC_MIXED
    rc, msg = _create(L, d, prec)
    assert rc == code, (rc, msg)
    assert msg


def test_null_arguments(L):
    h = C.c_void_p()
    assert L.lensed_create_model(None, 1, 1, C.byref(h)) == -1
    assert L.lensed_loglike_batch(None, None, 1, None, None) == -1
    assert L.lensed_render(None, 0, None, 0, None, None) == -1
    L.lensed_destroy(None)  # NULL-safe
