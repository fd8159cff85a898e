"""The allocation-free entry point, lensed_loglike_batch_noalloc.

It exists for callers that cannot allocate device memory while they
evaluate -- a sampler inside a framework that has already reserved almost
all of the GPU's memory for its own pool, or a service with a device-memory
budget fixed at start-up.  Its scratch is a fixed 32 MiB array inside the
library.  These tests call it through the C ABI and check it against
lensed_loglike_batch on the same points, on two calls in a row (the second
call reuses the array the first one left behind), in every precision mode:
the two calls run the same kernels with the same fixed-order reductions, so
the results must be equal bit for bit (in MIXED_FF also when the model's
configuration hands the float-float re-traces to a second kernel, which
this call never does).  An oversized request must be refused with a clear
message.  This file is collected last.
"""
import ctypes as C

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


def _noalloc(m, params, out):
    from paper_1505_07674_gb300 import _native as N
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = N.lib().lensed_loglike_batch_noalloc(m._h, C.c_void_p(params.data_ptr()),
                                              params.shape[1], C.c_void_p(out.data_ptr()), stream)
    return rc, N.lib().lensed_last_error().decode()


@pytest.mark.parametrize("which,P,precision,config", [
    ("c1", 96, "fp32", None), ("c1", 96, "mixed", None), ("c1", 96, "fp64", None),
    ("c1", 96, "mixed_ff", None), ("c1", 96, "mixed_ff", 13),
    ("c2", 256, "mixed", None), ("c2", 256, "mixed_ff", 13), ("c2", 256, "mixed_ff", 19),
])
def test_noalloc_equals_batched_on_two_calls(which, P, precision, config):
    from paper_1505_07674_gb300 import lensed as LZ
    spec = W.c1_small() if which == "c1" else W.c2_hst()
    obs = O.mock_observation(spec)
    m = LZ.Model(spec, obs, precision=precision)
    if config is not None:
        # 13: trace blocks of 256, re-traces in a second kernel; 19: the same
        # with the persistent, work-queued trace launch
        m.set_config(config)
    pts = W.draw_points(spec, P, 99)
    pts[3, spec["param_names"].index("q_L")] = 1.5  # one point outside the domain
    params = m.pack_params(pts)
    ref = m.loglike_batch(params).cpu().numpy()
    assert np.isneginf(ref[0, 3]) and np.isfinite(ref).sum() == P - 1
    out = torch.full((1, P), 7.0, dtype=torch.float64, device="cuda")
    for _ in range(2):
        out.fill_(7.0)
        rc, msg = _noalloc(m, params, out)
        assert rc == 0, msg
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.array_equal(ref, got), (precision, np.nanmax(np.abs(ref - got)))
    m.close()


def test_noalloc_refuses_oversized_batch():
    from paper_1505_07674_gb300 import lensed as LZ
    spec = W.c2_hst()
    obs = O.mock_observation(spec)
    m = LZ.Model(spec, obs, precision="mixed")
    P = 40000  # the per-point scratch alone exceeds the fixed array
    params = torch.zeros((1, P, m.n_params_max), dtype=torch.float64, device="cuda")
    out = torch.zeros((1, P), dtype=torch.float64, device="cuda")
    rc, msg = _noalloc(m, params, out)
    assert rc == -1 and "fixed scratch" in msg and "points fit" in msg
    m.close()
