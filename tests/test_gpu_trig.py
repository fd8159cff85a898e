"""The FP32 SIE's atan / atanh of a ratio on the GPU (Sec. 2.1, Eqs. 2-3).

lensed_eval_sie_trig runs the kernel's atan_ratio / atanh_ratio over device
arrays.  Their error against FP64 (of the exact quotient of the float inputs)
is held to a few units in the last place over the argument ranges the SIE
produces, next to CUDA's atanf / atanhf of the rounded quotient on the same
inputs.
"""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


def _run(n, d):
    from paper_1505_07674_gb300 import _native

    L = _native.lib()
    dev = torch.device("cuda:0")
    tn = torch.from_numpy(n.astype(np.float32)).to(dev)
    td = torch.from_numpy(d.astype(np.float32)).to(dev)
    out = torch.empty(4 * len(n), dtype=torch.float32, device=dev)
    rc = L.lensed_eval_sie_trig(C.c_void_p(tn.data_ptr()), C.c_void_p(td.data_ptr()),
                                C.c_longlong(len(n)), C.c_void_p(out.data_ptr()), None)
    assert rc == 0
    torch.cuda.synchronize()
    return out.cpu().numpy().reshape(4, len(n))


def _ulps(got, ref):
    tiny = np.float64(np.finfo(np.float32).tiny)
    return np.abs(got.astype(np.float64) - ref) / np.maximum(
        np.spacing(np.abs(ref).astype(np.float32)).astype(np.float64), tiny)


def _inputs(rng, count, ratio):
    d = np.float32(10.0 ** rng.uniform(-3, 2, count))
    r = ratio(rng, count)
    n = np.float32(r * d)
    return n, d


def test_atan_ratio_error():
    rng = np.random.default_rng(5)
    n, d = _inputs(rng, 2_000_000,
                   lambda g, k: g.choice([-1, 1], k) * 10.0 ** g.uniform(-6, 1.7, k))
    n[:4] = [0.0, 1.0, -1.0, 3.0]
    d[:4] = [0.0, 1.0, 1.0, 3.0]
    out = _run(n, d)
    ref = np.arctan2(n.astype(np.float64), d.astype(np.float64))
    mine, cuda = _ulps(out[0], ref), _ulps(out[2], ref)
    print(f"atan_ratio max {mine.max():.2f} ulp (atanf of the quotient {cuda.max():.2f})")
    assert out[0][0] == 0.0
    assert np.all(np.sign(out[0][1:]) == np.sign(n[1:]))
    assert mine.max() <= 3.0
    assert mine.mean() <= cuda.mean() + 0.5


def test_atanh_ratio_error():
    rng = np.random.default_rng(6)
    # |z| up to 0.995 (q down to 0.1); both branches, the switch at 1/2
    n, d = _inputs(rng, 2_000_000, lambda g, k: g.uniform(-0.995, 0.995, k))
    n[:3] = [0.0, 0.5, -0.5]
    d[:3] = [0.0, 1.0, 1.0]
    out = _run(n, d)
    z = n.astype(np.float64) / np.where(d > 0, d.astype(np.float64), 1.0)
    ref = np.arctanh(z)
    mine, cuda = _ulps(out[1], ref), _ulps(out[3], ref)
    small = np.abs(z) <= 0.5
    print(f"atanh_ratio max {mine[small].max():.2f} ulp (|z| <= 1/2), "
          f"{mine[~small].max():.2f} (beyond); atanhf of the quotient {cuda.max():.2f}")
    assert out[1][0] == 0.0
    assert np.all(np.sign(out[1][1:]) == np.sign(n[1:]))
    assert mine[small].max() <= 3.0
    assert mine[~small].max() <= 8.0
    assert mine.mean() <= cuda.mean() + 0.5
