"""Failure paths of the library, provoked without any GPU fault.

  * Allocation failure: the test hook lensed_debug_fail_alloc makes the
    library's own allocator refuse device allocations (on the host, before
    cudaMalloc).  A model or network whose creation is refused at any of its
    allocations returns LENSED_E_NOMEM and gives back every byte it had
    taken; a batch whose scratch cannot be allocated returns LENSED_E_NOMEM
    and leaves the model usable, with the same results as before.
  * Expired device wait: lensed_mlp_debug_spin_limit(net, 0) lets the
    pipeline waits of the network's tensor-core products give up at once.
    The kernels then record the expiry, drain their own tensor-core work,
    free their tensor memory and return; lensed_mlp_get_params reports
    LENSED_E_TIMEOUT, and afterwards the device still serves both the
    network and the likelihood with unchanged results.
"""
import ctypes as C
import gc

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


@pytest.fixture
def inject():
    """The injection hook, with Python's cycle collector paused so that no
    model left over from an earlier test is freed while buffers are counted."""
    from paper_1505_07674_gb300 import _native as N
    gc.collect()
    gc.disable()
    try:
        yield N.lib().lensed_debug_fail_alloc
    finally:
        N.lib().lensed_debug_fail_alloc(-1)
        gc.enable()


def _live():
    """Device buffers the library holds (the hook's return value; -1 keeps
    the injection off)."""
    from paper_1505_07674_gb300 import _native as N
    torch.cuda.synchronize()
    return N.lib().lensed_debug_fail_alloc(-1)


@pytest.fixture(scope="module")
def c1():
    spec = W.c1_small()
    return spec, O.mock_observation(spec)


def test_refused_model_creation_frees_everything(c1, inject):
    from paper_1505_07674_gb300 import lensed as LZ
    from paper_1505_07674_gb300 import _native as N
    spec, obs = c1
    pts = W.draw_points(spec, 32, 5)
    # warm-up: load the library's kernels and module globals once
    m = LZ.Model(spec, obs, precision="mixed_ff")
    ref = m.loglike_batch(pts).cpu().numpy()
    m.close()
    base = _live()
    refused = 0
    for after in range(200):
        inject(after)
        try:
            m = LZ.Model(spec, obs, precision="mixed_ff")
        except N.LensedError as e:
            assert e.code == -2 and "injected" in str(e), str(e)
            assert _live() == base, (after, _live() - base)
            refused += 1
            continue
        break
    else:
        pytest.fail("creation never succeeded")
    inject(-1)
    assert refused >= 10  # every allocation of the creation was refused once
    got = m.loglike_batch(pts).cpu().numpy()
    assert np.array_equal(ref, got)
    assert _live() > base
    m.close()
    assert _live() == base


def test_refused_batch_scratch_leaves_model_usable(c1, inject):
    from paper_1505_07674_gb300 import lensed as LZ
    from paper_1505_07674_gb300 import _native as N
    spec, obs = c1
    m = LZ.Model(spec, obs, precision="mixed")
    small = W.draw_points(spec, 16, 6)
    a = m.loglike_batch(small).cpu().numpy()
    big = m.pack_params(W.draw_points(spec, 700, 7))  # more points than any earlier call
    out = torch.empty((1, 700), dtype=torch.float64, device="cuda")
    for after in range(4):
        inject(after)
        with pytest.raises(N.LensedError) as ei:
            m.loglike_batch(big, out=out)
        assert ei.value.code == -2
    inject(-1)
    # the model still works, at the old and at the new size
    assert np.array_equal(m.loglike_batch(small).cpu().numpy(), a)
    b = m.loglike_batch(big, out=out).cpu().numpy()
    fresh = LZ.Model(spec, obs, precision="mixed")
    assert np.array_equal(b, fresh.loglike_batch(big).cpu().numpy())
    m.close()
    fresh.close()


def test_refused_network_creation_frees_everything(inject):
    from paper_1505_07674_gb300 import _native as N
    L = N.lib()
    h = C.c_void_p()
    N.check_mlp(L.lensed_mlp_create(13, 256, 4096, C.byref(h)))
    L.lensed_mlp_destroy(h)
    base = _live()
    refused = 0
    for after in range(60):
        inject(after)
        h = C.c_void_p()
        rc = L.lensed_mlp_create(13, 256, 4096, C.byref(h))
        if rc == 0:
            break
        assert rc == -2 and not h.value
        assert _live() == base, after
        refused += 1
    inject(-1)
    assert rc == 0 and refused >= 20
    assert _live() > base
    L.lensed_mlp_destroy(h)
    assert _live() == base


def test_expired_tensor_core_wait_reports_timeout_and_device_stays_healthy(c1):
    from paper_1505_07674_gb300 import _native as N
    from paper_1505_07674_gb300.surrogate import Surrogate
    from paper_1505_07674_gb300.posterior import _init_params
    from paper_1505_07674_gb300 import lensed as LZ
    net = Surrogate(13, 256, 4096)
    theta = _init_params(13, 256, 1)
    net.set_params(theta)
    X = np.random.default_rng(2).standard_normal((1000, 13)).astype(np.float32)
    y_ref = net.forward(X).cpu().numpy()
    torch.cuda.synchronize()
    # the pipeline waits of the 256-wide layers now give up at once
    N.check_mlp(N.lib().lensed_mlp_debug_spin_limit(net._h, 0))
    net.forward(X)
    torch.cuda.synchronize()
    with pytest.raises(N.LensedError) as ei:
        net.get_params()
    assert ei.value.code == -5 and "expired" in str(ei.value)
    # back to the normal limit; set_params clears the record
    N.check_mlp(N.lib().lensed_mlp_debug_spin_limit(net._h, 1 << 30))
    net.set_params(theta)
    y = net.forward(X).cpu().numpy()
    assert np.array_equal(y, y_ref)
    assert np.array_equal(net.get_params(), theta)
    # and the likelihood on the same device
    spec, obs = c1
    m = LZ.Model(spec, obs, precision="mixed")
    pts = W.draw_points(spec, 8, 3)
    g = m.loglike_batch(pts).cpu().numpy()[0]
    o = O.OracleSystem(spec, obs).loglike(pts)
    assert np.all(np.abs(g - o) <= 1e-2)
    m.close()
    net.close()
