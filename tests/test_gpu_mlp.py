"""Surrogate network on the GPU (BF16 tensor-core GEMMs) against the FP64
reference in oracle/mlp_oracle.py.

Tolerance, from the arithmetic: the CUDA network rounds each weight matrix and
each of the hidden activations (and, in the backward pass, each output
gradient) to BF16 (unit roundoff 2^-8); accumulation is FP32.  Comparing with
the FP64 reference evaluated on the BF16-rounded weights, the relative L2
error of the outputs is a few 1e-3 and of the gradients below 1e-2; the
tests allow 3e-2 and 5e-2 (cosine >= 0.998).
"""
import numpy as np
import pytest

from oracle import mlp_oracle as M

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

N_IN, H = 18, 256


@pytest.fixture(scope="module", autouse=True)
def built():
    import paper_1505_07674_gb300 as pkg
    pkg.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def bf16_round(a):
    t = torch.as_tensor(np.asarray(a, np.float32)).to(torch.bfloat16).to(torch.float32)
    return t.numpy().astype(np.float64)


def rounded_weights(theta):
    """theta with W1, W2, W3 rounded to BF16 (as the GPU multiplies them)."""
    th = np.asarray(theta, np.float64).copy()
    o = 0
    for shape, is_w in (((H, N_IN), True), ((H,), False), ((H, H), True), ((H,), False),
                        ((H, H), True), ((H,), False), ((H,), False), ((1,), False)):
        n = int(np.prod(shape))
        if is_w:
            th[o:o + n] = bf16_round(th[o:o + n])
        o += n
    return th


def make(seed=3, max_batch=2048):
    from paper_1505_07674_gb300.surrogate import Surrogate
    s = Surrogate(N_IN, H, max_batch)
    theta = M.init(N_IN, H, seed).astype(np.float32)
    rng = np.random.default_rng(seed)
    theta[-(H + 1):] = rng.standard_normal(H + 1) * 0.1  # nonzero output layer
    s.set_params(theta)
    return s, theta.astype(np.float64)


def rel_l2(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_forward_matches_reference():
    s, theta = make()
    X = np.random.default_rng(4).standard_normal((1000, N_IN))  # not a multiple of 64
    y = s.forward(X).cpu().numpy()
    ref = M.forward(rounded_weights(theta), bf16_round(X), N_IN, H)
    assert rel_l2(y, ref) < 3e-2, rel_l2(y, ref)


def test_gradient_matches_reference():
    s, theta = make(seed=5)
    rng = np.random.default_rng(6)
    X = rng.standard_normal((777, N_IN))
    t = rng.standard_normal(777)
    loss, g = s.gradient(X, t)
    rl, rg = M.loss_and_grad(rounded_weights(theta), bf16_round(X), t, N_IN, H)
    assert abs(loss.item() - rl) < 3e-2 * rl
    g = g.cpu().numpy().astype(np.float64)
    o = 0
    for name, n in (("W1", H * N_IN), ("b1", H), ("W2", H * H), ("b2", H), ("W3", H * H),
                    ("b3", H), ("w4", H), ("b4", 1)):
        a, b = g[o:o + n], rg[o:o + n]
        if n > 1:
            cos = a @ b / (np.linalg.norm(a) * np.linalg.norm(b))
            assert rel_l2(a, b) < 5e-2 and cos > 0.998, (name, rel_l2(a, b), cos)
        else:
            assert abs(a[0] - b[0]) < 5e-2 * abs(b[0]) + 1e-6, (name, a, b)
        o += n


def test_training_reduces_loss_and_is_deterministic():
    rng = np.random.default_rng(7)
    X = rng.uniform(-1, 1, (4096, N_IN))
    t = np.sin(2 * X[:, 0]) + X[:, 1] * X[:, 2] + 0.5 * np.cos(3 * X[:, 3])
    runs = []
    for _ in range(2):
        s, _ = make(seed=8, max_batch=1024)
        Xd = torch.as_tensor(X, dtype=torch.float32, device="cuda")
        td = torch.as_tensor(t, dtype=torch.float32, device="cuda")
        losses = []
        for step in range(400):
            k = (step * 1024) % 4096
            losses.append(s.train_step(Xd[k:k + 1024], td[k:k + 1024], 1e-3).item())
        runs.append((losses, s.get_params()))
        s.close()
    losses = runs[0][0]
    assert np.mean(losses[-20:]) < 0.05 * np.mean(losses[:5]), (losses[:5], losses[-5:])
    assert np.array_equal(runs[0][1], runs[1][1])


def test_forward_in_slices_equals_whole():
    s, _ = make(seed=9, max_batch=256)
    X = np.random.default_rng(10).standard_normal((1000, N_IN))
    y_all = s.forward(X).cpu().numpy()
    y_parts = np.concatenate([s.forward(X[k:k + 200]).cpu().numpy() for k in range(0, 1000, 200)])
    assert np.array_equal(y_all, y_parts)
