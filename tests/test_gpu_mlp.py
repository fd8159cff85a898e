"""Surrogate network on the GPU (BF16 tensor-core GEMMs) against the FP64
reference in oracle/mlp_oracle.py, element by element.

Tolerance, from the arithmetic: the CUDA network multiplies BF16 weights and
BF16 inputs exactly into FP32 accumulators, and rounds each hidden
activation (and, in the backward pass, each layer's output gradient) to BF16
(unit roundoff u = 2^-8) before the next product.  The reference runs in
FP64 on the same BF16-rounded weights and inputs, so the GPU's error in any
output comes only from those roundings, carried forward by the layers.  A
bound per element follows by propagating absolute values: with |.| applied
elementwise, an activation rounding adds u|h| to the error of h, a product
W h carries |W| times the error of h, and SiLU scales by at most
max|silu'| < 1.1.  The forward bound is computed that way for every output
(the FP32 accumulation adds far less); each gradient element is held to
c u G_abs, G_abs the same gradient formula evaluated on absolute values
(|dy|, |w|, |h|, |silu'|), with c = 8 for the roundings along the chain.
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


U = 2.0 ** -8
SILU_D = 1.1  # max |silu'(z)| = 1.0998...


def forward_error_bound(theta, Xb):
    """Per-output bound on |y_gpu - y_ref| from the BF16 roundings of h1, h2,
    h3, propagated with absolute values."""
    W1, b1, W2, b2, W3, b3, w4, b4 = M.unpack(theta, N_IN, H)
    _, (_, z1, h1, z2, h2, z3, h3) = M.forward(theta, Xb, N_IN, H, keep=True)
    e1 = U * np.abs(h1)                                   # h1 rounded
    e2 = SILU_D * (e1 @ np.abs(W2).T) + U * np.abs(h2)    # through W2, SiLU, rounded
    e3 = SILU_D * (e2 @ np.abs(W3).T) + U * np.abs(h3)
    return e3 @ np.abs(w4) + 1e-6 * (np.abs(h3) @ np.abs(w4))  # + FP32 accumulation


def test_forward_matches_reference_element_by_element():
    s, theta = make()
    X = np.random.default_rng(4).standard_normal((1000, N_IN))  # not a multiple of 64
    y = s.forward(X).cpu().numpy().astype(np.float64)
    th, Xb = rounded_weights(theta), bf16_round(X)
    ref = M.forward(th, Xb, N_IN, H)
    bound = forward_error_bound(th, Xb)
    err = np.abs(y - ref)
    k = int(np.argmax(err / bound))
    assert np.all(err <= bound), (k, y[k], ref[k], err[k], bound[k])
    # the bound is worst case; the errors themselves are far smaller
    assert rel_l2(y, ref) < 1e-2, rel_l2(y, ref)
    assert np.median(err / bound) < 0.1


def abs_gradient(theta, X, t):
    """The gradient formula of oracle/mlp_oracle.py with every factor
    replaced by its absolute value (the scale of each gradient element's
    rounding error)."""
    W1, b1, W2, b2, W3, b3, w4, b4 = M.unpack(theta, N_IN, H)
    y, (X, z1, h1, z2, h2, z3, h3) = M.forward(theta, X, N_IN, H, keep=True)
    B = X.shape[0]
    dy = np.abs(y - t) / B
    a3 = np.outer(dy, np.abs(w4)) * np.abs(M.silu_grad(z3))
    a2 = (a3 @ np.abs(W3)) * np.abs(M.silu_grad(z2))
    a1 = (a2 @ np.abs(W2)) * np.abs(M.silu_grad(z1))
    return np.concatenate([(a1.T @ np.abs(X)).ravel(), a1.sum(0), (a2.T @ np.abs(h1)).ravel(),
                           a2.sum(0), (a3.T @ np.abs(h2)).ravel(), a3.sum(0),
                           np.abs(h3).T @ dy, [dy.sum()]])


@pytest.mark.parametrize("B", [777, 8192])
def test_gradient_matches_reference_element_by_element(B):
    # 777 rows: 3 contraction ranges in the weight gradients; 8192: 32
    s, theta = make(seed=5, max_batch=8192)
    rng = np.random.default_rng(6)
    X = rng.standard_normal((B, N_IN))
    t = rng.standard_normal(B)
    loss, g = s.gradient(X, t)
    th, Xb = rounded_weights(theta), bf16_round(X)
    rl, rg = M.loss_and_grad(th, Xb, t, N_IN, H)
    assert abs(loss.item() - rl) < 3e-2 * rl
    g = g.cpu().numpy().astype(np.float64)
    bound = 8 * U * abs_gradient(th, Xb, t) + 1e-7
    err = np.abs(g - rg)
    k = int(np.argmax(err / bound))
    assert np.all(err <= bound), (k, g[k], rg[k], err[k], bound[k])
    o = 0
    for name, n in (("W1", H * N_IN), ("b1", H), ("W2", H * H), ("b2", H), ("W3", H * H),
                    ("b3", H), ("w4", H), ("b4", 1)):
        a, b = g[o:o + n], rg[o:o + n]
        if n > 1:
            assert rel_l2(a, b) < 5e-2, (name, rel_l2(a, b))
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
