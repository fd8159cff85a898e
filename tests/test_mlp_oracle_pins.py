"""Pins of the FP64 surrogate-network reference against what the mathematics
fixes: the SiLU closed form and its derivative, hand-computed outputs of tiny
networks, and the chain-rule gradient against central finite differences."""
import math

import numpy as np
import pytest

from oracle import mlp_oracle as M


def test_silu_and_derivative():
    for z in (-6.0, -1.3, 0.0, 0.4, 2.5, 9.0):
        assert abs(M.silu(z) - z / (1 + math.exp(-z))) < 1e-15
        h = 1e-6
        fd = (M.silu(z + h) - M.silu(z - h)) / (2 * h)
        assert abs(M.silu_grad(z) - fd) < 1e-9
    assert M.silu(0.0) == 0.0 and abs(M.silu_grad(0.0) - 0.5) < 1e-15


def test_zero_weights_give_the_output_bias():
    n_in, H = 3, 4
    th = np.zeros(M.n_params(n_in, H))
    th[-1] = 1.75
    y = M.forward(th, np.random.default_rng(0).random((5, n_in)), n_in, H)
    assert np.all(y == 1.75)


def test_hand_computed_one_unit_network():
    # H = 1: every layer is a scalar map; evaluate the chain by hand
    n_in, H = 2, 1
    W1, b1, W2, b2, W3, b3, w4, b4 = [0.5, -1.0], 0.1, 2.0, -0.3, 0.7, 0.2, 1.5, -0.4
    th = np.array(W1 + [b1, W2, b2, W3, b3, w4, b4])
    x = np.array([[1.2, 0.3]])
    s = lambda z: z / (1 + math.exp(-z))
    h1 = s(0.5 * 1.2 - 1.0 * 0.3 + 0.1)
    h2 = s(2.0 * h1 - 0.3)
    h3 = s(0.7 * h2 + 0.2)
    y = 1.5 * h3 - 0.4
    assert abs(M.forward(th, x, n_in, H)[0] - y) < 1e-15


@pytest.mark.parametrize("n_in,H,B", [(3, 5, 7), (18, 8, 4)])
def test_gradient_matches_finite_differences(n_in, H, B):
    rng = np.random.default_rng(1)
    th = M.init(n_in, H, 2) + 0.05 * rng.standard_normal(M.n_params(n_in, H))
    X = rng.standard_normal((B, n_in))
    t = rng.standard_normal(B)
    _, g = M.loss_and_grad(th, X, t, n_in, H)
    h = 1e-6
    idx = rng.choice(th.size, 40, replace=False)
    for k in idx:
        e = np.zeros_like(th)
        e[k] = h
        fd = (M.loss_and_grad(th + e, X, t, n_in, H)[0] -
              M.loss_and_grad(th - e, X, t, n_in, H)[0]) / (2 * h)
        assert abs(fd - g[k]) <= 1e-7 * max(1.0, abs(fd)), (k, fd, g[k])


def test_adam_first_step_moves_by_lr():
    # with bias correction the first step is lr * sign(g) (|g| >> eps)
    th = np.zeros(4)
    g = np.array([2.0, -0.5, 1e-3, -7.0])
    m, v = np.zeros(4), np.zeros(4)
    M.adam_step(th, g, m, v, 1, 0.01)
    assert np.allclose(th, -0.01 * np.sign(g), rtol=1e-4)


@pytest.mark.parametrize("seq", ["constant", "alternating", "random"])
def test_adam_matches_explicit_moment_sums_over_many_steps(seq):
    # Adam's moments after t steps are exponentially weighted sums of the
    # gradients, m_t = (1-b1) sum_i b1^(t-i) g_i and v_t = (1-b2) sum_i
    # b2^(t-i) g_i^2 (Kingma & Ba 2015, Sec. 3); the update uses them with
    # the bias corrections 1 - b^t.  Written out as sums here (not as the
    # reference's recurrence), over 12 steps, so a wrong decay, a swapped
    # b / 1-b or a missing correction at t > 1 shows.  A constant gradient
    # moves every step by lr sign(g) (m_t / (1-b1^t) = g, v_t / (1-b2^t) = g^2).
    b1, b2, eps, lr, T = 0.9, 0.999, 1e-8, 0.01, 12
    rng = np.random.default_rng(3)
    if seq == "constant":
        gs = [np.array([2.0, -0.5, 3e-3])] * T
    elif seq == "alternating":
        gs = [np.array([1.0, -2.0, 0.5]) * (-1) ** t for t in range(T)]
    else:
        gs = [rng.standard_normal(3) for _ in range(T)]
    th, m, v = np.zeros(3), np.zeros(3), np.zeros(3)
    expect = np.zeros(3)
    for t in range(1, T + 1):
        M.adam_step(th, gs[t - 1], m, v, t, lr)
        ms = (1 - b1) * sum(b1 ** (t - i) * gs[i - 1] for i in range(1, t + 1))
        vs = (1 - b2) * sum(b2 ** (t - i) * gs[i - 1] ** 2 for i in range(1, t + 1))
        expect -= lr * (ms / (1 - b1 ** t)) / (np.sqrt(vs / (1 - b2 ** t)) + eps)
        assert np.allclose(m, ms, rtol=1e-13, atol=0) and np.allclose(v, vs, rtol=1e-13, atol=0)
        assert np.allclose(th, expect, rtol=1e-12, atol=1e-15), (seq, t)
    if seq == "constant":
        assert np.allclose(th, -T * lr * np.sign(gs[0]), rtol=1e-4)
