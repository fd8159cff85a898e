"""Plain FP64 reference of the log-likelihood surrogate network.

TEST INFRASTRUCTURE ONLY (like the rest of oracle/): the tests and the
benchmark's CPU legs use it to check the CUDA network's forward pass and
gradients.  It shares no code with the CUDA library.

The network (the surrogate the likelihood driver uses to pre-screen sampler
proposals; the paper has no such component):
    h1 = silu(x W1^T + b1),  h2 = silu(h1 W2^T + b2),  h3 = silu(h2 W3^T + b3),
    y  = h3 . w4 + b4,       silu(z) = z / (1 + exp(-z)),
with W_l stored [out][in].  Loss = mean over the batch of (y - t)^2 / 2.

Flat parameter order (the CUDA library uses the same one):
    W1 [H][n_in], b1 [H], W2 [H][H], b2 [H], W3 [H][H], b3 [H], w4 [H], b4 [1].
"""
from __future__ import annotations

import numpy as np


def n_params(n_in, H):
    return H * n_in + H + 2 * (H * H + H) + H + 1


def unpack(theta, n_in, H):
    theta = np.asarray(theta, dtype=np.float64)
    o = 0

    def take(shape):
        nonlocal o
        n = int(np.prod(shape))
        a = theta[o:o + n].reshape(shape)
        o += n
        return a

    W1 = take((H, n_in)); b1 = take((H,))
    W2 = take((H, H)); b2 = take((H,))
    W3 = take((H, H)); b3 = take((H,))
    w4 = take((H,)); b4 = take((1,))
    assert o == theta.size
    return W1, b1, W2, b2, W3, b3, w4, b4


def silu(z):
    return z / (1.0 + np.exp(-z))


def silu_grad(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def forward(theta, X, n_in, H, keep=False):
    W1, b1, W2, b2, W3, b3, w4, b4 = unpack(theta, n_in, H)
    X = np.asarray(X, dtype=np.float64)
    z1 = X @ W1.T + b1
    h1 = silu(z1)
    z2 = h1 @ W2.T + b2
    h2 = silu(z2)
    z3 = h2 @ W3.T + b3
    h3 = silu(z3)
    y = h3 @ w4 + b4[0]
    if keep:
        return y, (X, z1, h1, z2, h2, z3, h3)
    return y


def loss_and_grad(theta, X, t, n_in, H):
    """Loss mean((y - t)^2)/2 and its gradient, by the chain rule."""
    W1, b1, W2, b2, W3, b3, w4, b4 = unpack(theta, n_in, H)
    y, (X, z1, h1, z2, h2, z3, h3) = forward(theta, X, n_in, H, keep=True)
    B = X.shape[0]
    r = y - np.asarray(t, dtype=np.float64)
    loss = 0.5 * np.mean(r * r)
    dy = r / B
    gw4 = h3.T @ dy
    gb4 = np.array([dy.sum()])
    dz3 = np.outer(dy, w4) * silu_grad(z3)
    gW3 = dz3.T @ h2
    gb3 = dz3.sum(0)
    dz2 = (dz3 @ W3) * silu_grad(z2)
    gW2 = dz2.T @ h1
    gb2 = dz2.sum(0)
    dz1 = (dz2 @ W2) * silu_grad(z1)
    gW1 = dz1.T @ X
    gb1 = dz1.sum(0)
    g = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3.ravel(), gb3, gw4, gb4])
    return loss, g


def init(n_in, H, seed):
    """He-style initialisation (weights N(0, 2/fan_in), zero biases)."""
    rng = np.random.default_rng(seed)
    parts = [rng.standard_normal((H, n_in)) * np.sqrt(2.0 / n_in), np.zeros(H),
             rng.standard_normal((H, H)) * np.sqrt(2.0 / H), np.zeros(H),
             rng.standard_normal((H, H)) * np.sqrt(2.0 / H), np.zeros(H),
             rng.standard_normal(H) * np.sqrt(1.0 / H), np.zeros(1)]
    return np.concatenate([p.ravel() for p in parts])


def adam_step(theta, g, m, v, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba 2015), in place; returns theta."""
    m *= b1
    m += (1 - b1) * g
    v *= b2
    v += (1 - b2) * g * g
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    theta -= lr * mh / (np.sqrt(vh) + eps)
    return theta
