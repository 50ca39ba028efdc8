"""Oracle of the warm-start network (TEST INFRASTRUCTURE ONLY; same import
rules as the rest of ``oracle/``).

A plain FP64 numpy statement of the network the CUDA path trains:

    z1 = W1 x + b1,  y1 = GELU(z1)
    z2 = W2 y1 + b2, y2 = GELU(z2)
    y  = W3 y2 + b3                       (training output)
    u  = clamp(y, lo, hi)                 (inference output)
    L  = mean over the B x n_out entries of (y - u*)^2

with GELU(z) = z Phi(z) = z (1 + erf(z / sqrt 2)) / 2, its derivative
Phi(z) + z phi(z), the gradients by the chain rule written out layer by
layer, and Adam (bias-corrected first and second moments).  Rows of X are
samples.  Parameters travel as the list [W1, b1, W2, b2, W3, b3].

Parity unpinned: none -- ``tests/test_oracle_mlp.py`` pins the forward pass
on a hand-computed scalar network, the gradients by central finite
differences, GELU by its limits and the standard normal CDF, and Adam's first
step by its closed form.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf

ADAM_B1, ADAM_B2, ADAM_EPS = 0.9, 0.999, 1e-8


def gelu(z):
    return 0.5 * z * (1.0 + erf(z / math.sqrt(2.0)))


def gelu_grad(z):
    return 0.5 * (1.0 + erf(z / math.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)


def forward(params, X):
    """Returns (y, cache) for inputs X (B x n_in)."""
    W1, b1, W2, b2, W3, b3 = params
    z1 = X @ W1.T + b1
    y1 = gelu(z1)
    z2 = y1 @ W2.T + b2
    y2 = gelu(z2)
    y = y2 @ W3.T + b3
    return y, (X, z1, y1, z2, y2)


def infer(params, X, lo, hi):
    y, _ = forward(params, X)
    return np.clip(y, lo, hi)


def loss(params, X, U):
    y, _ = forward(params, X)
    return float(np.mean((y - U) ** 2))


def grad(params, X, U):
    """Gradients of loss() with respect to [W1, b1, W2, b2, W3, b3], and the loss."""
    W1, b1, W2, b2, W3, b3 = params
    y, (X, z1, y1, z2, y2) = forward(params, X)
    B, n_out = U.shape
    g = 2.0 * (y - U) / (B * n_out)          # dL/dy
    dW3 = g.T @ y2
    db3 = g.sum(axis=0)
    g2 = (g @ W3) * gelu_grad(z2)             # dL/dz2
    dW2 = g2.T @ y1
    db2 = g2.sum(axis=0)
    g1 = (g2 @ W2) * gelu_grad(z1)            # dL/dz1
    dW1 = g1.T @ X
    db1 = g1.sum(axis=0)
    return [dW1, db1, dW2, db2, dW3, db3], float(np.mean((y - U) ** 2))


def adam_step(params, grads, m, v, t, lr):
    """One Adam step (t counts steps including this one); returns new (params, m, v)."""
    out_p, out_m, out_v = [], [], []
    c1, c2 = 1.0 - ADAM_B1 ** t, 1.0 - ADAM_B2 ** t
    for p, g, mi, vi in zip(params, grads, m, v):
        mi = ADAM_B1 * mi + (1.0 - ADAM_B1) * g
        vi = ADAM_B2 * vi + (1.0 - ADAM_B2) * g * g
        out_p.append(p - lr * (mi / c1) / (np.sqrt(vi / c2) + ADAM_EPS))
        out_m.append(mi)
        out_v.append(vi)
    return out_p, out_m, out_v


def unpack(flat, n_in, n_hidden, n_out):
    """Split a flat parameter array (the library's exchange order) into matrices."""
    shapes = [(n_hidden, n_in), (n_hidden,), (n_hidden, n_hidden), (n_hidden,), (n_out, n_hidden), (n_out,)]
    out, q = [], 0
    for s in shapes:
        k = int(np.prod(s))
        out.append(np.asarray(flat[q:q + k], dtype=np.float64).reshape(s))
        q += k
    assert q == len(flat)
    return out


def pack(params):
    return np.concatenate([np.asarray(p, dtype=np.float64).ravel() for p in params])
