"""Pins of the warm-start network oracle (oracle/mlp.py) against facts that do
not come from the oracle itself: a scalar network evaluated by hand with the
standard normal CDF, central finite differences of the loss, GELU's limits,
and the closed form of Adam's first step."""
import math

import numpy as np
import pytest

from oracle import mlp


def phi_cdf(z):
    return 0.5 * (1.0 + math.erf(z / math.sqrt(2.0)))


def test_gelu_limits_and_cdf_values():
    z = np.array([-30.0, -1.0, 0.0, 1.0, 30.0])
    g = mlp.gelu(z)
    assert g[0] == pytest.approx(0.0, abs=1e-12)
    assert g[2] == 0.0
    assert g[4] == pytest.approx(30.0, rel=1e-15)
    # Phi(1) = 0.8413447460685429 (standard normal table)
    assert g[3] == pytest.approx(0.8413447460685429, rel=1e-14)
    assert g[1] == pytest.approx(-1.0 * (1.0 - 0.8413447460685429), rel=1e-12)
    # the derivative by central differences
    h = 1e-6
    for zz in (-2.0, -0.3, 0.0, 0.7, 3.0):
        fd = (mlp.gelu(np.array(zz + h)) - mlp.gelu(np.array(zz - h))) / (2 * h)
        assert float(mlp.gelu_grad(np.array(zz))) == pytest.approx(float(fd), abs=1e-8)


def test_forward_scalar_network_by_hand():
    # n_in = n_hidden = n_out = 1: every layer is a scalar map
    W1, b1, W2, b2, W3, b3 = 2.0, 0.0, 1.0, -0.5, 3.0, 0.25
    x = 0.5
    z1 = W1 * x + b1                     # 1
    y1 = z1 * phi_cdf(z1)
    z2 = W2 * y1 + b2
    y2 = z2 * phi_cdf(z2)
    y = W3 * y2 + b3
    params = [np.array([[W1]]), np.array([b1]), np.array([[W2]]), np.array([b2]), np.array([[W3]]), np.array([b3])]
    out, _ = mlp.forward(params, np.array([[x]]))
    assert out[0, 0] == pytest.approx(y, rel=1e-14)
    # the projection clamps
    assert mlp.infer(params, np.array([[x]]), -0.1, 0.1)[0, 0] == pytest.approx(min(0.1, max(-0.1, y)))


def _rand_params(rng, n_in, n_h, n_out):
    return [rng.normal(0, 0.5, (n_h, n_in)), rng.normal(0, 0.1, n_h), rng.normal(0, 0.3, (n_h, n_h)),
            rng.normal(0, 0.1, n_h), rng.normal(0, 0.3, (n_out, n_h)), rng.normal(0, 0.1, n_out)]


def test_gradients_match_central_differences():
    rng = np.random.default_rng(5)
    n_in, n_h, n_out, B = 6, 5, 4, 7
    params = _rand_params(rng, n_in, n_h, n_out)
    X = rng.normal(size=(B, n_in))
    U = rng.normal(size=(B, n_out))
    grads, L = mlp.grad(params, X, U)
    assert L == pytest.approx(mlp.loss(params, X, U), rel=1e-15)
    h = 1e-6
    for k, p in enumerate(params):
        for idx in [tuple(rng.integers(0, s) for s in p.shape) for _ in range(6)]:
            pp = [q.copy() for q in params]
            pm = [q.copy() for q in params]
            pp[k][idx] += h
            pm[k][idx] -= h
            fd = (mlp.loss(pp, X, U) - mlp.loss(pm, X, U)) / (2 * h)
            assert grads[k][idx] == pytest.approx(fd, rel=1e-5, abs=1e-9), (k, idx)


def test_adam_first_step_closed_form():
    # after one step from zero moments, m_hat = g and v_hat = g^2, so each
    # parameter moves by lr g / (|g| + eps): lr sign(g) up to eps
    rng = np.random.default_rng(1)
    p = [rng.normal(size=(3, 4)), rng.normal(size=4)]
    g = [rng.normal(size=(3, 4)), np.array([0.0, 1e-3, -2.0, 5.0])]
    m = [np.zeros_like(a) for a in p]
    v = [np.zeros_like(a) for a in p]
    lr = 0.01
    q, m1, v1 = mlp.adam_step(p, g, m, v, 1, lr)
    for a, b, gg in zip(p, q, g):
        np.testing.assert_allclose(b, a - lr * gg / (np.abs(gg) + mlp.ADAM_EPS), rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(m1[1], 0.1 * g[1])
    np.testing.assert_allclose(v1[1], 0.001 * g[1] ** 2)


def test_planted_gradient_mistake_is_caught():
    """A dropped GELU' factor in the hidden layer must fail the difference check."""
    rng = np.random.default_rng(2)
    params = _rand_params(rng, 3, 4, 2)
    X = rng.normal(size=(5, 3))
    U = rng.normal(size=(5, 2))
    W1, b1, W2, b2, W3, b3 = params
    y, (Xc, z1, y1, z2, y2) = mlp.forward(params, X)
    g = 2.0 * (y - U) / U.size
    wrong_dW2 = (g @ W3).T @ y1              # GELU'(z2) left out
    h = 1e-6
    pp = [q.copy() for q in params]
    pm = [q.copy() for q in params]
    pp[2][1, 2] += h
    pm[2][1, 2] -= h
    fd = (mlp.loss(pp, X, U) - mlp.loss(pm, X, U)) / (2 * h)
    assert abs(wrong_dW2[1, 2] - fd) > 1e-4 * max(1.0, abs(fd))
    assert mlp.grad(params, X, U)[0][2][1, 2] == pytest.approx(fd, rel=1e-5, abs=1e-9)


def test_pack_unpack_roundtrip():
    rng = np.random.default_rng(3)
    params = _rand_params(rng, 4, 3, 2)
    flat = mlp.pack(params)
    back = mlp.unpack(flat, 4, 3, 2)
    for a, b in zip(params, back):
        np.testing.assert_array_equal(a, b)
