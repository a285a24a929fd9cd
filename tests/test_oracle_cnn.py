"""Pins for oracle.cnn: a library correlation, finite-difference gradients,
the closed-form Adam step."""
import numpy as np
import pytest
from scipy import signal

from oracle import cnn


def test_single_channel_layer_is_correlate2d():
    rng = np.random.default_rng(0)
    X = rng.standard_normal((1, 7, 9, 1))
    W = rng.standard_normal((1, 3, 3, 1))
    Y = cnn.conv3x3(X, W, np.zeros(1))
    ref = signal.correlate2d(X[0, :, :, 0], W[0, :, :, 0], mode='same', boundary='fill')
    np.testing.assert_allclose(Y[0, :, :, 0], ref, atol=1e-13)


def _small_params(seed):
    rng = np.random.default_rng(seed)
    return [(rng.standard_normal(ws) * 0.2, rng.standard_normal(bs) * 0.1) for ws, bs in cnn.param_shapes()]


def test_gradients_match_finite_differences():
    rng = np.random.default_rng(1)
    params = _small_params(2)
    X = rng.standard_normal((2, 5, 6, 3))
    T = rng.standard_normal((2, 5, 6, 2))
    loss, grads = cnn.loss_and_grad(params, X, T)
    theta = cnn.flatten(params)
    g = cnn.flatten(grads)
    idx = rng.choice(theta.size, 40, replace=False)
    h = 1e-6
    for i in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        lp, _ = cnn.loss_and_grad(cnn.unflatten(tp), X, T)
        lm, _ = cnn.loss_and_grad(cnn.unflatten(tm), X, T)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])


def test_bf16_rounding():
    a = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -9, -3.14159, 0.0])
    r = cnn.bf16_round(a)
    assert r[0] == 1.0
    assert r[1] == 1.0                      # tie -> even mantissa
    assert r[2] == 1.0 + 2 ** -7            # rounds up
    assert abs(r[3] + 3.140625) < 1e-12


def test_adam_closed_form():
    theta = np.array([1.0, -2.0])
    g = np.array([0.5, -0.25])
    m = np.zeros(2)
    v = np.zeros(2)
    t1, m1, v1 = cnn.adam_step(theta, g, m, v, 1, lr=0.1)
    # first step: m_hat = g, v_hat = g^2 -> update = lr * sign(g) (up to eps)
    np.testing.assert_allclose(t1, theta - 0.1 * np.sign(g), atol=1e-7)
