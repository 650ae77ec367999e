"""Pins of the FP64 surrogate-MLP oracle (CPU)."""
import math

import numpy as np
import pytest

from oracle import mlp_oracle as M


def _params(seed=0, scale=0.3):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(M.param_count()) * scale


def test_param_count_matches_the_architecture():
    assert M.param_count() == 5 * 128 + 128 + 128 * 128 + 128 + 128 * 128 + 128 + 128 * 4 + 4


def test_gelu_known_values():
    # Phi(1) = 0.841344746068543, so GELU(1) = Phi(1), GELU(-1) = -(1 - Phi(1))
    assert M.gelu(np.array([1.0]))[0] == pytest.approx(0.841344746068543, rel=1e-14)
    assert M.gelu(np.array([-1.0]))[0] == pytest.approx(-0.158655253931457, rel=1e-13)
    assert M.gelu(np.array([0.0]))[0] == 0.0
    x = np.linspace(-6, 6, 101)
    h = 1e-6
    np.testing.assert_allclose(M.gelu_grad(x), (M.gelu(x + h) - M.gelu(x - h)) / (2 * h),
                               rtol=1e-7, atol=1e-9)


def test_backprop_matches_finite_differences():
    rng = np.random.default_rng(1)
    theta = _params(1)
    x = rng.standard_normal((9, 5))
    t = rng.standard_normal((9, 4))
    L, g = M.loss_and_grad(theta, x, t)
    idx = rng.choice(theta.size, 40, replace=False)
    for i in idx:
        h = 1e-6
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        fd = (M.mse(M.forward(tp, x)[0], t) - M.mse(M.forward(tm, x)[0], t)) / (2 * h)
        # central differences in FP64 carry ~1e-9 absolute error here
        assert g[i] == pytest.approx(fd, rel=1e-4, abs=1e-8), i


def test_linear_limit_is_least_squares_gradient():
    """With one sample and only the output bias varying, dL/db = 2 (y - t) / 4."""
    theta = _params(2)
    x = np.ones((1, 5))
    t = np.zeros((1, 4))
    y, _ = M.forward(theta, x)
    _, g = M.loss_and_grad(theta, x, t)
    np.testing.assert_allclose(g[-4:], 2 * (y[0] - t[0]) / 4, rtol=1e-12)


def test_adam_first_step_is_signed_learning_rate():
    g = np.array([0.5, -2.0, 1e-3, 0.0])
    theta = np.zeros(4)
    new, m, v = M.adam_step(theta, g, np.zeros(4), np.zeros(4), 1, lr=0.01, eps=1e-12)
    # bias-corrected moments are g and g^2: the update is lr * g / |g|
    np.testing.assert_allclose(new[:3], -0.01 * np.sign(g[:3]), rtol=1e-9)
    assert new[3] == 0.0
    np.testing.assert_allclose(m, 0.1 * g)
    np.testing.assert_allclose(v, 0.001 * g * g)


def test_training_reduces_the_loss():
    rng = np.random.default_rng(3)
    theta = _params(3, scale=0.1)
    x = rng.standard_normal((64, 5))
    t = np.stack([np.tanh(x[:, 0]), x[:, 1] * 0.5, np.sin(x[:, 2]), x[:, 3] * x[:, 4] * 0.1], 1)
    m = np.zeros_like(theta)
    v = np.zeros_like(theta)
    L0, _ = M.loss_and_grad(theta, x, t)
    for k in range(1, 61):
        L, g = M.loss_and_grad(theta, x, t)
        theta, m, v = M.adam_step(theta, g, m, v, k, lr=3e-3)
    assert L < 0.5 * L0


def test_bf16_rounding():
    vals = np.array([1.0, 1.00390625, 1.005859375, -3.14159265], np.float32)
    r = M.bf16_round(vals)
    # bfloat16 keeps 8 significant bits: 1 + 2^-8 is a tie -> even (1.0),
    # 1.005859375 = 1 + 3*2^-9 rounds up to 1 + 2^-7
    assert r[0] == 1.0 and r[1] == 1.0 and r[2] == 1.0078125
    assert r[3] == pytest.approx(-3.140625)
    assert np.all(np.abs(r - vals) <= np.abs(vals) * 2.0 ** -8)
