"""Pins of the FP64 network reference: finite differences, the GELU closed form, Adam's first step."""
import math

import numpy as np
import pytest

from oracle import mlp


def test_gelu_known_values():
    x = np.array([-3.0, -1.0, 0.0, 0.5, 2.0])
    phi = 0.5 * (1 + np.array([math.erf(v / math.sqrt(2)) for v in x]))
    np.testing.assert_allclose(mlp.gelu(x), x * phi, rtol=0, atol=1e-15)
    assert mlp.gelu(np.array([0.0]))[0] == 0.0
    # symmetric identity of x Phi(x): gelu(x) - gelu(-x) = x
    np.testing.assert_allclose(mlp.gelu(x) - mlp.gelu(-x), x, atol=1e-14)


def test_gelu_grad_matches_difference_quotient():
    x = np.linspace(-4, 4, 41)
    h = 1e-6
    np.testing.assert_allclose(mlp.gelu_grad(x), (mlp.gelu(x + h) - mlp.gelu(x - h)) / (2 * h), rtol=1e-7, atol=1e-9)


def test_backward_matches_central_differences():
    rng = np.random.default_rng(3)
    p = mlp.init_params(1)
    x = rng.normal(size=(5, 32))
    t = rng.normal(size=(5, 3))
    w = np.array([1.0, 2.0, 0.5])
    g = mlp.backward(p, x, t, w)
    h = 1e-6
    for k in ("W1", "b1", "W2", "b2", "W3", "b3"):
        flat = p[k].ravel()
        for idx in rng.choice(flat.size, size=min(6, flat.size), replace=False):
            old = flat[idx]
            flat[idx] = old + h
            lp = mlp.loss(p, x, t, w)
            flat[idx] = old - h
            lm = mlp.loss(p, x, t, w)
            flat[idx] = old
            num = (lp - lm) / (2 * h)
            assert g[k].ravel()[idx] == pytest.approx(num, rel=1e-6, abs=1e-10), (k, idx)


def test_adam_first_step_is_signed_learning_rate():
    """With zero moments, the bias-corrected first step is -lr * g / (|g| + eps)."""
    p = {"W": np.array([1.0, -2.0, 3.0])}
    g = {"W": np.array([0.5, -1e-3, 0.0])}
    st = {}
    mlp.adam_step(p, g, st, lr=0.1, eps=1e-8)
    np.testing.assert_allclose(p["W"], [1.0 - 0.1 * 0.5 / (0.5 + 1e-8), -2.0 + 0.1 * 1e-3 / (1e-3 + 1e-8), 3.0])


def test_flatten_roundtrip_and_count():
    p = mlp.init_params(2)
    v = mlp.flatten(p)
    assert v.size == mlp.N_PARAMS == 32 * 128 + 128 + 128 * 128 + 128 + 128 * 3 + 3
    q = mlp.unflatten(v)
    for k in p:
        np.testing.assert_array_equal(p[k], q[k])
