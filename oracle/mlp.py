"""FP64 reference of the spectral-bound predictor network (test infrastructure).

TEST INFRASTRUCTURE: only the tests may import it; the library's kernels share nothing with it.

The network is a plain multilayer perceptron, 32 -> 128 -> 128 -> 3 with GELU activations
(GELU(x) = x Phi(x), Phi the standard normal CDF), trained on a mean-squared error with Adam
(Kingma & Ba 2015: first and second moment estimates with bias correction).  Everything below is
that definition written out; the gradients are the chain rule of the same expressions.
"""
from __future__ import annotations

import math

import numpy as np

SIZES = (32, 128, 128, 3)
SQRT2 = math.sqrt(2.0)


def _erf(x: np.ndarray) -> np.ndarray:
    return np.vectorize(math.erf)(x)


def gelu(x: np.ndarray) -> np.ndarray:
    return 0.5 * x * (1.0 + _erf(x / SQRT2))


def gelu_grad(x: np.ndarray) -> np.ndarray:
    """d/dx [x Phi(x)] = Phi(x) + x phi(x)."""
    phi = np.exp(-0.5 * x * x) / math.sqrt(2.0 * math.pi)
    return 0.5 * (1.0 + _erf(x / SQRT2)) + x * phi


def init_params(seed: int = 0) -> dict:
    """Uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights, zero biases."""
    rng = np.random.default_rng(seed)
    p = {}
    for i, (fi, fo) in enumerate(zip(SIZES[:-1], SIZES[1:]), start=1):
        lim = 1.0 / math.sqrt(fi)
        p[f"W{i}"] = rng.uniform(-lim, lim, size=(fo, fi))
        p[f"b{i}"] = np.zeros(fo)
    return p


def forward(p: dict, x: np.ndarray):
    """x: (B, 32).  Returns outputs (B, 3) and the intermediate values for backward."""
    h1 = x @ p["W1"].T + p["b1"]
    a1 = gelu(h1)
    h2 = a1 @ p["W2"].T + p["b2"]
    a2 = gelu(h2)
    y = a2 @ p["W3"].T + p["b3"]
    return y, (x, h1, a1, h2, a2)


def loss(p: dict, x: np.ndarray, t: np.ndarray, w: np.ndarray | None = None) -> float:
    """Mean over the batch of 1/2 sum_k w_k (y_k - t_k)^2."""
    y, _ = forward(p, x)
    w = np.ones(y.shape[1]) if w is None else np.asarray(w)
    return float(0.5 * np.mean(np.sum(w * (y - t) ** 2, axis=1)))


def backward(p: dict, x: np.ndarray, t: np.ndarray, w: np.ndarray | None = None) -> dict:
    """Gradients of `loss` with respect to every parameter."""
    y, (x, h1, a1, h2, a2) = forward(p, x)
    w = np.ones(y.shape[1]) if w is None else np.asarray(w)
    bsz = x.shape[0]
    dy = w * (y - t) / bsz
    g = {"W3": dy.T @ a2, "b3": dy.sum(0)}
    dh2 = (dy @ p["W3"]) * gelu_grad(h2)
    g["W2"] = dh2.T @ a1
    g["b2"] = dh2.sum(0)
    dh1 = (dh2 @ p["W2"]) * gelu_grad(h1)
    g["W1"] = dh1.T @ x
    g["b1"] = dh1.sum(0)
    return g


def adam_step(p: dict, g: dict, state: dict, lr: float = 1e-3, beta1: float = 0.9, beta2: float = 0.999,
              eps: float = 1e-8) -> None:
    """One Adam update in place; state holds m, v per parameter and the step count t."""
    state["t"] = state.get("t", 0) + 1
    t = state["t"]
    for k in p:
        m = state.setdefault("m_" + k, np.zeros_like(p[k]))
        v = state.setdefault("v_" + k, np.zeros_like(p[k]))
        m[:] = beta1 * m + (1 - beta1) * g[k]
        v[:] = beta2 * v + (1 - beta2) * g[k] ** 2
        mhat = m / (1 - beta1 ** t)
        vhat = v / (1 - beta2 ** t)
        p[k] -= lr * mhat / (np.sqrt(vhat) + eps)


def flatten(p: dict) -> np.ndarray:
    """Parameters in the library's order: W1, b1, W2, b2, W3, b3 (row-major weights)."""
    return np.concatenate([p[k].ravel() for k in ("W1", "b1", "W2", "b2", "W3", "b3")])


def unflatten(v: np.ndarray) -> dict:
    p, o = {}, 0
    for i, (fi, fo) in enumerate(zip(SIZES[:-1], SIZES[1:]), start=1):
        p[f"W{i}"] = np.asarray(v[o:o + fo * fi], np.float64).reshape(fo, fi)
        o += fo * fi
        p[f"b{i}"] = np.asarray(v[o:o + fo], np.float64)
        o += fo
    return p


N_PARAMS = sum(fo * fi + fo for fi, fo in zip(SIZES[:-1], SIZES[1:]))
