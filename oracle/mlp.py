"""FP64 reference of the learned-tau network: forward, backward, pinball loss, Adam.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Network: x (65 = 64 histogram bins + log10 target error) -> Linear(65, 64) ->
GELU -> Linear(64, 64) -> GELU -> Linear(64, 1) -> y = log10(tau / (||A|| ||B||)).
GELU is the exact form 0.5 x (1 + erf(x / sqrt 2)).  Weights are stored
(out, in) row-major, as in y = W x + b.  Parameter order: W1, b1, W2, b2, W3, b3
(65*64 + 64 + 64*64 + 64 + 64 + 1 = 8449 values).
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf

SIZES = (65, 64, 64, 1)
N_PARAMS = sum(SIZES[i + 1] * SIZES[i] + SIZES[i + 1] for i in range(3))
_INV_SQRT2 = 1.0 / math.sqrt(2.0)
_INV_SQRT2PI = 1.0 / math.sqrt(2.0 * math.pi)


def gelu(z):
    return 0.5 * z * (1.0 + erf(z * _INV_SQRT2))


def gelu_grad(z):
    """d/dz [0.5 z (1 + erf(z/sqrt2))] = 0.5 (1 + erf(z/sqrt2)) + z phi(z)."""
    return 0.5 * (1.0 + erf(z * _INV_SQRT2)) + z * _INV_SQRT2PI * np.exp(-0.5 * z * z)


def unflatten(theta: np.ndarray, sizes=SIZES):
    """Split a flat parameter vector into [(W1, b1), (W2, b2), (W3, b3)]."""
    out, o = [], 0
    for i in range(len(sizes) - 1):
        fi, fo = sizes[i], sizes[i + 1]
        w = theta[o:o + fo * fi].reshape(fo, fi)
        o += fo * fi
        b = theta[o:o + fo]
        o += fo
        out.append((w, b))
    return out


def flatten(layers) -> np.ndarray:
    return np.concatenate([np.concatenate([w.ravel(), b.ravel()]) for w, b in layers])


def forward(theta: np.ndarray, x: np.ndarray, sizes=SIZES):
    """y[B] and the cache (inputs, pre-activations) for a batch x[B, in]."""
    layers = unflatten(np.asarray(theta, dtype=np.float64), sizes)
    h = np.asarray(x, dtype=np.float64)
    cache = []
    for li, (w, b) in enumerate(layers):
        z = h @ w.T + b
        cache.append((h, z))
        h = gelu(z) if li < len(layers) - 1 else z
    return h[:, 0], cache


def pinball_loss(y_pred, y_true, q: float) -> float:
    """mean rho_q(y_true - y_pred), rho_q(r) = max(q r, (q - 1) r)."""
    r = np.asarray(y_true, dtype=np.float64) - np.asarray(y_pred, dtype=np.float64)
    return float(np.mean(np.maximum(q * r, (q - 1.0) * r)))


def pinball_grad(y_pred, y_true, q: float) -> np.ndarray:
    """d loss / d y_pred; slope of rho_q is q for r > 0 and q - 1 for r <= 0."""
    r = np.asarray(y_true, dtype=np.float64) - np.asarray(y_pred, dtype=np.float64)
    slope = np.where(r > 0, q, q - 1.0)
    return -slope / r.size


def backward(theta: np.ndarray, cache, dy: np.ndarray, sizes=SIZES) -> np.ndarray:
    """Gradient of sum_b dy[b] * y[b] with respect to the flat parameters."""
    layers = unflatten(np.asarray(theta, dtype=np.float64), sizes)
    g = np.asarray(dy, dtype=np.float64)[:, None]          # d/d(output of last layer)
    grads = [None] * len(layers)
    for li in range(len(layers) - 1, -1, -1):
        h_in, z = cache[li]
        if li < len(layers) - 1:
            g = g * gelu_grad(z)                             # through the GELU
        w, _ = layers[li]
        grads[li] = (g.T @ h_in, g.sum(axis=0))
        g = g @ w
    return flatten(grads)


def loss_and_grad(theta, x, y_true, q: float, sizes=SIZES):
    y, cache = forward(theta, x, sizes)
    return pinball_loss(y, y_true, q), backward(theta, cache, pinball_grad(y, y_true, q), sizes)


def adam_step(theta, grad, m, v, t: int, lr: float, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (bias-corrected moments); returns new (theta, m, v)."""
    m = beta1 * m + (1.0 - beta1) * grad
    v = beta2 * v + (1.0 - beta2) * grad * grad
    mhat = m / (1.0 - beta1 ** t)
    vhat = v / (1.0 - beta2 ** t)
    return theta - lr * mhat / (np.sqrt(vhat) + eps), m, v


def finite_difference_grad(f, theta: np.ndarray, h: float = 1e-6) -> np.ndarray:
    """Central differences of a scalar function f(theta)."""
    g = np.zeros_like(theta, dtype=np.float64)
    for i in range(theta.size):
        tp = theta.copy()
        tm = theta.copy()
        tp[i] += h
        tm[i] -= h
        g[i] = (f(tp) - f(tm)) / (2 * h)
    return g
