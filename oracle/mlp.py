"""The learned surrogate's network in plain FP64 NumPy (test infrastructure only).

A multilayer perceptron: layer l maps a[l-1] to z[l] = a[l-1] W_l^T + b_l with
W_l of shape (out, in), and a[l] = SiLU(z[l]) = z / (1 + e^{-z}) on hidden
layers, a[L] = z[L] on the output layer.  The loss is the mean squared error.
The backward pass applies the chain rule layer by layer; Adam (Kingma and Ba
2015) updates the parameters with bias-corrected first and second moments.

Pins (tests/test_oracle_mlp.py): every gradient against central finite
differences of the loss; SiLU's derivative against finite differences; Adam's
first step (moments equal to g and g^2 after bias correction, so the step is
lr * g / (|g| + eps) elementwise) and its response to a constant gradient.
"""
from __future__ import annotations

import numpy as np


def silu(z):
    return z / (1.0 + np.exp(-z))


def silu_grad(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def init(sizes, seed):
    """Weights ~ N(0, 2/in) (He), biases 0, float64; list of (W, b)."""
    rng = np.random.default_rng(seed)
    return [(rng.standard_normal((o, i)) * np.sqrt(2.0 / i), np.zeros(o))
            for i, o in zip(sizes[:-1], sizes[1:])]


def forward(params, x):
    """Returns (output, cache) with cache = list of (a_in, z) per layer."""
    a = np.asarray(x, dtype=np.float64)
    cache = []
    for l, (w, b) in enumerate(params):
        z = a @ w.T + b
        cache.append((a, z))
        a = z if l == len(params) - 1 else silu(z)
    return a, cache


def mse(y, t):
    e = np.asarray(y, dtype=np.float64) - np.asarray(t, dtype=np.float64)
    return float(np.mean(e * e)), 2.0 * e / e.size


def backward(params, cache, dy):
    """Gradients [(dW, db)] of the loss given dL/d(output) = dy."""
    grads = [None] * len(params)
    g = np.asarray(dy, dtype=np.float64)
    for l in range(len(params) - 1, -1, -1):
        a_in, z = cache[l]
        if l != len(params) - 1:
            g = g * silu_grad(z)
        w, _ = params[l]
        grads[l] = (g.T @ a_in, g.sum(axis=0))
        g = g @ w
    return grads


def adam(p, g, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step on arrays (returns new p, m, v)."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mh = m / (1.0 - beta1 ** step)
    vh = v / (1.0 - beta2 ** step)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v
