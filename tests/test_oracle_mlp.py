"""Pins for the surrogate network's oracle: gradients against finite differences,
SiLU's derivative, and Adam's special cases."""
import numpy as np

from oracle import mlp


def test_silu_and_its_derivative():
    z = np.linspace(-8, 8, 33)
    assert np.allclose(mlp.silu(z), z * 0.5 * (1 + np.tanh(z / 2)), rtol=1e-14, atol=1e-15)
    h = 1e-6
    fd = (mlp.silu(z + h) - mlp.silu(z - h)) / (2 * h)
    assert np.allclose(mlp.silu_grad(z), fd, rtol=1e-8, atol=1e-9)


def test_backward_matches_finite_differences():
    rng = np.random.default_rng(2)
    params = mlp.init([5, 7, 6, 1], seed=3)
    params = [(w, rng.standard_normal(b.shape) * 0.1) for w, b in params]
    x = rng.standard_normal((9, 5))
    t = rng.standard_normal((9, 1))
    y, cache = mlp.forward(params, x)
    loss, dy = mlp.mse(y, t)
    grads = mlp.backward(params, cache, dy)
    h = 1e-6
    for l, (w, b) in enumerate(params):
        for arr, gref in ((w, grads[l][0]), (b, grads[l][1])):
            for idx in list(np.ndindex(arr.shape))[:12]:
                old = arr[idx]
                arr[idx] = old + h
                lp = mlp.mse(mlp.forward(params, x)[0], t)[0]
                arr[idx] = old - h
                lm = mlp.mse(mlp.forward(params, x)[0], t)[0]
                arr[idx] = old
                assert abs((lp - lm) / (2 * h) - gref[idx]) < 1e-7 * (1 + abs(gref[idx]))


def test_adam_first_step_and_constant_gradient():
    g = np.array([0.3, -2.0, 1e-3])
    p, m, v = mlp.adam(np.zeros(3), g, np.zeros(3), np.zeros(3), 1, lr=0.01, eps=0.0)
    assert np.allclose(p, -0.01 * np.sign(g))
    # a constant gradient keeps the bias-corrected moments at g and g^2: every step is lr * sign(g)
    for step in range(2, 6):
        p2, m, v = mlp.adam(p, g, m, v, step, lr=0.01, eps=0.0)
        assert np.allclose(p2 - p, -0.01 * np.sign(g))
        p = p2
