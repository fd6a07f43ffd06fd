"""Pins of the network oracle (CPU): its hand-written gradient against
central finite differences; closed forms for special parameter vectors."""

import numpy as np

from oracle import mlp


def _rng_case(D=7, H=9, n=13, seed=0):
    rng = np.random.default_rng(seed)
    p = rng.uniform(-0.8, 0.8, mlp.param_count(D, H))
    X = rng.uniform(-1, 1, (n, D))
    t = rng.uniform(-1, 1, n)
    return p, X, t, D, H


def test_gradient_matches_central_differences():
    p, X, t, D, H = _rng_case()
    g = mlp.grad(p, X, t, D, H)
    h = 1e-6
    fd = np.empty_like(p)
    for i in range(p.size):
        e = np.zeros_like(p)
        e[i] = h
        fd[i] = (mlp.loss(p + e, X, t, D, H) - mlp.loss(p - e, X, t, D, H)) / (2 * h)
    assert np.max(np.abs(g - fd)) <= 1e-8 * max(1.0, np.max(np.abs(fd)))


def test_constant_network_closed_form():
    """With every weight zero the output is b3 and only b3 has a gradient:
    dL/db3 = 2 mean(b3 - t)."""
    D, H = 4, 5
    p = np.zeros(mlp.param_count(D, H))
    p[-1] = 0.25
    X = np.random.default_rng(1).uniform(-1, 1, (6, D))
    t = np.linspace(-1, 1, 6)
    assert np.allclose(mlp.forward(p, X, D, H), 0.25)
    g = mlp.grad(p, X, t, D, H)
    assert np.allclose(g[:-1], 0.0)
    assert np.isclose(g[-1], 2 * np.mean(0.25 - t))


def test_single_unit_closed_form():
    """D = H = 1: y = w3 tanh(W2 tanh(W1 x + b1) + b2) + b3 evaluated by hand."""
    W1, b1, W2, b2, w3, b3 = 0.7, -0.2, 1.3, 0.1, -0.9, 0.05
    p = np.array([W1, b1, W2, b2, w3, b3])
    x = 0.4
    y = w3 * np.tanh(W2 * np.tanh(W1 * x + b1) + b2) + b3
    assert np.isclose(mlp.forward(p, [[x]], 1, 1)[0], y, rtol=0, atol=1e-15)


def test_adam_first_step_is_sign_times_lr():
    """Kingma & Ba: the bias-corrected first step is lr * g / (|g| + eps')."""
    g = np.array([0.3, -2.0, 1e-3])
    p, m, v = mlp.adam(np.zeros(3), g, np.zeros(3), np.zeros(3), 1, lr=0.01, eps=1e-12)
    assert np.allclose(p, -0.01 * np.sign(g), rtol=1e-6)
