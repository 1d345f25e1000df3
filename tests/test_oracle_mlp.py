"""Pins of the CPU reference network (oracle/mlp.py): central finite
differences of the loss, closed forms of GELU, and the closed form of the
first AdamW step."""
import math

import numpy as np

from oracle import mlp


def _net(rng, sizes):
    ps = []
    for a, b in zip(sizes[:-1], sizes[1:]):
        ps += [rng.standard_normal((a, b)) / math.sqrt(a), 0.1 * rng.standard_normal(b)]
    return ps


def test_gelu_closed_forms():
    assert mlp.gelu(np.array([0.0]))[0] == 0.0
    assert abs(mlp.gelu(np.array([10.0]))[0] - 10.0) < 1e-12
    assert abs(mlp.gelu(np.array([-10.0]))[0]) < 1e-12
    # GELU(1) = Phi(1) = 0.841344746...
    assert abs(mlp.gelu(np.array([1.0]))[0] - 0.8413447460685429) < 1e-12
    z = np.linspace(-4, 4, 41)
    h = 1e-6
    fd = (mlp.gelu(z + h) - mlp.gelu(z - h)) / (2 * h)
    assert np.max(np.abs(fd - mlp.gelu_grad(z))) < 1e-8


def test_backward_matches_finite_differences():
    rng = np.random.default_rng(0)
    sizes = [7, 6, 5, 4]
    p = _net(rng, sizes)
    x = rng.standard_normal((3, 7))
    t = rng.standard_normal((3, 4))
    y, cache = mlp.forward(p, x)
    g = mlp.backward(p, cache, y, t)
    h = 1e-6
    for k, P in enumerate(p):
        fd = np.zeros_like(P)
        it = np.nditer(P, flags=["multi_index"])
        for _ in it:
            idx = it.multi_index
            old = P[idx]
            P[idx] = old + h
            lp = mlp.loss(mlp.forward(p, x)[0], t)
            P[idx] = old - h
            lm = mlp.loss(mlp.forward(p, x)[0], t)
            P[idx] = old
            fd[idx] = (lp - lm) / (2 * h)
        assert np.max(np.abs(fd - g[k])) < 1e-7, k


def test_first_adamw_step_closed_form():
    """Step 1: m = (1-b1) g, v = (1-b2) g^2, bias-corrected m/(1-b1) = g and
    v/(1-b2) = g^2, so p <- p (1 - lr wd) - lr g / (|g| + eps)."""
    rng = np.random.default_rng(1)
    p0 = rng.standard_normal(10)
    g = rng.standard_normal(10)
    p = p0.copy()
    m = np.zeros(10)
    v = np.zeros(10)
    mlp.adamw_step(p, g, m, v, 1, lr=1e-3, wd=0.01)
    expect = p0 * (1 - 1e-3 * 0.01) - 1e-3 * g / (np.abs(g) + 1e-8)
    assert np.max(np.abs(p - expect)) < 1e-15
