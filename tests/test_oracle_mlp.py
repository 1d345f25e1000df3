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


def test_adamw_constant_gradient_closed_form_over_steps():
    """With a constant gradient g the bias-corrected moments are exact at every
    step: m_k = (1 - b1^k) g and v_k = (1 - b2^k) g^2, so m_k / (1 - b1^k) = g
    and v_k / (1 - b2^k) = g^2.  Each of steps 1..5 then moves p by the same
    -lr g / (|g| + eps) after the decay.  A bias correction with a fixed
    exponent (1 - b1 instead of 1 - b1^k) is off by (1 - b1^k) / (1 - b1) from
    step 2 on."""
    rng = np.random.default_rng(4)
    p0 = rng.standard_normal(12)
    g = rng.standard_normal(12)
    lr, wd = 1e-2, 0.05
    p = p0.copy()
    m = np.zeros(12)
    v = np.zeros(12)
    expect = p0.copy()
    for k in range(1, 6):
        mlp.adamw_step(p, g, m, v, k, lr=lr, wd=wd)
        expect = expect * (1 - lr * wd) - lr * g / (np.abs(g) + 1e-8)
        assert np.max(np.abs(m - (1 - 0.9 ** k) * g)) < 1e-15, k
        assert np.max(np.abs(v - (1 - 0.999 ** k) * g * g)) < 1e-15, k
        assert np.max(np.abs(p - expect)) < 1e-13, k


def test_adamw_two_gradients_worked_example():
    """Two steps with gradients g1 then g2, worked by hand with b1 = 0.9,
    b2 = 0.999, wd = 0: m_2 = 0.09 g1 + 0.1 g2, bias-corrected by 1 - 0.81 =
    0.19; v_2 = 0.000999 g1^2 + 0.001 g2^2, bias-corrected by 1 - 0.998001 =
    0.001999.  For g1 = 1, g2 = -3 (one coordinate): m_hat = (0.09 - 0.3) /
    0.19 = -21/19 and v_hat = (0.000999 + 0.009) / 0.001999 = 9999/1999."""
    lr = 0.1
    p = np.array([0.0])
    m = np.zeros(1)
    v = np.zeros(1)
    mlp.adamw_step(p, np.array([1.0]), m, v, 1, lr=lr)
    p1 = -lr * 1.0 / (1.0 + 1e-8)
    assert abs(p[0] - p1) < 1e-15
    mlp.adamw_step(p, np.array([-3.0]), m, v, 2, lr=lr)
    m_hat = -21.0 / 19.0
    v_hat = 9999.0 / 1999.0
    expect = p1 - lr * m_hat / (math.sqrt(v_hat) + 1e-8)
    assert abs(p[0] - expect) < 1e-14


def test_forward_hand_worked_network():
    """A 2-2-2-1 network whose pre-activations land on tabulated points of the
    standard normal distribution: Phi(1) = 0.8413447460685429, Phi(2) =
    0.9772498680518208.  Row 1, x = (1, 1): z1 = x W1 + b1 = (1, 2), h1 =
    (Phi(1), 2 Phi(2)); W2 divides by those values so that z2 = (1, 2) and
    h2 = (Phi(1), 2 Phi(2)) again; y = h2_1 - h2_2 + 0.5.  Row 2, x = (-20, 0):
    z1 = (-20, -39), GELU ~ 0, so z2 = 0, h2 = 0 and y = b3 = 0.5.  A dropped
    GELU, a transposed weight or a missing bias changes y."""
    phi1, phi2 = 0.8413447460685429, 0.9772498680518208
    g1, g2 = phi1, 2.0 * phi2  # GELU(1), GELU(2)
    W1 = np.array([[1.0, 2.0], [0.0, -1.0]])
    b1 = np.array([0.0, 1.0])
    W2 = np.array([[1.0 / g1, 1.0 / g1], [0.0, 1.0 / g2]])
    b2 = np.zeros(2)
    W3 = np.array([[1.0], [-1.0]])
    b3 = np.array([0.5])
    x = np.array([[1.0, 1.0], [-20.0, 0.0]])
    y, (x_, z1, h1, z2, h2) = mlp.forward([W1, b1, W2, b2, W3, b3], x)
    assert np.allclose(z1[0], [1.0, 2.0], rtol=0, atol=1e-15)
    assert np.allclose(h1[0], [g1, g2], rtol=0, atol=1e-15)
    assert np.allclose(z2[0], [1.0, 2.0], rtol=0, atol=1e-15)
    assert abs(y[0, 0] - (g1 - g2 + 0.5)) < 1e-15
    assert abs(y[0, 0] - (-0.6131549900350987)) < 1e-15
    assert abs(y[1, 0] - 0.5) < 1e-15
    assert y.shape == (2, 1)
