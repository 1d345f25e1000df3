"""FP64 reference of the warm-start network: forward pass, loss, backward pass
and one AdamW step, written out plainly for checking the GPU kernels.

TEST INFRASTRUCTURE ONLY (tests/, smoke(), bench.py's CPU arm).

Network (the learned warm start: per-bus injections -> initial voltages):
  h1 = GELU(x W1 + b1), h2 = GELU(h1 W2 + b2), y = h2 W3 + b3,
  GELU(z) = z * Phi(z) = 0.5 z (1 + erf(z / sqrt(2)))   (exact form),
  loss = mean over the batch and the outputs of (y - t)^2.
Weights W_l are stored [fan_in, fan_out].  AdamW: decoupled weight decay
(Loshchilov & Hutter), bias-corrected first/second moments.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf

SQRT2 = math.sqrt(2.0)
INV_SQRT_2PI = 1.0 / math.sqrt(2.0 * math.pi)


def gelu(z):
    return 0.5 * z * (1.0 + erf(z / SQRT2))


def gelu_grad(z):
    """d/dz [z Phi(z)] = Phi(z) + z phi(z)."""
    return 0.5 * (1.0 + erf(z / SQRT2)) + z * INV_SQRT_2PI * np.exp(-0.5 * z * z)


def forward(params, x):
    """Returns (y, cache).  params = [W1, b1, W2, b2, W3, b3]."""
    W1, b1, W2, b2, W3, b3 = params
    z1 = x @ W1 + b1
    h1 = gelu(z1)
    z2 = h1 @ W2 + b2
    h2 = gelu(z2)
    y = h2 @ W3 + b3
    return y, (x, z1, h1, z2, h2)


def loss(y, t):
    return float(np.mean((y - t) ** 2))


def backward(params, cache, y, t):
    """Gradients of the mean-squared loss, by the chain rule, layer by layer."""
    W1, b1, W2, b2, W3, b3 = params
    x, z1, h1, z2, h2 = cache
    dy = 2.0 * (y - t) / y.size
    gW3 = h2.T @ dy
    gb3 = dy.sum(axis=0)
    dh2 = dy @ W3.T
    dz2 = dh2 * gelu_grad(z2)
    gW2 = h1.T @ dz2
    gb2 = dz2.sum(axis=0)
    dh1 = dz2 @ W2.T
    dz1 = dh1 * gelu_grad(z1)
    gW1 = x.T @ dz1
    gb1 = dz1.sum(axis=0)
    return [gW1, gb1, gW2, gb2, gW3, gb3]


def adamw_step(p, g, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8, wd=0.0):
    """One AdamW update of one tensor (in place on p, m, v); step counts from 1."""
    p *= 1.0 - lr * wd
    m[...] = beta1 * m + (1.0 - beta1) * g
    v[...] = beta2 * v + (1.0 - beta2) * g * g
    mh = m / (1.0 - beta1 ** step)
    vh = v / (1.0 - beta2 ** step)
    p -= lr * mh / (np.sqrt(vh) + eps)
