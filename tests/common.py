"""Shared helpers of the test-suite: seeded cases and oracle runs."""
from __future__ import annotations

import numpy as np

import gridgen
from oracle import nrpf


def case(name, batch=None, seed=1):
    g = gridgen.make_grid(name)
    sc = gridgen.config_scenarios(name, g, batch=batch, seed=seed)
    return g, sc.sbus(g), sc.v0_flat(g)


def oracle_ybus(g):
    return nrpf.make_ybus(g.n, g.f, g.t, g.r, g.x, g.b)


def perturbed(V, seed=0, mag=0.02, ang=0.05):
    rng = np.random.default_rng(seed)
    return V * (1 + mag * rng.standard_normal(V.shape)) * np.exp(1j * ang * rng.standard_normal(V.shape))


def permuted_dense(colptr, rowidx, vals, m):
    """Dense matrix from CCS pattern + values."""
    A = np.zeros((m, m))
    for j in range(m):
        A[rowidx[colptr[j]:colptr[j + 1]], j] = vals[colptr[j]:colptr[j + 1]]
    return A
