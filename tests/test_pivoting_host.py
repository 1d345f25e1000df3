"""The pivoting host solver (the second chance for instances that fail
without pivoting) against the FP64 oracle, on CPU: plain scenarios, a grid
whose Jacobian has a zero diagonal at flat start (purely resistive leaf line:
dP/dtheta of the leaf bus is exactly 0 there), and failure/maxit semantics."""
import numpy as np
import pytest

import gridgen
from oracle import nrpf

TOL = 1e-8


def _pf():
    return pytest.importorskip("paper_2101_02270_gb300")


def _plan(g):
    return _pf().Plan.from_branches(g.n, g.f, g.t, g.r, g.x, g.b, g.bus_type, host_only=True)


def resistive_leaf_grid():
    """The 30-bus grid plus bus 30 (PQ, small load) hanging on bus 5 by a line
    with r = 0.02, x = 0, no charging: at flat start the leaf's dP/dtheta is
    V30 V5 (G sin 0 - B cos 0) with B = 0, exactly zero, and minimum degree
    eliminates the leaf first, so a refactorisation without pivoting meets
    that zero on its first pivot."""
    g = gridgen.make_grid("mesh30_b64")
    n = g.n + 1
    f = np.append(g.f, 5).astype(np.int32)
    t = np.append(g.t, g.n).astype(np.int32)
    grow = lambda a, v: np.append(a, v)
    return gridgen.Grid("mesh30_leaf", n, f, t, grow(g.r, 0.02), grow(g.x, 0.0), grow(g.b, 0.0),
                        grow(g.bus_type, 1).astype(np.int8), grow(g.p_gen, 0.0), grow(g.p_load, 0.05),
                        grow(g.q_load, 0.0), grow(g.v_set, 1.0), g.load_scale)


def _scen(g, B, seed=1):
    rng = np.random.default_rng(seed)
    fac = rng.uniform(0.7, 1.3, size=(B, g.n))
    base = g.p_gen - g.p_load - 1j * g.q_load
    S = g.load_scale * fac * base[None, :]
    V0 = np.broadcast_to(g.v_set.astype(np.complex128), S.shape).copy()
    return S, V0


def _compare(g, S, V0, v, it, st, maxit=10, iters_exact=True):
    Y = nrpf.make_ybus(g.n, g.f, g.t, g.r, g.x, g.b)
    for b in range(S.shape[0]):
        Vo, ito, sto = nrpf.newton(Y, S[b], V0[b], g.bus_type, TOL, maxit)
        assert st[b] == sto
        if iters_exact:
            assert it[b] == ito
        if sto == 0:
            assert np.max(np.abs(v[b] - Vo)) < 1e-9


def test_pivoting_host_matches_oracle_mesh30():
    g = gridgen.make_grid("mesh30_b64")
    sc = gridgen.config_scenarios("mesh30_b64", g, batch=24)
    S, V0 = sc.sbus(g), sc.v0_flat(g)
    p = _plan(g)
    v, it, st = p.solve_pivoting_host(S, V0, TOL, 10)
    assert np.all(st == 0)
    _compare(g, S, V0, v, it, st)
    # maxit semantics: 2 updates, then status 1
    v2, it2, st2 = p.solve_pivoting_host(S[:4], V0[:4], TOL, 2)
    assert np.all(st2 == 1) and np.all(it2 == 2)
    p.close()


def test_zero_diagonal_at_flat_start_is_pivoted_around():
    g = resistive_leaf_grid()
    Y = nrpf.make_ybus(g.n, g.f, g.t, g.r, g.x, g.b)
    _, pv, pq, pvpq = nrpf.bus_sets(g.bus_type)
    J = nrpf.jacobian(Y, np.ones(g.n, complex) * g.v_set, pv, pq).toarray()
    leaf = list(pvpq).index(g.n - 1)
    assert J[leaf, leaf] == 0.0  # the zero diagonal the test is about
    S, V0 = _scen(g, 12)
    p = _plan(g)
    v, it, st = p.solve_pivoting_host(S, V0, TOL, 10)
    assert np.all(st == 0)
    _compare(g, S, V0, v, it, st)
    p.close()


def test_non_finite_injection_fails_cleanly():
    g = gridgen.make_grid("mesh30_b64")
    sc = gridgen.config_scenarios("mesh30_b64", g, batch=3)
    S, V0 = sc.sbus(g), sc.v0_flat(g)
    S[1, 7] = np.nan
    p = _plan(g)
    v, it, st = p.solve_pivoting_host(S, V0, TOL, 10)
    assert st.tolist() == [0, 2, 0] and it[1] == 0
    p.close()
