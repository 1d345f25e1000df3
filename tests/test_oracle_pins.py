"""Pins of the CPU oracle to facts that do not come from the oracle itself.

Each test checks the oracle against a closed form, an invariant of the power
network, finite differences, an independent textbook algorithm (Gauss-Seidel
power flow) or a library routine, chosen so that a dropped term, a wrong sign,
a wrong index or a transposed operand in the oracle fails at least one of them.
"""
import math

import numpy as np
import pytest
import scipy.optimize

import gridgen
from oracle import nrpf


def two_bus(R, X, P, Q, b=0.0):
    """Slack bus 0 at 1.0 p.u., one line, PQ load P+jQ at bus 1."""
    Y = nrpf.make_ybus(2, [0], [1], [R], [X], [b])
    S = np.array([0.0, -(P + 1j * Q)])
    V0 = np.array([1.0 + 0j, 1.0 + 0j])
    bt = np.array([3, 1], np.int8)
    return Y, S, V0, bt


def two_bus_closed_form(R, X, P, Q):
    """|V2|^4 + (2(PR+QX) - 1)|V2|^2 + (P^2+Q^2)(R^2+X^2) = 0, larger root;
    angle from V1 conj(V2) = |V2|^2 + (R+jX)(P-jQ)."""
    bq = 2 * (P * R + Q * X) - 1.0
    cq = (P * P + Q * Q) * (R * R + X * X)
    u = (-bq + math.sqrt(bq * bq - 4 * cq)) / 2.0
    vm = math.sqrt(u)
    delta = -math.asin((X * P - R * Q) / vm)
    return vm * np.exp(1j * delta)


@pytest.mark.parametrize("R,X,P,Q", [(0.02, 0.1, 0.5, 0.2), (0.05, 0.2, 1.0, 0.3),
                                     (0.1, 0.05, 0.8, -0.1), (0.01, 0.3, 0.2, 0.4)])
def test_two_bus_closed_form(R, X, P, Q):
    Y, S, V0, bt = two_bus(R, X, P, Q)
    V, it, st = nrpf.newton(Y, S, V0, bt, tol=1e-12, maxit=20)
    assert st == nrpf.STATUS_CONVERGED
    assert abs(V[1] - two_bus_closed_form(R, X, P, Q)) < 1e-10
    assert V[0] == 1.0


def test_two_bus_shunt_only():
    """No load, line charging b: V2 = V1 / (1 + j Z b/2) exactly."""
    R, X, b = 0.03, 0.15, 0.4
    Y, S, V0, bt = two_bus(R, X, 0.0, 0.0, b)
    V, it, st = nrpf.newton(Y, S, V0, bt, tol=1e-13, maxit=20)
    assert st == nrpf.STATUS_CONVERGED
    expect = 1.0 / (1.0 + 1j * complex(R, X) * b / 2)
    assert abs(V[1] - expect) < 1e-12


def test_ybus_two_bus_entries():
    r, x, b = 0.02, 0.08, 0.1
    Y = nrpf.make_ybus(2, [0], [1], [r], [x], [b]).toarray()
    ys = 1 / complex(r, x)
    assert np.allclose(Y, [[ys + 0.5j * b, -ys], [-ys, ys + 0.5j * b]], rtol=0, atol=1e-14)


def test_ybus_invariants():
    g = gridgen.make_grid("mesh30_b64")
    Y = nrpf.make_ybus(g.n, g.f, g.t, g.r, g.x, g.b)
    D = Y.toarray()
    assert np.allclose(D, D.T, atol=1e-14)
    # each row sums to the shunt admittance at that bus (half line charging of
    # every incident branch): the series parts cancel
    shunt = np.zeros(g.n, complex)
    for f, t, b in zip(g.f, g.t, g.b):
        shunt[f] += 0.5j * b
        shunt[t] += 0.5j * b
    assert np.allclose(D.sum(axis=1), shunt, atol=1e-12)
    # diagonal present everywhere, sorted columns
    assert all(Y[i, i] != 0 for i in range(g.n))
    assert Y.has_sorted_indices


def branch_losses(g, V):
    """Total complex power absorbed by the branches, from branch currents."""
    tot = 0j
    for f, t, r, x, b in zip(g.f, g.t, g.r, g.x, g.b):
        Is = (V[f] - V[t]) / complex(r, x)
        tot += abs(Is) ** 2 * complex(r, x) - 0.5j * b * (abs(V[f]) ** 2 + abs(V[t]) ** 2)
    return tot


def _mesh30():
    g = gridgen.make_grid("mesh30_b64")
    Y = nrpf.make_ybus(g.n, g.f, g.t, g.r, g.x, g.b)
    sc = gridgen.config_scenarios("mesh30_b64", g, batch=8)
    return g, Y, sc.sbus(g), sc.v0_flat(g)


def test_power_balance_any_voltage():
    """Sum of nodal injections = power absorbed by the network, at any V."""
    g, Y, S, V0 = _mesh30()
    rng = np.random.default_rng(5)
    V = (1 + 0.05 * rng.standard_normal(g.n)) * np.exp(0.1j * rng.standard_normal(g.n))
    tot = nrpf.power_injection(Y, V).sum()
    assert abs(tot - branch_losses(g, V)) < 1e-10


def test_power_balance_at_solution():
    g, Y, S, V0 = _mesh30()
    for b in range(4):
        V, it, st = nrpf.newton(Y, S[b], V0[b], g.bus_type)
        assert st == nrpf.STATUS_CONVERGED
        Sc = nrpf.power_injection(Y, V)
        assert abs(Sc.sum() - branch_losses(g, V)) < 1e-10
        _, pv, pq, pvpq = nrpf.bus_sets(g.bus_type)
        assert np.max(np.abs(Sc[pvpq].real - S[b][pvpq].real)) < 1e-8
        assert np.max(np.abs(Sc[pq].imag - S[b][pq].imag)) < 1e-8
        assert np.allclose(np.abs(V[pv]), g.v_set[pv], atol=1e-14)


def test_mismatch_matches_alg1_polar_form():
    """Alg. 1 accumulates |V_i||Y_ij||V_j| cos/sin(theta_i - angle(Y_ij) - theta_j)."""
    g, Y, S, V0 = _mesh30()
    rng = np.random.default_rng(3)
    V = (1 + 0.03 * rng.standard_normal(g.n)) * np.exp(0.05j * rng.standard_normal(g.n))
    _, pv, pq, pvpq = nrpf.bus_sets(g.bus_type)
    Yc = Y.tocsr()
    dP = -S[0].real.copy()
    dQ = -S[0].imag.copy()
    for row in range(g.n):
        for d in range(Yc.indptr[row], Yc.indptr[row + 1]):
            col = Yc.indices[d]
            mag = abs(V[row]) * abs(Yc.data[d]) * abs(V[col])
            ang = np.angle(V[row]) - np.angle(Yc.data[d]) - np.angle(V[col])
            dP[row] += mag * math.cos(ang)
            dQ[row] += mag * math.sin(ang)
    F = nrpf.mismatch(Y, V, S[0], pv, pq)
    assert np.allclose(F, np.concatenate([dP[pvpq], dQ[pq]]), rtol=0, atol=1e-12)


def test_jacobian_central_differences():
    g, Y, S, V0 = _mesh30()
    _, pv, pq, pvpq = nrpf.bus_sets(g.bus_type)
    rng = np.random.default_rng(7)
    Va = 0.05 * rng.standard_normal(g.n)
    Vm = 1 + 0.03 * rng.standard_normal(g.n)
    Vm[pv] = g.v_set[pv]

    def F(x):
        a = Va.copy()
        m = Vm.copy()
        a[pvpq] = x[:pvpq.size]
        m[pq] = x[pvpq.size:]
        return nrpf.mismatch(Y, m * np.exp(1j * a), S[0], pv, pq)

    x0 = np.concatenate([Va[pvpq], Vm[pq]])
    J = nrpf.jacobian(Y, Vm * np.exp(1j * Va), pv, pq).toarray()
    h = 1e-6
    Jfd = np.empty_like(J)
    for k in range(x0.size):
        e = np.zeros_like(x0)
        e[k] = h
        Jfd[:, k] = (F(x0 + e) - F(x0 - e)) / (2 * h)
    assert np.max(np.abs(J - Jfd)) <= 1e-6 * np.max(np.abs(J))
    # structurally: the J pattern is the Ybus pattern expanded to 2x2 blocks
    assert J.shape == (pvpq.size + pq.size,) * 2


def test_dense_lu_against_library():
    rng = np.random.default_rng(11)
    for m in (1, 2, 5, 17, 40):
        A = rng.standard_normal((m, m))
        perm, L, U = nrpf.lu_partial_pivot(A)
        assert np.allclose(A[perm], L @ U, atol=1e-12)
        assert np.allclose(np.diag(L), 1.0)
        rhs = rng.standard_normal(m)
        assert np.allclose(nrpf.lu_solve(A, rhs), np.linalg.solve(A, rhs), rtol=1e-10, atol=1e-10)
    # pivoting is exercised: a zero leading entry
    A = np.array([[0.0, 1.0], [2.0, 3.0]])
    assert np.allclose(nrpf.lu_solve(A, [1.0, 2.0]), np.linalg.solve(A, [1.0, 2.0]))
    with pytest.raises(np.linalg.LinAlgError):
        nrpf.lu_partial_pivot(np.zeros((3, 3)))


def test_jacobian_solve_against_library():
    g, Y, S, V0 = _mesh30()
    _, pv, pq, _ = nrpf.bus_sets(g.bus_type)
    J = nrpf.jacobian(Y, V0[0], pv, pq)
    F = nrpf.mismatch(Y, V0[0], S[0], pv, pq)
    x1 = nrpf.lu_solve(J.toarray(), F)
    x2 = np.linalg.solve(J.toarray(), F)
    x3 = nrpf._solve(J, F, "sparse")
    assert np.allclose(x1, x2, rtol=1e-10, atol=1e-12)
    assert np.allclose(x3, x2, rtol=1e-10, atol=1e-12)


def test_sparse_and_dense_newton_agree():
    g, Y, S, V0 = _mesh30()
    for b in range(4):
        Vs, its, sts = nrpf.newton(Y, S[b], V0[b], g.bus_type, solver="sparse")
        Vd, itd, std = nrpf.newton(Y, S[b], V0[b], g.bus_type, solver="dense")
        assert (its, sts) == (itd, std)
        assert np.max(np.abs(Vs - Vd)) < 1e-12


def gauss_seidel(Y, S, V0, bus_type, tol=1e-11, sweeps=20000):
    """Textbook Gauss-Seidel power flow (independent of Newton's method)."""
    Yd = Y.toarray()
    V = np.array(V0, complex)
    vset = np.abs(V0)
    n = V.size
    _, pv, pq, pvpq = nrpf.bus_sets(bus_type)
    is_pv = np.isin(np.arange(n), pv)
    for _ in range(sweeps):
        for i in pvpq:
            s = S[i]
            if is_pv[i]:
                q = (V[i] * np.conj(Yd[i] @ V)).imag
                s = complex(S[i].real, q)
            acc = Yd[i] @ V - Yd[i, i] * V[i]
            V[i] = (np.conj(s) / np.conj(V[i]) - acc) / Yd[i, i]
            if is_pv[i]:
                V[i] *= vset[i] / abs(V[i])
        F = nrpf.mismatch(Y, V, S, pv, pq)
        if np.max(np.abs(F)) < tol:
            return V
    raise AssertionError("Gauss-Seidel did not converge")


def test_newton_matches_gauss_seidel():
    g, Y, S, V0 = _mesh30()
    for b in range(2):
        Vn, it, st = nrpf.newton(Y, S[b], V0[b], g.bus_type, tol=1e-11)
        assert st == nrpf.STATUS_CONVERGED
        Vg = gauss_seidel(Y, S[b], V0[b], g.bus_type)
        assert np.max(np.abs(Vn - Vg)) < 1e-8


def test_three_bus_brute_force_root():
    """A 3-bus grid with a PV bus, solved as a root problem in rectangular
    coordinates by a library root finder (no Jacobian from the oracle)."""
    Y = nrpf.make_ybus(3, [0, 1, 0], [1, 2, 2], [0.02, 0.03, 0.025], [0.1, 0.12, 0.09], [0.01, 0.0, 0.02])
    bt = np.array([3, 2, 1], np.int8)
    S = np.array([0, 0.4, -(0.7 + 0.25j)])
    V0 = np.array([1.0, 1.03, 1.0], complex)
    Vn, it, st = nrpf.newton(Y, S, V0, bt, tol=1e-12)
    assert st == nrpf.STATUS_CONVERGED
    Yd = Y.toarray()

    def res(z):
        e1, f1, e2, f2 = z
        V = np.array([1.0, e1 + 1j * f1, e2 + 1j * f2])
        Sc = V * np.conj(Yd @ V)
        return [Sc[1].real - 0.4, abs(V[1]) ** 2 - 1.03 ** 2,
                Sc[2].real - S[2].real, Sc[2].imag - S[2].imag]

    z = scipy.optimize.fsolve(res, [1.0, 0.0, 1.0, 0.0], xtol=1e-14)
    Vb = np.array([1.0, z[0] + 1j * z[1], z[2] + 1j * z[3]])
    assert np.max(np.abs(np.array(res(z)))) < 1e-12
    assert np.max(np.abs(Vn - Vb)) < 1e-10


def test_quadratic_convergence():
    g, Y, S, V0 = _mesh30()
    h = []
    V, it, st = nrpf.newton(Y, S[0], V0[0], g.bus_type, tol=1e-13, history=h)
    assert st == nrpf.STATUS_CONVERGED and it == len(h) - 1
    # from the second step on, ||F_{k+1}|| <= C ||F_k||^2 with a modest C
    ratios = [h[k + 1] / h[k] ** 2 for k in range(1, len(h) - 1) if h[k] > 1e-7]
    assert ratios and max(ratios) < 50


def test_iteration_count_semantics():
    g, Y, S, V0 = _mesh30()
    h = []
    Vs, it, st = nrpf.newton(Y, S[0], V0[0], g.bus_type, history=h)
    assert st == nrpf.STATUS_CONVERGED
    # iters = number of updates = index of the first iterate under tol
    assert it == next(k for k, v in enumerate(h) if v < 1e-8)
    # starting at the solution: zero updates
    V2, it2, st2 = nrpf.newton(Y, S[0], Vs, g.bus_type)
    assert (it2, st2) == (0, nrpf.STATUS_CONVERGED)
    # maxit = 0 from flat start: no update, not converged
    _, it3, st3 = nrpf.newton(Y, S[0], V0[0], g.bus_type, maxit=0)
    assert (it3, st3) == (0, nrpf.STATUS_MAXIT)
    # maxit = 1
    _, it4, st4 = nrpf.newton(Y, S[0], V0[0], g.bus_type, maxit=1)
    assert (it4, st4) == (1, nrpf.STATUS_MAXIT)


def test_failure_status():
    g, Y, S, V0 = _mesh30()
    Sbad = S[0].copy()
    Sbad[3] = np.nan
    _, it, st = nrpf.newton(Y, Sbad, V0[0], g.bus_type)
    assert st == nrpf.STATUS_FAILED and it == 0
    # an isolated PQ bus makes J singular
    Yi = nrpf.make_ybus(3, [0], [1], [0.02], [0.1], [0.0])
    bt = np.array([3, 1, 1], np.int8)
    _, it, st = nrpf.newton(Yi, np.array([0, -0.1, -0.1 + 0j]), np.ones(3, complex), bt)
    assert st == nrpf.STATUS_FAILED


def test_batch_helper_and_pool():
    g, Y, S, V0 = _mesh30()
    V1, it1, st1 = nrpf.newton_batch(Y, S, V0, g.bus_type)
    V2, it2, st2 = nrpf.newton_batch(Y, S, V0, g.bus_type, workers=2)
    assert np.array_equal(it1, it2) and np.array_equal(st1, st2)
    assert np.max(np.abs(V1 - V2)) == 0.0
    assert np.all(st1 == 0)


def test_tolerance_threshold_is_strict():
    """The stopping test is max|F| < tol, evaluated before every update."""
    g, Y, S, V0 = _mesh30()
    h = []
    nrpf.newton(Y, S[0], V0[0], g.bus_type, tol=1e-14, history=h)
    for k in range(1, len(h) - 1):
        _, it, st = nrpf.newton(Y, S[0], V0[0], g.bus_type, tol=h[k] * 1.5)
        assert (it, st) == (k, nrpf.STATUS_CONVERGED)
        _, it, st = nrpf.newton(Y, S[0], V0[0], g.bus_type, tol=h[k])
        assert (it, st) == (k + 1, nrpf.STATUS_CONVERGED)
        _, it, st = nrpf.newton(Y, S[0], V0[0], g.bus_type, tol=h[k] / 1.5)
        assert (it, st) == (k + 1, nrpf.STATUS_CONVERGED)


def test_branch_flows_sum_to_nodal_injections():
    """Kirchhoff: at every bus the powers entering its branch ends add up to
    the nodal injection V conj(Y V) of the independently assembled Ybus, at any
    V (no bus shunts in these grids)."""
    g, Y, S, V0 = _mesh30()
    rng = np.random.default_rng(8)
    V = (1 + 0.05 * rng.standard_normal(g.n)) * np.exp(0.1j * rng.standard_normal(g.n))
    Sf, St = nrpf.branch_flows(g.f, g.t, g.r, g.x, g.b, V)
    acc = np.zeros(g.n, complex)
    np.add.at(acc, g.f, Sf)
    np.add.at(acc, g.t, St)
    assert np.max(np.abs(acc - nrpf.power_injection(Y, V))) < 1e-12


def test_branch_flows_closed_form_losses():
    """S_f + S_t = conj(ys) |V_f - V_t|^2 - j b/2 (|V_f|^2 + |V_t|^2) per
    branch, and a lossless open-ended line (V_t = V_f) carries only its
    charging."""
    g, Y, S, V0 = _mesh30()
    rng = np.random.default_rng(9)
    V = (1 + 0.05 * rng.standard_normal(g.n)) * np.exp(0.1j * rng.standard_normal(g.n))
    Sf, St = nrpf.branch_flows(g.f, g.t, g.r, g.x, g.b, V)
    ys = 1.0 / (g.r + 1j * g.x)
    vf, vt = V[g.f], V[g.t]
    want = np.conj(ys) * np.abs(vf - vt) ** 2 - 0.5j * g.b * (np.abs(vf) ** 2 + np.abs(vt) ** 2)
    assert np.max(np.abs(Sf + St - want)) < 1e-12
    Sf1, St1 = nrpf.branch_flows([0], [1], [0.02], [0.1], [0.04], np.array([1.02 + 0.0j, 1.02 + 0.0j]))
    assert abs(Sf1[0] - (-0.02j * 1.02 ** 2)) < 1e-15 and abs(St1[0] - Sf1[0]) < 1e-15
