"""FP64 reference Newton-Raphson power flow (polar form), one instance at a time.

TEST INFRASTRUCTURE ONLY: imported by tests/, __graft_entry__.smoke() and the
CPU-baseline / reference arm of bench.py; never by the library.

What it computes (paper Sec. 3): find the complex bus voltages V such that the
nodal power S_calc = V * conj(Ybus V) (Eq. 1) matches the specified injection at
every bus, for the quantities each bus type fixes: slack (V given), PV (P and
|V| given), PQ (P and Q given).  Each Newton iteration (Sec. 3, steps 1-4)
  1. evaluates the nodal power mismatch F (Alg. 1): dP at PV and PQ buses, dQ at
     PQ buses, each being computed minus specified power;
  2. builds the Jacobian of F with respect to the unknowns [angle at PV+PQ
     buses, |V| at PQ buses] (Sec. 3.1.2, four sub-matrices d{P,Q}/d{angle,|V|});
  3. solves J dx = -F exactly (Eq. 2; the refactorisation of Sec. 4 reaches the
     same solution up to rounding);
  4. adds dx to the angles and magnitudes.
It stops when max|F| < tol (the paper's "maximum of the power injection
mismatch", Sec. 3) or after maxit updates.  The Newton iterates are exactly the
textbook ones, so the oracle is that definition written out; the linear solve
is a library sparse direct solve (scipy SuperLU) or, for small systems, the
dense LU with partial pivoting below.

Readings where the paper is silent (each also listed in the design notes):
  * convergence norm: infinity norm over the dP (PV+PQ) and dQ (PQ) entries,
    strict "<", tested before every update;
  * iteration count: number of Newton updates performed (0 when V0 already
    satisfies the tolerance);
  * update sign: dx = -J^{-1} F with F = computed - specified;
  * status: 0 converged, 1 maxit reached, 2 numerical failure (a non-finite
    mismatch or a singular/non-finite linear solve).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

STATUS_CONVERGED, STATUS_MAXIT, STATUS_FAILED = 0, 1, 2
SLACK, PV, PQ = 3, 2, 1


def make_ybus(n, f, t, r, x, b):
    """Nodal admittance matrix of pi-model branches (MATPOWER convention, Sec. 3).

    Series admittance ys = 1/(r + jx); each end carries half of the total line
    charging b.  Y_ff += ys + jb/2, Y_tt += ys + jb/2, Y_ft -= ys, Y_tf -= ys.
    Built entry by entry in a Python loop so it can be checked by eye.
    Returns a complex128 CSR matrix with sorted column indices and every
    diagonal entry present.
    """
    acc = {}

    def add(i, k, v):
        acc[(i, k)] = acc.get((i, k), 0.0) + v

    for i in range(n):
        add(i, i, 0.0)
    for fb, tb, rr, xx, bb in zip(f, t, r, x, b):
        ys = 1.0 / complex(rr, xx)
        add(int(fb), int(fb), ys + 0.5j * bb)
        add(int(tb), int(tb), ys + 0.5j * bb)
        add(int(fb), int(tb), -ys)
        add(int(tb), int(fb), -ys)
    keys = sorted(acc)
    rows = np.array([k[0] for k in keys], dtype=np.int64)
    cols = np.array([k[1] for k in keys], dtype=np.int64)
    vals = np.array([acc[k] for k in keys], dtype=np.complex128)
    Y = sp.csr_matrix((vals, (rows, cols)), shape=(n, n))
    Y.sort_indices()
    return Y


def branch_flows(f, t, r, x, b, V):
    """Complex power entering each branch at its two ends (the post-processing
    after convergence that the paper's second-chance step precedes, Sec. 3.2).

    pi model: series admittance ys = 1/(r + jx), half of the line charging b at
    each end.  The current leaving bus f into the branch is
    I_f = ys (V_f - V_t) + j b/2 V_f, and symmetrically I_t at bus t; the power
    entering the branch there is S_f = V_f conj(I_f), S_t = V_t conj(I_t).
    Written branch by branch.  Returns (Sf, St) complex128 [nbr].
    """
    nbr = len(f)
    Sf = np.zeros(nbr, np.complex128)
    St = np.zeros(nbr, np.complex128)
    for e in range(nbr):
        vf, vt = V[int(f[e])], V[int(t[e])]
        ys = 1.0 / complex(r[e], x[e])
        i_f = ys * (vf - vt) + 0.5j * b[e] * vf
        i_t = ys * (vt - vf) + 0.5j * b[e] * vt
        Sf[e] = vf * np.conj(i_f)
        St[e] = vt * np.conj(i_t)
    return Sf, St


def bus_sets(bus_type):
    """Index sets (ascending): slack, PV, PQ and PV+PQ (the angle unknowns)."""
    bt = np.asarray(bus_type)
    ref = np.flatnonzero(bt == SLACK)
    pv = np.flatnonzero(bt == PV)
    pq = np.flatnonzero(bt == PQ)
    pvpq = np.concatenate([pv, pq])
    return ref, pv, pq, pvpq


def power_injection(Y, V):
    """Eq. 1: S_calc = V * conj(Ybus V)."""
    return V * np.conj(Y @ V)


def mismatch(Y, V, S, pv, pq):
    """Alg. 1: F = [Re(S_calc - S) at PV+PQ buses ; Im(S_calc - S) at PQ buses].

    Alg. 1 starts each row at -P0 (resp. -Q0) and adds the computed injection;
    slack rows are skipped and PV buses contribute no Q row.
    """
    dS = power_injection(Y, V) - S
    pvpq = np.concatenate([pv, pq])
    return np.concatenate([dS[pvpq].real, dS[pq].imag])


def dS_dV(Y, V):
    """Partial derivatives of S_calc with respect to the angles and magnitudes.

    With S_i = V_i conj(I_i), I = Y V and V_k = |V_k| exp(j theta_k):
      dS_i/dtheta_k = delta_ik j S_i - j V_i conj(Y_ik V_k)
        -> dS/dtheta = j diag(V) conj(diag(I) - Y diag(V))
      dS_i/d|V_k|   = delta_ik conj(I_i) V_i/|V_i| + V_i conj(Y_ik V_k/|V_k|)
        -> dS/d|V|   = diag(V) conj(Y diag(V/|V|)) + conj(diag(I)) diag(V/|V|)
    """
    n = V.shape[0]
    I = Y @ V
    dV = sp.diags(V, format="csr")
    dI = sp.diags(I, format="csr")
    dVn = sp.diags(V / np.abs(V), format="csr")
    dS_dth = 1j * (dV @ np.conj(dI - Y @ dV))
    dS_dvm = dV @ np.conj(Y @ dVn) + np.conj(dI) @ dVn
    assert dS_dth.shape == (n, n)
    return sp.csr_matrix(dS_dth), sp.csr_matrix(dS_dvm)


def jacobian(Y, V, pv, pq):
    """Sec. 3.1.2: J = [[dP/dtheta, dP/d|V|], [dQ/dtheta, dQ/d|V|]].

    Rows: P equations of PV+PQ buses, then Q equations of PQ buses.
    Columns: angles of PV+PQ buses, then magnitudes of PQ buses.
    """
    pvpq = np.concatenate([pv, pq])
    dth, dvm = dS_dV(Y, V)
    J11 = dth[pvpq][:, pvpq].real
    J12 = dvm[pvpq][:, pq].real
    J21 = dth[pq][:, pvpq].imag
    J22 = dvm[pq][:, pq].imag
    return sp.vstack([sp.hstack([J11, J12]), sp.hstack([J21, J22])], format="csr")


def lu_partial_pivot(A):
    """Dense Doolittle LU with partial (row) pivoting: P A = L U.

    Returns (perm, L, U) with perm the row order, L unit lower triangular.
    Column-by-column elimination written out for small systems.
    """
    A = np.array(A, dtype=np.float64, copy=True)
    m = A.shape[0]
    perm = np.arange(m)
    for k in range(m):
        p = k + int(np.argmax(np.abs(A[k:, k])))
        if A[p, k] == 0.0 or not np.isfinite(A[p, k]):
            raise np.linalg.LinAlgError("singular matrix")
        if p != k:
            A[[k, p]] = A[[p, k]]
            perm[[k, p]] = perm[[p, k]]
        for i in range(k + 1, m):
            A[i, k] /= A[k, k]
            A[i, k + 1:] -= A[i, k] * A[k, k + 1:]
    L = np.tril(A, -1) + np.eye(m)
    U = np.triu(A)
    return perm, L, U


def lu_solve(A, rhs):
    """Solve A x = rhs with lu_partial_pivot, then forward/backward substitution."""
    perm, L, U = lu_partial_pivot(A)
    m = L.shape[0]
    y = np.array(rhs, dtype=np.float64)[perm]
    for i in range(m):
        y[i] -= L[i, :i] @ y[:i]
    x = np.empty(m)
    for i in range(m - 1, -1, -1):
        x[i] = (y[i] - U[i, i + 1:] @ x[i + 1:]) / U[i, i]
    return x


def _solve(J, rhs, solver):
    if solver == "dense":
        return lu_solve(J.toarray(), rhs)
    if solver == "sparse":
        return spla.spsolve(sp.csc_matrix(J), rhs)
    raise ValueError(solver)


def newton(Y, S, V0, bus_type, tol=1e-8, maxit=10, solver="sparse", history=None):
    """Polar Newton-Raphson (Sec. 3, steps 1-4) for one instance.

    Y: complex CSR Ybus; S: complex specified injections [n]; V0: complex start
    [n] whose slack voltage and PV magnitudes are the fixed set-points.
    Returns (V, iters, status).  If ``history`` is a list, the infinity norm of
    F at every visited iterate is appended to it.
    """
    _, pv, pq, pvpq = bus_sets(bus_type)
    npvpq = pvpq.shape[0]
    V = np.array(V0, dtype=np.complex128)
    Va = np.angle(V)
    Vm = np.abs(V)
    it = 0
    while True:
        F = mismatch(Y, V, S, pv, pq)
        if not np.all(np.isfinite(F)):
            return V, it, STATUS_FAILED
        nrm = float(np.max(np.abs(F))) if F.size else 0.0
        if history is not None:
            history.append(nrm)
        if nrm < tol:
            return V, it, STATUS_CONVERGED
        if it >= maxit:
            return V, it, STATUS_MAXIT
        J = jacobian(Y, V, pv, pq)
        try:
            with np.errstate(all="ignore"):
                dx = -_solve(J, F, solver)
        except (np.linalg.LinAlgError, RuntimeError):
            return V, it, STATUS_FAILED
        if not np.all(np.isfinite(dx)):
            return V, it, STATUS_FAILED
        Va[pvpq] += dx[:npvpq]
        Vm[pq] += dx[npvpq:]
        V = Vm * np.exp(1j * Va)
        it += 1


def _newton_rows(args):
    Y, S, V0, bus_type, tol, maxit, solver = args
    out_v = np.empty_like(V0)
    out_it = np.empty(V0.shape[0], np.int32)
    out_st = np.empty(V0.shape[0], np.uint8)
    for b in range(V0.shape[0]):
        out_v[b], out_it[b], out_st[b] = newton(Y, S[b], V0[b], bus_type, tol, maxit, solver)
    return out_v, out_it, out_st


def newton_batch(Y, S, V0, bus_type, tol=1e-8, maxit=10, solver="sparse", workers=1):
    """Run ``newton`` over a batch [B, n]; optionally over a process pool.

    The pool is started with the 'spawn' method so it is safe to use after the
    parent process has touched a GPU.
    """
    S = np.asarray(S, np.complex128)
    V0 = np.asarray(V0, np.complex128)
    B = S.shape[0]
    if workers <= 1 or B < 2:
        return _newton_rows((Y, S, V0, bus_type, tol, maxit, solver))
    import multiprocessing as mp
    chunks = np.array_split(np.arange(B), min(workers, B))
    ctx = mp.get_context("spawn")
    with ctx.Pool(len(chunks)) as pool:
        parts = pool.map(_newton_rows, [(Y, S[c], V0[c], bus_type, tol, maxit, solver) for c in chunks])
    return (np.concatenate([p[0] for p in parts]), np.concatenate([p[1] for p in parts]),
            np.concatenate([p[2] for p in parts]))
