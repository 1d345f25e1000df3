"""GPU parity: every stage and the whole solve, through the C ABI, against the
CPU FP64 oracle on the same seeded inputs.

Tolerances (float64 everywhere on the FP64 path):
  * mismatch F, Jacobian entries: 1e-10 absolute (sums of a handful of O(10)
    products; only the summation order differs);
  * factorisation: ||L U - P J P^T||_max <= 1e-10 ||J||_max;
  * linear solve: ||dx - dx_oracle||_max <= 1e-8 (1 + ||dx_oracle||_max);
  * Newton result: equal status and iteration counts, |d|V|| <= 1e-6 p.u.,
    |d theta| <= 1e-6 rad, and the oracle's mismatch at the GPU's voltages
    below the tolerance 1e-8 p.u.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

torch = pytest.importorskip("torch")

from oracle import nrpf  # noqa: E402
from tests.common import case, oracle_ybus, perturbed, permuted_dense  # noqa: E402

pytestmark = pytest.mark.gpu

TOL = 1e-8


def _pf():
    import paper_2101_02270_gb300 as pf
    return pf


def _plan(g, **kw):
    return _pf().Plan.from_branches(g.n, g.f, g.t, g.r, g.x, g.b, g.bus_type, **kw)


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _oracle_solve(g, S, V0, tol=TOL, maxit=10, idx=None):
    Y = oracle_ybus(g)
    idx = range(S.shape[0]) if idx is None else idx
    out = [nrpf.newton(Y, S[b], V0[b], g.bus_type, tol, maxit) for b in idx]
    return (np.array([o[0] for o in out]), np.array([o[1] for o in out]), np.array([o[2] for o in out]))


def _compare_newton(g, Vg, itg, stg, Vo, ito, sto, S, check_iters=True):
    assert np.array_equal(stg, sto)
    if check_iters:
        assert np.array_equal(itg, ito)
    ok = sto == 0
    dvm = np.abs(np.abs(Vg[ok]) - np.abs(Vo[ok]))
    dth = np.abs(np.angle(Vg[ok] * np.conj(Vo[ok])))
    assert dvm.max(initial=0) <= 1e-6 and dth.max(initial=0) <= 1e-6
    Y = oracle_ybus(g)
    _, pv, pq, _ = nrpf.bus_sets(g.bus_type)
    for b in np.flatnonzero(ok):
        F = nrpf.mismatch(Y, Vg[b], S[b], pv, pq)
        assert np.max(np.abs(F)) < TOL


@pytest.mark.parametrize("name,B", [("mesh30_b64", 64), ("mesh30_b64", 37), ("mesh2000_b10k", 45)])
def test_mismatch_stage(name, B):
    g, S, V0 = case(name, batch=B)
    V = perturbed(V0, seed=3)
    with _plan(g) as p:
        F, norm = p.stage_mismatch(_dev(S), _dev(V))
        F = F.cpu().numpy()
        norm = norm.cpu().numpy()
    Y = oracle_ybus(g)
    _, pv, pq, _ = nrpf.bus_sets(g.bus_type)
    for b in range(B):
        Fo = nrpf.mismatch(Y, V[b], S[b], pv, pq)
        assert np.max(np.abs(F[b] - Fo)) < 1e-10
        assert abs(norm[b] - np.max(np.abs(Fo))) < 1e-10


@pytest.mark.parametrize("name,B,kw", [("mesh30_b64", 40, {}), ("mesh30_b64", 33, {"ordering": "natural"}),
                                       ("mesh2000_b10k", 3, {}),
                                       ("mesh30_b64", 40, {"lu_precision": "fp32"}),
                                       ("mesh30_b64", 35, {"lu_precision": "fp32", "panel": 8}),
                                       ("mesh2000_b10k", 3, {"lu_precision": "fp32"}),
                                       ("mesh30_b64", 36, {"panel": 32}),
                                       ("mesh2000_b10k", 3, {"lu_precision": "fp32", "panel": 32}),
                                       ("mesh2000_b10k", 2, {"lu_precision": "fp32", "panel": 64}),
                                       # instance-major dense block: ndp 64 (one last panel of 64),
                                       # 320 (full, half and corner GEMM tiles), 384 (full tiles only)
                                       ("mesh30_b64", 40, {"lu_precision": "fp32", "dense_layout": "instance_major"}),
                                       ("mesh2000_b10k", 3, {"lu_precision": "fp32",
                                                             "dense_layout": "instance_major"}),
                                       ("mesh2000_b10k", 2, {"lu_precision": "fp32", "dense_layout": "instance_major",
                                                             "dense_frac": 0.12})])
def test_jacobian_and_factor_stage(name, B, kw):
    g, S, V0 = case(name, batch=B)
    V = perturbed(V0, seed=4)
    with _plan(g, **kw) as p:
        pos, colptr, rowidx = p.pattern()
        A = p.stage_factor(_dev(V), factor=False).cpu().numpy()
        LU = p.stage_factor(_dev(V), factor=True).cpu().numpy()
        m = p.info["m"]
    Y = oracle_ybus(g)
    _, pv, pq, _ = nrpf.bus_sets(g.bus_type)
    inv = np.empty(m, int)
    inv[pos] = np.arange(m)
    fp32 = kw.get("lu_precision") == "fp32"
    for b in range(B):
        J = nrpf.jacobian(Y, V[b], pv, pq).toarray()
        PJP = J[np.ix_(inv, inv)]  # row/col r of A is J row/col inv[r]
        Ag = permuted_dense(colptr, rowidx, A[b], m)
        # FP32 storage of J: relative rounding 2^-24
        assert np.max(np.abs(Ag - PJP)) < (1e-6 * np.max(np.abs(J)) if fp32 else 1e-10)
        F = permuted_dense(colptr, rowidx, LU[b], m)
        L = np.tril(F, -1) + np.eye(m)
        U = np.triu(F)
        assert np.max(np.abs(L @ U - PJP)) <= (1e-4 if fp32 else 1e-10) * np.max(np.abs(J))


@pytest.mark.parametrize("name,B,kw", [("mesh30_b64", 64, {}), ("mesh30_b64", 70, {"panel": 4}),
                                       ("mesh30_b64", 32, {"panel": 16}), ("mesh2000_b10k", 8, {}),
                                       ("mesh30_b64", 64, {"lu_precision": "fp32"}),
                                       ("mesh2000_b10k", 8, {"lu_precision": "fp32"}),
                                       ("mesh30_b64", 40, {"lu_precision": "fp32", "panel": 32}),
                                       ("mesh2000_b10k", 8, {"lu_precision": "fp32", "panel": 32}),
                                       ("mesh30_b64", 33, {"panel": 64}),
                                       ("mesh2000_b10k", 8, {"lu_precision": "fp32", "panel": 64}),
                                       ("mesh30_b64", 45, {"lu_precision": "fp32", "dense_layout": "instance_major"}),
                                       ("mesh2000_b10k", 8, {"lu_precision": "fp32",
                                                             "dense_layout": "instance_major"}),
                                       ("mesh2000_b10k", 8, {"lu_precision": "fp32", "dense_layout": "instance_major",
                                                             "dense_frac": 0.12})])
def test_linear_solve_stage(name, B, kw):
    g, S, V0 = case(name, batch=B)
    V = perturbed(V0, seed=5)
    rng = np.random.default_rng(9)
    with _plan(g, **kw) as p:
        m = p.info["m"]
        rhs = rng.standard_normal((B, m))
        dx = p.stage_linear_solve(_dev(V), _dev(rhs)).cpu().numpy()
    Y = oracle_ybus(g)
    _, pv, pq, _ = nrpf.bus_sets(g.bus_type)
    for b in range(B):
        J = nrpf.jacobian(Y, V[b], pv, pq)
        xo = spla.spsolve(J.tocsc(), rhs[b])
        tol = 1e-3 if kw.get("lu_precision") == "fp32" else 1e-8  # FP32 LU: cond(J) * 2^-24
        assert np.max(np.abs(dx[b] - xo)) <= tol * (1 + np.max(np.abs(xo)))


@pytest.mark.parametrize("B", [64, 1, 45])
def test_newton_mesh30(B):
    g, S, V0 = case("mesh30_b64", batch=B)
    with _plan(g) as p:
        v, it, st = p.solve(_dev(S), _dev(V0), TOL, 10)
        Vg, itg, stg = v.cpu().numpy(), it.cpu().numpy(), st.cpu().numpy()
    Vo, ito, sto = _oracle_solve(g, S, V0)
    _compare_newton(g, Vg, itg, stg, Vo, ito, sto, S)


def test_newton_mesh2000_ragged():
    g, S, V0 = case("mesh2000_b10k", batch=70)
    with _plan(g) as p:
        v, it, st = p.solve(_dev(S), _dev(V0), TOL, 10)
        Vg, itg, stg = v.cpu().numpy(), it.cpu().numpy(), st.cpu().numpy()
    idx = list(range(0, 70, 3))
    Vo, ito, sto = _oracle_solve(g, S, V0, idx=idx)
    _compare_newton(g, Vg[idx], itg[idx], stg[idx], Vo, ito, sto, S[idx])


def test_newton_mesh2000_full_batch_sampled():
    """The benchmark's launch configuration (10,000 scenarios); outputs sampled."""
    g, S, V0 = case("mesh2000_b10k")
    with _plan(g) as p:
        v, it, st = p.solve(_dev(S), _dev(V0), TOL, 10)
        Vg, itg, stg = v.cpu().numpy(), it.cpu().numpy(), st.cpu().numpy()
    idx = list(np.random.default_rng(0).choice(S.shape[0], 24, replace=False)) + [0, S.shape[0] - 1]
    Vo, ito, sto = _oracle_solve(g, S, V0, idx=idx)
    _compare_newton(g, Vg[idx], itg[idx], stg[idx], Vo, ito, sto, S[idx])
    # properties at any size: every instance converged, the recomputed
    # mismatch of a further sample is below tolerance
    assert np.all(stg == 0)


def test_edge_cases():
    pf = _pf()
    g, S, V0 = case("mesh30_b64", batch=8)
    Vo, ito, sto = _oracle_solve(g, S, V0, tol=1e-12, maxit=20)
    with _plan(g) as p:
        # B == 0 is a no-op
        assert pf.lib.pf_solve_batch(p._h, 0, None, None, 1e-8, 10, None, None, None, None) == 0
        # maxit = 0
        v, it, st = p.solve(_dev(S), _dev(V0), TOL, 0)
        assert np.all(it.cpu().numpy() == 0) and np.all(st.cpu().numpy() == 1)
        # starting at the solution: zero updates
        v, it, st = p.solve(_dev(S), _dev(Vo), TOL, 10)
        assert np.all(it.cpu().numpy() == 0) and np.all(st.cpu().numpy() == 0)
        # tol = 0 cannot be met: maxit updates
        v, it, st = p.solve(_dev(S), _dev(V0), 0.0, 6)
        assert np.all(it.cpu().numpy() == 6) and np.all(st.cpu().numpy() == 1)
        # a non-finite injection fails that instance only
        Sb = S.copy()
        Sb[3, 5] = np.nan
        v, it, st = p.solve(_dev(Sb), _dev(V0), TOL, 10)
        st = st.cpu().numpy()
        it = it.cpu().numpy()
        assert st[3] == 2 and it[3] == 0
        assert np.all(np.delete(st, 3) == 0)
        # bad arguments
        assert pf.lib.pf_solve_batch(p._h, -1, None, None, 1e-8, 10, None, None, None, None) == -1
        assert pf.lib.pf_solve_batch(p._h, 1, None, None, float("nan"), 10, None, None, None, None) == -1


def test_instance_major_edge_cases():
    """Instance-major FP32 dense block: a non-finite injection fails its own
    instance only, an instance that starts at the solution takes no update,
    and maxit = 0 reports every instance at its limit."""
    g, S, V0 = case("mesh2000_b10k", batch=36)
    Vo, ito, sto = _oracle_solve(g, S[:2], V0[:2], tol=1e-12, maxit=20)
    with _plan(g, lu_precision="fp32", dense_layout="instance_major") as p:
        assert p.info["dense_layout"] == 2
        Sb = S.copy()
        Sb[33, 17] = np.nan
        V0b = V0.copy()
        V0b[:2] = Vo
        v, it, st = p.solve(_dev(Sb), _dev(V0b), TOL, 20)
        st, it = st.cpu().numpy(), it.cpu().numpy()
        assert st[33] == 2 and it[33] == 0
        assert np.all(np.delete(st, 33) == 0)
        assert np.all(it[:2] == 0)
        v, it, st = p.solve(_dev(S), _dev(V0), TOL, 0)
        assert np.all(it.cpu().numpy() == 0) and np.all(st.cpu().numpy() == 1)


def test_singular_instance_reports_failure():
    """An instance whose Jacobian is singular (a PQ bus with zero voltage)
    stops with status 2 while the rest of the batch converges."""
    g, S, V0 = case("mesh30_b64", batch=4)
    V0 = V0.copy()
    V0[1, 7] = 0.0
    with _plan(g) as p:
        v, it, st = p.solve(_dev(S), _dev(V0), TOL, 10)
        st = st.cpu().numpy()
    assert st[1] == 2 and np.all(st[[0, 2, 3]] == 0)


def test_plan_reuse_and_capacity_growth():
    g, S, V0 = case("mesh30_b64", batch=64)
    with _plan(g, max_batch=16) as p:
        a = p.solve(_dev(S[:16]), _dev(V0[:16]), TOL, 10)
        b = p.solve(_dev(S), _dev(V0), TOL, 10)  # grows the workspace
        c = p.solve(_dev(S[:16]), _dev(V0[:16]), TOL, 10)
        assert torch.equal(a[0], c[0]) and torch.equal(a[1], c[1])
        assert torch.equal(b[0][:16], a[0])
        assert p.info["capacity"] >= 64


@pytest.mark.parametrize("name,B,panel,layout", [("mesh30_b64", 64, 0, "auto"), ("mesh2000_b10k", 40, 0, "auto"),
                                                 ("mesh2000_b10k", 40, 32, "auto"), ("mesh2000_b10k", 40, 64, "auto"),
                                                 ("mesh30_b64", 64, 0, "instance_major"),
                                                 ("mesh2000_b10k", 70, 0, "instance_major")])
def test_mixed_precision_lu(name, B, panel, layout):
    """FP32 LU + FS/BS, FP64 mismatch/update: same statuses, same tolerance,
    a few more iterations at most (default panel, the two-level panels of
    32 and 64 factorised in steps of 16, and the instance-major dense block)."""
    g, S, V0 = case(name, batch=B)
    with _plan(g, lu_precision="fp32", panel=panel, dense_layout=layout) as p:
        v, it, st = p.solve(_dev(S), _dev(V0), TOL, 20)
        Vg, itg, stg = v.cpu().numpy(), it.cpu().numpy(), st.cpu().numpy()
    idx = list(range(0, B, max(1, B // 10)))
    Vo, ito, sto = _oracle_solve(g, S, V0, idx=idx)
    _compare_newton(g, Vg[idx], itg[idx], stg[idx], Vo, ito, sto, S[idx], check_iters=False)
    assert np.all(itg[idx] >= ito) and np.all(itg[idx] <= ito + 3)


def test_fresh_workspace_ignores_stale_memory():
    """A plan whose workspace reuses memory freed by another plan (here full of
    NaN from a failed instance) still gives clean results: nothing of the
    solve reads workspace it did not write first."""
    g, S, V0 = case("mesh30_b64", batch=32)
    Sb = S.copy()
    Sb[:, 4] = np.nan
    with _plan(g) as p:
        p.solve(_dev(Sb), _dev(V0), TOL, 10)
        torch.cuda.synchronize()
    for _ in range(3):
        with _plan(g) as p:
            v, it, st = p.solve(_dev(S), _dev(V0), TOL, 10)
            assert np.all(st.cpu().numpy() == 0)


@pytest.mark.parametrize("lu,maxit", [("fp64", 10), ("fp32", 10), ("fp64", 2)])
def test_loop_graph_matches_host_loops(lu, maxit):
    """The Newton loop run as a graph WHILE node (default), as a host loop
    ended from the host (profiled solves) and as a fixed-count loop inside a
    caller's stream capture give identical results; the graph runs one body
    per check up to the last active instance's, not maxit."""
    g, S, V0 = case("mesh30_b64", batch=64)
    Sd, Vd = _dev(S), _dev(V0)
    with _plan(g, lu_precision=lu) as p:
        outs = [tuple(torch.empty_like(t) for t in p.solve(Sd, Vd, TOL, maxit)) for _ in range(3)]
        p.profile_start([])
        p.solve(Sd, Vd, TOL, maxit, out=outs[0])
        counts = p.profile_read()
        p.profile_start(["dense_update"])
        p.solve(Sd, Vd, TOL, maxit, out=outs[1])
        p.profile_read()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            p.solve(Sd, Vd, TOL, maxit, out=outs[2])
        graph.replay()
        torch.cuda.synchronize()
    a, b, c = outs
    for x, y in ((a, b), (a, c)):
        assert torch.equal(x[0], y[0]) and torch.equal(x[1], y[1]) and torch.equal(x[2], y[2])
    st, it = a[2].cpu().numpy(), a[1].cpu().numpy()
    if maxit == 10:
        assert np.all(st == 0)
        bodies = int(it.max()) + 1  # the check that finds no instance active ends the loop
    else:
        assert np.all(st == 1) and np.all(it == maxit)
        bodies = maxit
    assert counts["check"][0] == bodies + 1  # plus the final test after the loop
    assert counts["update"][0] == bodies


@pytest.mark.parametrize("lu,B,chunk", [("fp64", 100, 32), ("fp32", 100, 0), ("fp64", 64, 64), ("fp64", 45, 200)])
def test_host_batch_chunks_match_device_solve(lu, B, chunk):
    """pf_solve_batch_host (chunks copied in and out around the solves,
    ragged last chunk) gives exactly the device-resident solve's results, and
    those match the oracle (FP64 LU: same iterations; FP32 LU: at most three
    more)."""
    g, S, V0 = case("mesh30_b64", batch=B)
    with _plan(g, lu_precision=lu) as p:
        v, it, st = p.solve(_dev(S), _dev(V0), TOL, 10)
        Sh = torch.from_numpy(np.ascontiguousarray(S)).pin_memory()
        Vh = torch.from_numpy(np.ascontiguousarray(V0)).pin_memory()
        vh, ith, sth = p.solve_host(Sh, Vh, TOL, 10, chunk=chunk)
        torch.cuda.current_stream().synchronize()
        # pageable host memory works too
        vp, itp, stp = p.solve_host(torch.from_numpy(np.ascontiguousarray(S)),
                                    torch.from_numpy(np.ascontiguousarray(V0)), TOL, 10, chunk=chunk)
        torch.cuda.current_stream().synchronize()
    for a, b, c in ((v, vh, vp), (it, ith, itp), (st, sth, stp)):
        assert torch.equal(a.cpu(), b) and torch.equal(a.cpu(), c)
    # and the host-batch results against the oracle, instance by instance
    Vo, ito, sto = _oracle_solve(g, S, V0)
    ith_np = ith.numpy()
    _compare_newton(g, vh.numpy(), ith_np, sth.numpy(), Vo, ito, sto, S, check_iters=lu == "fp64")
    if lu == "fp32":
        ok = sto == 0
        assert np.all(ith_np[ok] >= ito[ok]) and np.all(ith_np[ok] <= ito[ok] + 3)


def test_host_batch_back_to_back_calls():
    """Consecutive host-batch calls without a synchronisation in between (the
    second call's copy-in overlaps the first call's solve) each return the
    device solve of their own inputs, and the oracle's solution of them."""
    g, S1, V0 = case("mesh30_b64", batch=64)
    S2 = S1 * 0.9
    with _plan(g) as p:
        ref = [p.solve(_dev(S), _dev(V0), TOL, 10) for S in (S1, S2, S1)]
        ref = [tuple(t.cpu() for t in r) for r in ref]
        hs = [torch.from_numpy(np.ascontiguousarray(S)).pin_memory() for S in (S1, S2, S1)]
        hv = torch.from_numpy(np.ascontiguousarray(V0)).pin_memory()
        outs = [p.solve_host(h, hv, TOL, 10) for h in hs]
        torch.cuda.current_stream().synchronize()
    for r, o in zip(ref, outs):
        for a, b in zip(r, o):
            assert torch.equal(a, b)
    # each call's results against the oracle on its own inputs
    for S, o in zip((S1, S2, S1), outs):
        Vo, ito, sto = _oracle_solve(g, S, V0)
        _compare_newton(g, o[0].numpy(), o[1].numpy(), o[2].numpy(), Vo, ito, sto, S)
