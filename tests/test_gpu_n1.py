"""Per-instance admittances on a shared pattern (static N-1 contingency
analysis) on the GPU, against the FP64 oracle run on each post-outage grid."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import gridgen  # noqa: E402
from oracle import nrpf  # noqa: E402

pytestmark = pytest.mark.gpu
TOL = 1e-8


def _pf():
    import paper_2101_02270_gb300 as pf
    return pf


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _plan(g, **kw):
    return _pf().Plan.from_branches(g.n, g.f, g.t, g.r, g.x, g.b, g.bus_type, **kw)


def _oracle_case(g, keep, S, V0, maxit=10):
    Y = nrpf.make_ybus(g.n, g.f[keep], g.t[keep], g.r[keep], g.x[keep], g.b[keep])
    return nrpf.newton(Y, S, V0, g.bus_type, TOL, maxit) + (Y,)


def _check(g, ins, S, V0, Vg, itg, stg, idx, exact_iters=True):
    _, pv, pq, _ = nrpf.bus_sets(g.bus_type)
    for b in idx:
        Vo, ito, sto, Y = _oracle_case(g, ins[b], S[b], V0[b])
        assert stg[b] == sto, b
        if exact_iters:
            assert itg[b] == ito, b
        else:
            assert ito <= itg[b] <= ito + 3, b
        if sto == 0:
            assert np.max(np.abs(np.abs(Vg[b]) - np.abs(Vo))) <= 1e-6
            assert np.max(np.abs(np.angle(Vg[b] * np.conj(Vo)))) <= 1e-6
            assert np.max(np.abs(nrpf.mismatch(Y, Vg[b], S[b], pv, pq))) < TOL


@pytest.mark.parametrize("lu", ["fp64", "fp32"])
def test_shared_values_per_instance_equal_plain_solve(lu):
    """Every instance given the plan's own admittances: bit-identical to the
    shared-admittance solve."""
    g = gridgen.make_grid("mesh30_b64")
    sc = gridgen.config_scenarios("mesh30_b64", g, batch=70)
    S, V0 = sc.sbus(g), sc.v0_flat(g)
    with _plan(g, lu_precision=lu) as p:
        Y = np.repeat(p.ybus_values(), 70, axis=0)
        a = p.solve(_dev(S), _dev(V0), TOL, 10)
        b = p.solve_y(_dev(Y), _dev(S), _dev(V0), TOL, 10)
        c = p.solve(_dev(S), _dev(V0), TOL, 10)  # back on the shared values
        for x, y, z in zip(a, b, c):
            assert torch.equal(x, y) and torch.equal(x, z)


@pytest.mark.parametrize("lu", ["fp64", "fp32"])
def test_n1_mesh30_all_cases(lu):
    """All 41 single-branch outages of the 30-bus grid at five load levels
    (205 instances), each against the oracle on its own grid."""
    g = gridgen.make_grid("mesh30_b64")
    outage, level, ins, S = gridgen.n1_batch(g)
    V0 = np.broadcast_to(g.v_set.astype(np.complex128), S.shape).copy()
    with _plan(g, lu_precision=lu) as p:
        Y = p.ybus_values(ins)
        v, it, st = p.solve_y(_dev(Y), _dev(S), _dev(V0), TOL, 10)
        Vg, itg, stg = v.cpu().numpy(), it.cpu().numpy(), st.cpu().numpy()
    _check(g, ins, S, V0, Vg, itg, stg, range(len(outage)), exact_iters=lu == "fp64")


def test_n1_mesh2000_full_batch_sampled():
    """The 2,000-bus N-1 workload (1,913 connected outages x 5 load levels,
    9,565 instances) in one launch; sampled instances against the oracle."""
    g = gridgen.make_grid("mesh2000_b10k")
    outage, level, ins, S = gridgen.n1_batch(g)
    V0 = np.broadcast_to(g.v_set.astype(np.complex128), S.shape).copy()
    with _plan(g) as p:
        Y = p.ybus_values(ins)
        v, it, st = p.solve_y(_dev(Y), _dev(S), _dev(V0), TOL, 10)
        Vg, itg, stg = v.cpu().numpy(), it.cpu().numpy(), st.cpu().numpy()
    rng = np.random.default_rng(0)
    idx = [0, len(outage) - 1] + list(rng.choice(len(outage), 6, replace=False))
    _check(g, ins, S, V0, Vg, itg, stg, idx)


def test_branch_flows_against_oracle():
    """Branch flows of solved N-1 cases: every end against the oracle's
    branch-by-branch formula at the GPU's voltages (outaged branches carry
    nothing), and the flows at each bus add up to its specified injection."""
    g = gridgen.make_grid("mesh30_b64")
    outage, level, ins, S = gridgen.n1_batch(g)
    V0 = np.broadcast_to(g.v_set.astype(np.complex128), S.shape).copy()
    with _plan(g) as p:
        Y = p.ybus_values(ins)
        v, it, st = p.solve_y(_dev(Y), _dev(S), _dev(V0), TOL, 10)
        sf, stt = p.branch_flows(v, torch.from_numpy(ins).cuda())
        Vg, sf, stt = v.cpu().numpy(), sf.cpu().numpy(), stt.cpu().numpy()
        assert np.all(st.cpu().numpy() == 0)
    _, pv, pq, _ = nrpf.bus_sets(g.bus_type)
    for k in range(0, len(outage), 7):
        keep = ins[k]
        Sfo, Sto = nrpf.branch_flows(g.f[keep], g.t[keep], g.r[keep], g.x[keep], g.b[keep], Vg[k])
        assert np.max(np.abs(sf[k][keep] - Sfo)) < 1e-12 and np.max(np.abs(stt[k][keep] - Sto)) < 1e-12
        assert np.all(sf[k][~keep] == 0) and np.all(stt[k][~keep] == 0)
        acc = np.zeros(g.n, complex)
        np.add.at(acc, g.f, sf[k])
        np.add.at(acc, g.t, stt[k])
        assert np.max(np.abs(acc[pq] - S[k][pq])) < 1e-8
        assert np.max(np.abs(acc.real[pv] - S[k].real[pv])) < 1e-8


@pytest.mark.parametrize("lu", ["fp64", "fp32"])
def test_device_built_outage_cases(lu):
    """Outage cases whose admittances are built on the device (base values
    minus the outaged branches' stamps) give the results of the host-built
    per-instance admittances; N-2 cases with a repeated index and an empty
    slot match the oracle on their grids."""
    g = gridgen.make_grid("mesh30_b64")
    outage, level, ins, S = gridgen.n1_batch(g)
    V0 = np.broadcast_to(g.v_set.astype(np.complex128), S.shape).copy()
    with _plan(g, lu_precision=lu) as p:
        Y = p.ybus_values(ins)
        a = [t.cpu().numpy() for t in p.solve_y(_dev(Y), _dev(S), _dev(V0), TOL, 10)]
        o = torch.from_numpy(outage.astype(np.int32)[:, None]).cuda()
        b = [t.cpu().numpy() for t in p.solve_outages(o, _dev(S), _dev(V0), TOL, 10)]
        assert np.array_equal(a[2], b[2])
        assert np.max(np.abs(a[0] - b[0])) < 1e-10
        if lu == "fp64":
            assert np.array_equal(a[1], b[1])
        # N-2: pairs of outages (plus a repeated index and an empty slot)
        rng = np.random.default_rng(4)
        B = 24
        pairs = np.stack([rng.choice(len(outage) // 5, 2, replace=False) for _ in range(B)]).astype(np.int32)
        pairs = outage[:len(outage) // 5][pairs].astype(np.int32)
        extra = np.full((B, 2), -1, np.int32)
        extra[0, 0] = pairs[0, 0]  # repeated: removed once
        o2 = np.concatenate([pairs, extra], axis=1)
        S2, V2 = S[:B], V0[:B]
        v, it, st = (t.cpu().numpy() for t in p.solve_outages(torch.from_numpy(o2).cuda(), _dev(S2), _dev(V2), TOL, 10))
    for bi in range(0, B, 3):
        keep = np.ones(g.n_branch, bool)
        keep[o2[bi][o2[bi] >= 0]] = False
        Vo, ito, sto, Yo = _oracle_case(g, keep, S2[bi], V2[bi])
        assert st[bi] == sto
        if sto == 0:
            assert np.max(np.abs(v[bi] - Vo)) < 1e-6
