"""Second chance on the GPU path: instances whose refactorisation without
pivoting breaks down are re-solved by the pivoting host solver and then match
the FP64 oracle; instances that converged are left untouched."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import gridgen  # noqa: E402
from oracle import nrpf  # noqa: E402
from tests.test_pivoting_host import _scen, resistive_leaf_grid  # noqa: E402

pytestmark = pytest.mark.gpu
TOL = 1e-8


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _plan(g, **kw):
    import paper_2101_02270_gb300 as pf
    return pf.Plan.from_branches(g.n, g.f, g.t, g.r, g.x, g.b, g.bus_type, **kw)


@pytest.mark.parametrize("lu", ["fp64", "fp32"])
def test_zero_pivot_cases_recovered_by_second_chance(lu):
    g = resistive_leaf_grid()
    S, V0 = _scen(g, 40)
    Sd, Vd = _dev(S), _dev(V0)
    with _plan(g, lu_precision=lu) as p:
        out = p.solve(Sd, Vd, TOL, 10)
        assert bool((out[2] == 2).all())  # the zero first pivot breaks every instance
        n = p.retry_failed(Sd, Vd, out, TOL, 10)
        v, it, st = (t.cpu().numpy() for t in out)
    assert n == 40 and np.all(st == 0)
    Y = nrpf.make_ybus(g.n, g.f, g.t, g.r, g.x, g.b)
    for b in range(0, 40, 3):
        Vo, ito, sto = nrpf.newton(Y, S[b], V0[b], g.bus_type, TOL, 10)
        assert sto == 0 and it[b] == ito
        assert np.max(np.abs(v[b] - Vo)) < 1e-9


def test_second_chance_leaves_converged_instances_alone():
    g = gridgen.make_grid("mesh30_b64")
    sc = gridgen.config_scenarios("mesh30_b64", g, batch=33)
    S, V0 = sc.sbus(g), sc.v0_flat(g)
    S[5, 3] = np.nan
    Sd, Vd = _dev(S), _dev(V0)
    with _plan(g) as p:
        out = p.solve(Sd, Vd, TOL, 10)
        before = tuple(t.clone() for t in out)
        n = p.retry_failed(Sd, Vd, out, TOL, 10)
    assert n == 1
    keep = torch.ones(33, dtype=torch.bool)
    keep[5] = False
    for a, b in zip(before, out):
        assert torch.equal(a[keep.cuda()], b[keep.cuda()])
    assert int(out[2][5]) == 2 and int(out[1][5]) == 0
