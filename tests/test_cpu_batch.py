"""The batched host solver (instances in SIMD lanes, threads over mini-batches)
against the FP64 oracle, on CPU: statuses, iteration counts and voltages,
ragged mini-batches, maxit and failure semantics, and both dense cuts."""
import numpy as np
import pytest

import gridgen
from oracle import nrpf

TOL = 1e-8


def _plan(g, **kw):
    pf = pytest.importorskip("paper_2101_02270_gb300")
    return pf.Plan.from_branches(g.n, g.f, g.t, g.r, g.x, g.b, g.bus_type, host_only=True, **kw)


def _compare(g, S, V0, v, it, st, idx, maxit=10):
    Y = nrpf.make_ybus(g.n, g.f, g.t, g.r, g.x, g.b)
    for b in idx:
        Vo, ito, sto = nrpf.newton(Y, S[b], V0[b], g.bus_type, TOL, maxit)
        assert st[b] == sto and it[b] == ito, b
        if sto == 0:
            assert np.max(np.abs(v[b] - Vo)) < 1e-9


@pytest.mark.parametrize("kw", [{}, {"dense_frac": 0.3}, {"dense_frac": 1.0}, {"ordering": "natural"}])
def test_cpu_batch_mesh30_against_oracle(kw):
    g = gridgen.make_grid("mesh30_b64")
    sc = gridgen.config_scenarios("mesh30_b64", g, batch=29)  # 3 full mini-batches and a ragged one
    S, V0 = sc.sbus(g), sc.v0_flat(g)
    p = _plan(g, **kw)
    v, it, st = p.solve_cpu(S, V0, TOL, 10, threads=3)
    assert np.all(st == 0)
    _compare(g, S, V0, v, it, st, range(29))
    p.close()


def test_cpu_batch_mesh2000_sample():
    g = gridgen.make_grid("mesh2000_b10k")
    sc = gridgen.config_scenarios("mesh2000_b10k", g, batch=10)
    S, V0 = sc.sbus(g), sc.v0_flat(g)
    p = _plan(g)
    v, it, st = p.solve_cpu(S, V0, TOL, 10)
    assert np.all(st == 0)
    _compare(g, S, V0, v, it, st, [0, 4, 9])
    p.close()


def test_cpu_batch_maxit_and_failure():
    g = gridgen.make_grid("mesh30_b64")
    sc = gridgen.config_scenarios("mesh30_b64", g, batch=10)
    S, V0 = sc.sbus(g), sc.v0_flat(g)
    S[3, 6] = np.nan
    p = _plan(g)
    v, it, st = p.solve_cpu(S, V0, TOL, 2)
    assert st[3] == 2 and it[3] == 0
    ok = np.arange(10) != 3
    assert np.all(st[ok] == 1) and np.all(it[ok] == 2)
    v0, it0, st0 = p.solve_cpu(S[:1], V0[:1], TOL, 0)
    assert st0[0] == 1 and it0[0] == 0 and np.array_equal(v0, V0[:1])
    p.close()
