"""Parity at the benchmark's full sizes and launch configurations, on sampled
outputs that the CPU oracle recomputes one by one (spawned oracle processes,
so the pool is safe next to a CUDA context), plus properties that hold at any
size (every instance converged, recomputed mismatch below tolerance)."""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import gridgen  # noqa: E402
from oracle import nrpf  # noqa: E402
from tests.common import oracle_ybus  # noqa: E402

pytestmark = pytest.mark.gpu
TOL = 1e-8


def _pf():
    import paper_2101_02270_gb300 as pf
    return pf


def _cores():
    return max(1, min(16, os.cpu_count() or 1))


def _check(g, S, V0, Vg, itg, stg, idx, maxit, exact_iters):
    Y = oracle_ybus(g)
    Vo, ito, sto = nrpf.newton_batch(Y, S[idx], V0[idx], g.bus_type, TOL, maxit, workers=min(len(idx), _cores()))
    assert np.array_equal(stg[idx], sto)
    if exact_iters:
        assert np.array_equal(itg[idx], ito)
    else:
        assert np.all(itg[idx] >= ito) and np.all(itg[idx] <= ito + 3)
    ok = sto == 0
    assert np.max(np.abs(np.abs(Vg[idx][ok]) - np.abs(Vo[ok])), initial=0) <= 1e-6
    assert np.max(np.abs(np.angle(Vg[idx][ok] * np.conj(Vo[ok]))), initial=0) <= 1e-6


def test_mesh9000_fp32_full_batch_sampled():
    """9,000 buses x 10,000 scenarios, FP32 LU with the default dense block
    (instance-major, factorised by the CTA-tiled kernels: the mixed-precision
    benchmark's configuration, about 206 GB of LU workspace)."""
    pf = _pf()
    g = gridgen.make_grid("mesh9000_b10k")
    sc = gridgen.config_scenarios("mesh9000_b10k", g)
    S, V0 = sc.sbus(g), sc.v0_flat(g)
    with pf.Plan.from_branches(g.n, g.f, g.t, g.r, g.x, g.b, g.bus_type, lu_precision="fp32") as p:
        assert p.info["dense_layout"] == 2
        v, it, st = p.solve(torch.from_numpy(S).cuda(), torch.from_numpy(V0).cuda(), TOL, 10)
        Vg, itg, stg = v.cpu().numpy(), it.cpu().numpy(), st.cpu().numpy()
    assert np.all(stg == 0)
    idx = np.array([0, 4999, 9999] + list(np.random.default_rng(1).choice(10000, 5, replace=False)))
    _check(g, S, V0, Vg, itg, stg, idx, 10, exact_iters=False)
    # any size: the oracle's mismatch at the GPU's voltages, further sample
    Y = oracle_ybus(g)
    _, pv, pq, _ = nrpf.bus_sets(g.bus_type)
    for b in np.random.default_rng(2).choice(10000, 16, replace=False):
        assert np.max(np.abs(nrpf.mismatch(Y, Vg[b], S[b], pv, pq))) < TOL


def test_feeders_full_group_sampled():
    """256 feeders x 100 scenarios in one persistent launch (FP32 LU)."""
    pf = _pf()
    fs = gridgen.make_feeders()
    scen = gridgen.grids.feeder_scenarios(fs)
    plans = [pf.Plan.from_branches(g.n, g.f, g.t, g.r, g.x, g.b, g.bus_type, lu_precision="fp32", dense_frac=1.0)
             for g in fs]
    mp = pf.MultiPlan(plans, [sc.batch for sc in scen])
    S = [sc.sbus(g) for g, sc in zip(fs, scen)]
    V0 = [sc.v0_flat(g) for g, sc in zip(fs, scen)]
    Sd = torch.from_numpy(np.concatenate([s.ravel() for s in S])).cuda()
    Vd = torch.from_numpy(np.concatenate([v.ravel() for v in V0])).cuda()
    mp.autotune(Sd, Vd, TOL, 20)
    v, it, st = mp.solve(Sd, Vd, TOL, 20)
    v, it, st = v.cpu().numpy(), it.cpu().numpy(), st.cpu().numpy()
    assert np.all(st == 0)
    off = ioff = 0
    rng = np.random.default_rng(3)
    for k, (g, s, v0) in enumerate(zip(fs, S, V0)):
        B = s.shape[0]
        if k % 32 == 0:  # eight feeders of the group, four scenarios each
            idx = rng.choice(B, 4, replace=False)
            Vg = v[off:off + B * g.n].reshape(B, g.n)
            _check(g, s, v0, Vg, it[ioff:ioff + B], st[ioff:ioff + B], idx, 20, exact_iters=False)
        off += B * g.n
        ioff += B
    mp.close()
