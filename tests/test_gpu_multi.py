"""Uneven batching (pf_multi_*): grids of different sizes and patterns, each
with its own scenario count, in one persistent graph-captured launch, checked
instance by instance against the CPU oracle."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import gridgen  # noqa: E402
from oracle import nrpf  # noqa: E402
from tests.common import case, oracle_ybus  # noqa: E402

pytestmark = pytest.mark.gpu
TOL = 1e-8


def _pf():
    import paper_2101_02270_gb300 as pf
    return pf


def _group(grids, scen, lu="fp64"):
    pf = _pf()
    plans = [pf.Plan.from_branches(g.n, g.f, g.t, g.r, g.x, g.b, g.bus_type, lu_precision=lu, dense_frac=1.0)
             for g in grids]
    S = [sc.sbus(g) for g, sc in zip(grids, scen)]
    V0 = [sc.v0_flat(g) for g, sc in zip(grids, scen)]
    mp = pf.MultiPlan(plans, [s.shape[0] for s in S])
    Sc = torch.from_numpy(np.concatenate([s.ravel() for s in S])).cuda()
    Vc = torch.from_numpy(np.concatenate([v.ravel() for v in V0])).cuda()
    return plans, mp, S, V0, Sc, Vc


def _check(grids, S, V0, v, it, st, exact_iters):
    v, it, st = v.cpu().numpy(), it.cpu().numpy(), st.cpu().numpy()
    off = ioff = 0
    for g, s, v0 in zip(grids, S, V0):
        B = s.shape[0]
        Vg = v[off:off + B * g.n].reshape(B, g.n)
        Y = oracle_ybus(g)
        _, pv, pq, _ = nrpf.bus_sets(g.bus_type)
        for b in range(B):
            Vo, ito, sto = nrpf.newton(Y, s[b], v0[b], g.bus_type, TOL, 10)
            assert st[ioff + b] == sto
            if exact_iters:
                assert it[ioff + b] == ito
            else:
                assert ito <= it[ioff + b] <= ito + 3
            if sto == 0:
                assert np.max(np.abs(np.abs(Vg[b]) - np.abs(Vo))) <= 1e-6
                assert np.max(np.abs(np.angle(Vg[b] * np.conj(Vo)))) <= 1e-6
                assert np.max(np.abs(nrpf.mismatch(Y, Vg[b], s[b], pv, pq))) < TOL
        off += B * g.n
        ioff += B


def _feeders(sizes_batches):
    fs = gridgen.make_feeders(count=len(sizes_batches))
    scen = gridgen.grids.feeder_scenarios(fs, per_feeder=1)
    out_s = []
    rng = np.random.default_rng(3)
    for g, (B,) in zip(fs, sizes_batches):
        out_s.append(gridgen.Scenarios(rng.uniform(0.6, 1.4, size=(B, g.n)), g.load_scale))
    return fs, out_s


@pytest.mark.parametrize("lu,exact", [("fp64", True), ("fp32", False)])
def test_multi_feeders_uneven(lu, exact):
    fs, scen = _feeders([(37,), (5,), (64,), (1,), (33,), (20,)])
    plans, mp, S, V0, Sc, Vc = _group(fs, scen, lu)
    for w, b in [(1, 4), (4, 2), (8, 1)]:
        mp.set_config(w, b)
        v, it, st = mp.solve(Sc, Vc, TOL, 10)
        _check(fs, S, V0, v, it, st, exact)
    mp.close()


@pytest.mark.parametrize("lu,exact", [("fp64", True), ("fp32", False)])
@pytest.mark.parametrize("per_item,smem", [(32, True), (8, True), (4, True), (1, True), (8, False)])
def test_multi_scenarios_per_item_and_shared_memory(lu, exact, per_item, smem):
    """Items of S scenarios (lanes split into S scenarios x 32/S workers),
    state in shared memory where it fits: every instance equals the oracle's
    (ragged tiles: batches not multiples of S)."""
    fs, scen = _feeders([(13,), (3,), (21,), (1,), (9,)])
    plans, mp, S, V0, Sc, Vc = _group(fs, scen, lu)
    mp.set_scenarios(per_item, smem)
    cfg = mp.config
    assert cfg["scenarios_per_item"] == per_item and cfg["shared_memory"] == smem
    assert cfg["items"] == sum(-(-s.shape[0] // per_item) for s in S)
    assert cfg["smem_bytes"] <= 200 * 1024 and (cfg["smem_items"] > 0) == (cfg["smem_bytes"] > 0)
    if not smem:
        assert cfg["smem_items"] == 0
    elif per_item <= 4:  # a few scenarios of a feeder fit in 200 KB
        assert cfg["smem_items"] > 0
    for w, b in [(1, 2), (4, 1)]:
        mp.set_config(w, b)
        v, it, st = mp.solve(Sc, Vc, TOL, 10)
        _check(fs, S, V0, v, it, st, exact)
    mp.close()


def test_multi_meshed_and_feeders_mixed():
    """A meshed 30-bus grid and two feeders in one group."""
    g, S0, V00 = case("mesh30_b64", batch=40)
    fs, scen = _feeders([(7,), (50,)])
    sc0 = gridgen.config_scenarios("mesh30_b64", g, batch=40)
    grids = [g] + fs
    plans, mp, S, V0, Sc, Vc = _group(grids, [sc0] + scen)
    v, it, st = mp.solve(Sc, Vc, TOL, 10)
    _check(grids, S, V0, v, it, st, True)
    mp.close()


def test_multi_autotune_and_graph_replay():
    fs, scen = _feeders([(40,), (9,), (70,)])
    plans, mp, S, V0, Sc, Vc = _group(fs, scen, "fp32")
    cfg = mp.autotune(Sc, Vc, TOL, 10)
    assert cfg["ms"] > 0 and 1 <= cfg["warps"] <= 16 and cfg["scenarios_per_item"] in (1, 2, 4, 8, 16, 32)
    out = mp._outs(Sc)
    a = mp.solve(Sc, Vc, TOL, 10, out=out)
    a = [t.clone() for t in a]
    b = mp.solve(Sc, Vc, TOL, 10, out=out)  # replayed graph
    assert all(torch.equal(x, y) for x, y in zip(a, b))
    Sc2 = Sc * 0.9  # new data, new buffers: graph rebuilt
    v, it, st = mp.solve(Sc2, Vc, TOL, 10)
    S2 = [s * 0.9 for s in S]
    _check(fs, S2, V0, v, it, st, False)
    mp.close()


def test_multi_rejects_bad_groups():
    pf = _pf()
    g = gridgen.make_grid("mesh30_b64")
    p_dense = pf.Plan.from_branches(g.n, g.f, g.t, g.r, g.x, g.b, g.bus_type)  # has a dense block
    with pytest.raises(pf.NrpfError):
        pf.MultiPlan([p_dense], [4])
    p64 = pf.Plan.from_branches(g.n, g.f, g.t, g.r, g.x, g.b, g.bus_type, dense_frac=1.0)
    p32 = pf.Plan.from_branches(g.n, g.f, g.t, g.r, g.x, g.b, g.bus_type, dense_frac=1.0, lu_precision="fp32")
    with pytest.raises(pf.NrpfError):
        pf.MultiPlan([p64, p32], [4, 4])
