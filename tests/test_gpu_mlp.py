"""Learned warm start on the GPU: the tcgen05 BF16 GEMM against a PyTorch FP32
reference, the network's forward/backward against the FP64 CPU reference
(oracle/mlp.py), the AdamW update, and the end-to-end gain of a trained
network over flat start on the 2,000-bus grid."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import gridgen  # noqa: E402
from oracle import mlp as omlp  # noqa: E402
from oracle import nrpf  # noqa: E402
from tests.common import oracle_ybus  # noqa: E402

pytestmark = pytest.mark.gpu


def _ws():
    import paper_2101_02270_gb300.warmstart as ws
    return ws


@pytest.mark.parametrize("variant", [0, 1])
@pytest.mark.parametrize("M,N,K", [(128, 128, 64), (256, 384, 192), (512, 1024, 4096), (1024, 256, 1024),
                                   (128, 256, 320)])
def test_tc_gemm_matches_fp32_reference(M, N, K, variant):
    ws = _ws()
    g = torch.Generator(device="cuda").manual_seed(M + N + K)
    A = torch.randn(M, K, device="cuda", generator=g).to(torch.bfloat16)
    B = torch.randn(N, K, device="cuda", generator=g).to(torch.bfloat16)
    C, err = ws.gemm_bf16(A, B, variant)
    torch.cuda.synchronize()
    assert err.item() == 0
    ref = A.float() @ B.float().T
    assert ((C - ref).abs().max() / ref.abs().max()).item() < 5e-4


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


def test_mlp_forward_backward_vs_fp64_reference():
    ws = _ws()
    nin, nh1, nh2, nout, B = 200, 128, 256, 90, 96
    rng = np.random.default_rng(0)
    net = ws.MLP(nin, nh1, nh2, nout, bmax=128, seed=1)
    shapes = [(nh1, nin), (nh1,), (nh2, nh1), (nh2,), (nout, nh2), (nout,)]
    fan = [nin, nin, nh1, nh1, nh2, nh2]
    P = [(rng.standard_normal(s) / np.sqrt(f)).astype(np.float32) for s, f in zip(shapes, fan)]
    net.set_params(P)
    X = rng.standard_normal((B, nin)).astype(np.float32)
    T = rng.standard_normal((B, nout)).astype(np.float32)
    Xd, Td = torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda()
    Y = net.predict(Xd).cpu().numpy()
    loss = net.train_step(Xd, Td, update=False).cpu().numpy()[0]
    G = net.grads()
    assert net.error() == 0
    Po = [P[0].T.astype(np.float64), P[1].astype(np.float64), P[2].T.astype(np.float64), P[3].astype(np.float64),
          P[4].T.astype(np.float64), P[5].astype(np.float64)]
    Yo, cache = omlp.forward(Po, X.astype(np.float64))
    Go = omlp.backward(Po, cache, Yo, T.astype(np.float64))
    assert _rel(Y, Yo) < 1e-2
    assert abs(loss - omlp.loss(Yo, T)) / omlp.loss(Yo, T) < 2e-2
    for k, (g, go) in enumerate(zip(G, Go)):
        go = go.T if go.ndim == 2 else go
        assert _rel(g, go) < 3e-2, (k, _rel(g, go))


def test_mlp_adamw_update():
    """Six AdamW steps on the GPU against oracle.mlp.adamw_step, element by
    element after every step.  The oracle keeps its own FP64 moments from
    zero and takes the gradients the GPU computed at its own weights, so the
    bias corrections of steps 2..6 and the changing learning rate are checked
    as well as the first step."""
    ws = _ws()
    nin, nh1, nh2, nout, B = 64, 128, 128, 40, 50
    rng = np.random.default_rng(2)
    net = ws.MLP(nin, nh1, nh2, nout, bmax=64, seed=3)
    P = [p.astype(np.float64) for p in net.params()]
    M = [np.zeros_like(p) for p in P]
    V = [np.zeros_like(p) for p in P]
    wd = 0.01
    for step in range(1, 7):
        X = torch.from_numpy(rng.standard_normal((B, nin)).astype(np.float32)).cuda()
        T = torch.from_numpy(rng.standard_normal((B, nout)).astype(np.float32)).cuda()
        lr = 1e-3 * (1.0 + 0.25 * step)
        net.train_step(X, T, lr=lr, wd=wd, update=True)
        G = net.grads()
        P1 = net.params()
        assert net.error() == 0
        for k, (g, p1) in enumerate(zip(G, P1)):
            omlp.adamw_step(P[k], g.astype(np.float64), M[k], V[k], step, lr=lr, wd=wd if k % 2 == 0 else 0.0)
            assert np.max(np.abs(P[k] - p1)) < 1e-6 * step, (step, k, np.max(np.abs(P[k] - p1)))


def test_warm_start_gain_on_2000_bus_grid():
    """Train on solver-made solutions (8,192 scenarios), then solve 512
    held-out scenarios from the network's guess: every instance converges to
    the same solution as from flat start, in fewer Newton iterations."""
    import paper_2101_02270_gb300 as pf
    ws = _ws()
    g = gridgen.make_grid("mesh2000_b10k")
    plan = pf.Plan.from_branches(g.n, g.f, g.t, g.r, g.x, g.b, g.bus_type)
    tr = gridgen.config_scenarios("mesh2000_b10k", g, batch=8192, seed=2)
    S = torch.from_numpy(tr.sbus(g)).cuda()
    Vf = torch.from_numpy(tr.v0_flat(g)).cuda()
    V, it, st = plan.solve(S, Vf, 1e-8, 10)
    assert bool((st == 0).all())
    nns = int(np.sum(g.bus_type != 3))
    net = ws.MLP(2 * g.n, 1024, 1024, 2 * nns, bmax=1024, seed=0)
    w = ws.WarmStart(plan, g.bus_type, net)
    X, T = w.features(S), w.targets(V)
    net.fit_norm(X, T)
    gen = torch.Generator(device="cuda").manual_seed(0)
    for step in range(300):
        idx = torch.randint(0, X.shape[0], (1024,), device="cuda", generator=gen)
        loss = net.train_step(X[idx].contiguous(), T[idx].contiguous(), lr=1e-3 if step < 200 else 3e-4)
    assert net.error() == 0
    assert float(loss.item()) < 0.2
    ho = gridgen.config_scenarios("mesh2000_b10k", g, batch=512, seed=1)
    Sh = torch.from_numpy(ho.sbus(g)).cuda()
    Vh = torch.from_numpy(ho.v0_flat(g)).cuda()
    vf, itf, stf = plan.solve(Sh, Vh, 1e-8, 10)
    vw, itw, stw, fb = w.solve(Sh, Vh, 1e-8, 10)
    assert bool((stf == 0).all()) and bool((stw == 0).all())
    assert float((vw - vf).abs().max()) < 1e-6
    assert itw.float().mean() < itf.float().mean() - 0.5
    # the guess is a physical voltage profile: check one instance with the oracle
    Y = oracle_ybus(g)
    _, pv, pq, _ = nrpf.bus_sets(g.bus_type)
    F = nrpf.mismatch(Y, vw[0].cpu().numpy(), Sh[0].cpu().numpy(), pv, pq)
    assert np.max(np.abs(F)) < 1e-8


def test_mlp_checkpoint_roundtrip(tmp_path):
    ws = _ws()
    a = ws.MLP(64, 128, 128, 40, bmax=64, seed=5)
    b = ws.MLP(64, 128, 128, 40, bmax=64, seed=6)
    norm = [np.full(64, 0.5), np.full(64, 2.0), np.zeros(40), np.ones(40)]
    a.set_norm(*norm)
    a.save(tmp_path / "w.npz", norm=norm)
    b.load(tmp_path / "w.npz")
    X = torch.from_numpy(np.random.default_rng(0).standard_normal((16, 64)).astype(np.float32)).cuda()
    assert torch.equal(a.predict(X), b.predict(X))
    for p, q in zip(a.params(), b.params()):
        assert np.array_equal(p, q)


def test_warm_start_falls_back_to_flat_start():
    """A network whose guesses are useless (angles far off) makes Newton fail
    from them; those instances are re-solved from flat start and reach the
    flat-start solutions."""
    import paper_2101_02270_gb300 as pf
    ws = _ws()
    g = gridgen.make_grid("mesh30_b64")
    plan = pf.Plan.from_branches(g.n, g.f, g.t, g.r, g.x, g.b, g.bus_type)
    nns = int(np.sum(g.bus_type != 3))
    net = ws.MLP(2 * g.n, 128, 128, 2 * nns, bmax=64, seed=0)
    arrs = [np.zeros_like(a) for a in net.params()]
    arrs[5][:nns] = 0.05            # |V| guess of 0.05 p.u. (far from the solution)
    arrs[5][nns:] = 3.0             # angles of 3 rad
    net.set_params(arrs)
    w = ws.WarmStart(plan, g.bus_type, net)
    sc = gridgen.config_scenarios("mesh30_b64", g, batch=64)
    S = torch.from_numpy(sc.sbus(g)).cuda()
    Vf = torch.from_numpy(sc.v0_flat(g)).cuda()
    v, it, st, fb = w.solve(S, Vf, 1e-8, 10)
    vf, itf, stf = plan.solve(S, Vf, 1e-8, 10)
    assert bool((st == 0).all())
    assert int(fb.sum()) > 0
    # every fallback instance equals the flat-start result exactly
    assert torch.equal(v[fb], vf[fb]) and torch.equal(it[fb], itf[fb])


def test_warm_start_low_voltage_root_is_redone_from_flat_start():
    """Newton from a guess with one load bus at 0.1 p.u. converges on the
    30-bus grid, but to a low-voltage root of the power-flow equations
    (min |V| of a few hundredths).  The screen flags those instances and they
    are re-solved from flat start: every result is then the flat-start
    solution, which the oracle confirms."""
    import paper_2101_02270_gb300 as pf
    ws = _ws()
    g = gridgen.make_grid("mesh30_b64")
    plan = pf.Plan.from_branches(g.n, g.f, g.t, g.r, g.x, g.b, g.bus_type)
    ns = np.flatnonzero(g.bus_type != 3)
    nns = ns.size
    low_bus = int(np.flatnonzero(g.bus_type == 1)[0])
    net = ws.MLP(2 * g.n, 128, 128, 2 * nns, bmax=64, seed=0)
    arrs = [np.zeros_like(a) for a in net.params()]
    arrs[5][:nns] = 1.0                                  # flat magnitudes ...
    arrs[5][int(np.flatnonzero(ns == low_bus)[0])] = 0.1  # ... but one load bus at 0.1 p.u.
    net.set_params(arrs)
    w = ws.WarmStart(plan, g.bus_type, net)
    sc = gridgen.config_scenarios("mesh30_b64", g, batch=64)
    S_np, V0_np = sc.sbus(g), sc.v0_flat(g)
    S = torch.from_numpy(S_np).cuda()
    Vf = torch.from_numpy(V0_np).cuda()
    # the planted guess: Newton converges, to the wrong root, for some instances
    vg, itg, stg = plan.solve(S, w.guess(S, Vf), 1e-8, 10)
    low = (stg == 0) & (vg.abs().min(dim=1).values < 0.5)
    assert int(low.sum()) > 0
    v, it, st, fb = w.solve(S, Vf, 1e-8, 10)
    assert bool(fb[low].all())
    vf, itf, stf = plan.solve(S, Vf, 1e-8, 10)
    assert torch.equal(v[fb], vf[fb]) and torch.equal(it[fb], itf[fb])
    Vo, ito, sto = nrpf.newton_batch(oracle_ybus(g), S_np, V0_np, g.bus_type, 1e-8, 10)
    assert np.array_equal(st.cpu().numpy(), sto)
    assert np.max(np.abs(v.cpu().numpy() - Vo)) < 1e-6
    # the screen itself: status, non-finite values and the floor
    vt = torch.ones((3, 4), dtype=torch.complex128, device="cuda")
    vt[1, 2] = 0.3
    vt[2, 0] = float("nan")
    stt = torch.tensor([0, 0, 0], dtype=torch.uint8, device="cuda")
    w4 = ws.WarmStart.__new__(ws.WarmStart)
    w4.n = 4
    assert w4.screen(vt, stt, 0.5).tolist() == [False, True, True]
    stt[0] = 1
    assert w4.screen(vt, stt, 0.0).tolist() == [True, False, True]
