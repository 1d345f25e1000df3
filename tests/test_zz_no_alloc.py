"""pf_stage_mismatch_noalloc: the mismatch entry point for callers that cannot
allocate device memory (their GPU memory belongs to another allocator, or they
cannot afford cudaMalloc's latency and implicit synchronisation).  Its F and
max|F| must match the oracle's mismatch (oracle/nrpf.py) and the staged
pf_stage_mismatch, which computes them through the plan's workspace, on
consecutive calls that share its static scratch array; and a call must leave
the device's free memory unchanged.  Named to run last in the suite."""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import nrpf  # noqa: E402
from tests.common import case, oracle_ybus, perturbed  # noqa: E402

pytestmark = pytest.mark.gpu

TOL = 1e-10  # the mismatch tolerance of the parity tests


def _pf():
    import paper_2101_02270_gb300 as pf
    return pf


def _noalloc(plan, S, V, out=None):
    pf = _pf()
    B, m = S.shape[0], plan.info["m"]
    if out is None:
        out = (torch.full((B, m), float("nan"), dtype=torch.float64, device="cuda"),
               torch.full((B,), float("nan"), dtype=torch.float64, device="cuda"))
    F, norm = out
    rc = pf.lib.pf_stage_mismatch_noalloc(plan._h, B, C.c_void_p(S.data_ptr()), C.c_void_p(V.data_ptr()),
                                         C.c_void_p(F.data_ptr()), C.c_void_p(norm.data_ptr()),
                                         C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0, pf.lib.pf_status_str(rc)
    return F, norm


@pytest.mark.parametrize("name,B,lu", [("mesh30_b64", 64, "fp64"), ("mesh2000_b10k", 45, "fp64"),
                                       ("mesh2000_b10k", 45, "fp32")])
def test_noalloc_mismatch_matches_oracle_and_staged_entry_point(name, B, lu):
    pf = _pf()
    g, S, V0 = case(name, batch=B)
    plan = pf.Plan.from_branches(g.n, g.f, g.t, g.r, g.x, g.b, g.bus_type, lu_precision=lu)
    pos, _, _ = plan.pattern()
    Y = oracle_ybus(g)
    _, pv, pq, _ = nrpf.bus_sets(g.bus_type)
    Sd = torch.from_numpy(S).cuda()
    # two calls in a row; the second has much smaller mismatches, so maxima
    # left over from the first call would show up in its norms
    for V in (perturbed(V0, seed=11, mag=0.05, ang=0.1), perturbed(V0, seed=12, mag=1e-4, ang=1e-4)):
        Vd = torch.from_numpy(V).cuda()
        Fn, nn = _noalloc(plan, Sd, Vd)
        Fs, ns = plan.stage_mismatch(Sd, Vd)
        Fn, nn, Fs, ns = Fn.cpu().numpy()[:, pos], nn.cpu().numpy(), Fs.cpu().numpy(), ns.cpu().numpy()
        for b in range(B):
            Fo = nrpf.mismatch(Y, V[b], S[b], pv, pq)
            assert np.max(np.abs(Fn[b] - Fo)) < TOL
            assert abs(nn[b] - np.max(np.abs(Fo))) < TOL
        assert np.max(np.abs(nn - ns)) < TOL
        if lu == "fp64":
            assert np.max(np.abs(Fn - Fs)) < TOL
        else:
            # the staged F of an FP32-LU plan is rounded to float32
            assert np.all(np.abs(Fn - Fs) <= 2.0 ** -24 * np.abs(Fn) + 1e-30)
    plan.close()


def test_noalloc_calls_leave_device_memory_unchanged():
    """After one warm-up call (module load), repeated calls on a batch whose
    staged workspace would take hundreds of MB leave cudaMemGetInfo's free
    bytes as they were; the staged entry point on a fresh plan, for contrast,
    takes that workspace."""
    pf = _pf()
    g, S, V0 = case("mesh2000_b10k", batch=512)
    Sd = torch.from_numpy(S).cuda()
    Vd = torch.from_numpy(perturbed(V0, seed=13)).cuda()
    plan = pf.Plan.from_branches(g.n, g.f, g.t, g.r, g.x, g.b, g.bus_type)
    out = (torch.empty((512, plan.info["m"]), dtype=torch.float64, device="cuda"),
           torch.empty(512, dtype=torch.float64, device="cuda"))
    _noalloc(plan, Sd, Vd, out)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(5):
        _noalloc(plan, Sd, Vd, out)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    plan.close()
    fresh = pf.Plan.from_branches(g.n, g.f, g.t, g.r, g.x, g.b, g.bus_type)
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    fresh.stage_mismatch(Sd, Vd)
    torch.cuda.synchronize()
    assert free1 - torch.cuda.mem_get_info()[0] > 100 * 2 ** 20
    fresh.close()


def test_noalloc_rejects_oversized_batch():
    pf = _pf()
    g, S, V0 = case("mesh30_b64", batch=2)
    plan = pf.Plan.from_branches(g.n, g.f, g.t, g.r, g.x, g.b, g.bus_type)
    too_many = 65536 + 1
    rc = pf.lib.pf_stage_mismatch_noalloc(plan._h, too_many, None, None, None, None, None)
    assert rc == -5  # NRPF_ERR_CAPACITY
    assert pf.lib.pf_stage_mismatch_noalloc(plan._h, 0, None, None, None, None, None) == 0
    plan.close()
