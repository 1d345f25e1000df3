"""pf_stage_mismatch_noalloc: the mismatch entry point for callers that cannot
allocate device memory (their GPU memory belongs to another allocator, or they
cannot afford cudaMalloc's latency and implicit synchronisation).  It must give
the same F and max|F| as pf_stage_mismatch, which stages the same computation
through the plan's workspace, on consecutive calls that share its static
scratch array.  Named to run last in the suite."""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from tests.common import case, perturbed  # noqa: E402

pytestmark = pytest.mark.gpu

TOL = 1e-10  # the mismatch tolerance of the parity tests


def _pf():
    import paper_2101_02270_gb300 as pf
    return pf


def _noalloc(plan, S, V):
    pf = _pf()
    B, m = S.shape[0], plan.info["m"]
    F = torch.full((B, m), float("nan"), dtype=torch.float64, device="cuda")
    norm = torch.full((B,), float("nan"), dtype=torch.float64, device="cuda")
    rc = pf.lib.pf_stage_mismatch_noalloc(plan._h, B, C.c_void_p(S.data_ptr()), C.c_void_p(V.data_ptr()),
                                         C.c_void_p(F.data_ptr()), C.c_void_p(norm.data_ptr()),
                                         C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0, pf.lib.pf_status_str(rc)
    return F, norm


@pytest.mark.parametrize("name,B", [("mesh30_b64", 64), ("mesh2000_b10k", 45)])
def test_noalloc_mismatch_matches_staged_entry_point(name, B):
    pf = _pf()
    g, S, V0 = case(name, batch=B)
    plan = pf.Plan.from_branches(g.n, g.f, g.t, g.r, g.x, g.b, g.bus_type)
    pos, _, _ = plan.pattern()
    Sd = torch.from_numpy(S).cuda()
    # two calls in a row; the second has much smaller mismatches, so maxima
    # left over from the first call would show up in its norms
    for V in (perturbed(V0, seed=11, mag=0.05, ang=0.1), perturbed(V0, seed=12, mag=1e-4, ang=1e-4)):
        Vd = torch.from_numpy(V).cuda()
        Fn, nn = _noalloc(plan, Sd, Vd)
        Fs, ns = plan.stage_mismatch(Sd, Vd)
        Fn, nn, Fs, ns = Fn.cpu().numpy(), nn.cpu().numpy(), Fs.cpu().numpy(), ns.cpu().numpy()
        assert np.max(np.abs(Fn[:, pos] - Fs)) < TOL
        assert np.max(np.abs(nn - ns)) < TOL
    plan.close()


def test_noalloc_rejects_oversized_batch():
    pf = _pf()
    g, S, V0 = case("mesh30_b64", batch=2)
    plan = pf.Plan.from_branches(g.n, g.f, g.t, g.r, g.x, g.b, g.bus_type)
    too_many = 65536 + 1
    rc = pf.lib.pf_stage_mismatch_noalloc(plan._h, too_many, None, None, None, None, None)
    assert rc == -5  # NRPF_ERR_CAPACITY
    assert pf.lib.pf_stage_mismatch_noalloc(plan._h, 0, None, None, None, None, None) == 0
    plan.close()
