"""Static N-1 contingency inputs (no GPU): the connected-outage list against a
brute-force connectivity check, and the library's per-case Ybus values on a
shared pattern against the oracle's assembly of each post-outage grid."""
import numpy as np
import pytest
import scipy.sparse as sp
from scipy.sparse.csgraph import connected_components

import gridgen
from oracle import nrpf


def _pf():
    return pytest.importorskip("paper_2101_02270_gb300")


def _connected(n, f, t):
    a = sp.coo_matrix((np.ones(len(f)), (f, t)), shape=(n, n))
    return connected_components(a, directed=False)[0] == 1


@pytest.mark.parametrize("name", ["mesh30_b64", "mesh2000_b10k"])
def test_bridges_match_brute_force(name):
    g = gridgen.make_grid(name)
    br = gridgen.bridges(g.n, g.f, g.t)
    rng = np.random.default_rng(0)
    idx = np.arange(g.n_branch) if g.n_branch <= 64 else rng.choice(g.n_branch, 64, replace=False)
    for e in idx:
        keep = np.arange(g.n_branch) != e
        assert br[e] == (not _connected(g.n, g.f[keep], g.t[keep]))


def test_bridges_of_a_tree_and_a_cycle():
    # path 0-1-2-3 plus chord 1-3: branches 0-1 is a bridge, the cycle 1-2-3 is not
    f = np.array([0, 1, 2, 1])
    t = np.array([1, 2, 3, 3])
    assert gridgen.bridges(4, f, t).tolist() == [True, False, False, False]
    # parallel branches are never bridges
    assert gridgen.bridges(2, np.array([0, 0]), np.array([1, 1])).tolist() == [False, False]


@pytest.mark.parametrize("name", ["mesh30_b64", "mesh2000_b10k"])
def test_case_ybus_values_match_oracle_assembly(name):
    pf = _pf()
    g = gridgen.make_grid(name)
    outage, level, ins, sbus = gridgen.n1_batch(g)
    rng = np.random.default_rng(1)
    pick = rng.choice(len(outage), 6, replace=False)
    plan = pf.Plan.from_branches(g.n, g.f, g.t, g.r, g.x, g.b, g.bus_type, host_only=True)
    Y = plan.ybus_values(ins[pick])
    rowptr, colidx = plan._rowptr, plan._colidx
    rows = np.repeat(np.arange(g.n), np.diff(rowptr))
    for k, c in enumerate(pick):
        keep = ins[c]
        Yo = nrpf.make_ybus(g.n, g.f[keep], g.t[keep], g.r[keep], g.x[keep], g.b[keep]).toarray()
        dense = np.zeros((g.n, g.n), complex)
        dense[rows, colidx] = Y[k]
        assert np.max(np.abs(dense - Yo)) < 1e-12
    # all in service: the plan's own values
    Y0 = plan.ybus_values(np.ones((1, g.n_branch), bool))[0]
    assert np.max(np.abs(Y0 - (plan._yre + 1j * plan._yim))) < 1e-12
    plan.close()
