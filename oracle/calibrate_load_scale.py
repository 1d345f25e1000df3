"""Find the global load scale (lambda) of each synthetic configuration.

TEST INFRASTRUCTURE: calls only the oracle and the seeded generators.  For each
configuration it tries lambda = 1, 1/2, 1/4, ... and keeps the first value for
which the FP64 oracle converges from flat start (tol 1e-8, maxit 10) both for
the base loading (all factors 1) and for every bus at the top of its scenario
range, with min |V| >= 0.8 p.u.  The values printed here are the ``load_scale``
entries of ``gridgen.grids``.

usage: python -m oracle.calibrate_load_scale [name ...]
"""
import sys

import numpy as np

import gridgen
from gridgen.grids import CONFIGS, FEEDERS, Scenarios
from oracle.nrpf import make_ybus, newton, STATUS_CONVERGED


def _ok(g, Y, lam, hi):
    for fac in (1.0, hi):
        sc = Scenarios(np.full((1, g.n), fac), lam)
        V, it, st = newton(Y, sc.sbus(g)[0], sc.v0_flat(g)[0], g.bus_type, 1e-8, 10)
        if st != STATUS_CONVERGED or np.abs(V).min() < 0.8:
            return False
    return True


def calibrate(g, hi):
    Y = make_ybus(g.n, g.f, g.t, g.r, g.x, g.b)
    for k in range(12):
        lam = 2.0 ** -k
        if _ok(g, Y, lam, hi):
            return lam
    raise RuntimeError("no load scale found")


def main(names):
    for name in names:
        if name == "feeders":
            gs = gridgen.make_feeders()
            lam = min(calibrate(g, FEEDERS["scen"][1]) for g in gs)
        else:
            g = gridgen.make_grid(name)
            lam = calibrate(g, CONFIGS[name]["scen"][1])
        print(f"{name}: load_scale = {lam}")


if __name__ == "__main__":
    main(sys.argv[1:] or list(CONFIGS) + ["feeders"])
