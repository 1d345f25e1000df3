"""Seeded synthetic grids and load scenarios for batched Newton-Raphson power flow.

This module is shared by the CPU oracle and the CUDA path and holds none of the
method's arithmetic: it only draws topologies, branch parameters, bus types and
per-scenario injections from fixed seeds, in a documented draw order.  Nodal
admittance assembly, mismatch, Jacobian and solves live in the oracle and in the
library, separately.
"""
from .grids import (  # noqa: F401
    Grid,
    Scenarios,
    CONFIGS,
    make_grid,
    make_scenarios,
    make_feeders,
    config_grid,
    config_scenarios,
    bridges,
    n1_contingencies,
    n1_batch,
    N1_LEVELS,
)
