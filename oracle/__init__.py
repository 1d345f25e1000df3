"""CPU FP64 oracle for batched Newton-Raphson AC power flow.

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, obviously correct
restatement of what the GPU library computes; it shares no code with the CUDA
path and is imported only by ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference arm of ``bench.py``.  The product path never calls it.

Pinned by ``tests/test_oracle_pins.py`` against closed forms (two-bus line),
the power-balance invariant, finite differences, an independent Gauss-Seidel
power flow and a library dense solve.
"""
from .nrpf import (  # noqa: F401
    STATUS_CONVERGED,
    STATUS_MAXIT,
    STATUS_FAILED,
    make_ybus,
    bus_sets,
    power_injection,
    mismatch,
    jacobian,
    lu_partial_pivot,
    lu_solve,
    newton,
    newton_batch,
)
