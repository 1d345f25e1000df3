"""Batched Newton-Raphson AC power flow on GB300 (sm_103a).

Many power flows that share one Ybus sparsity pattern are solved at once by
hand-written CUDA kernels behind a C ABI (include/nrpf.h): nodal power
mismatch, Jacobian refill into a permuted LU workspace, sparse + dense LU
refactorisation, forward/backward substitution and the voltage update.
"""
from ._lib import NrpfError, lib, ybus_from_branches  # noqa: F401
from .solver import MultiPlan, Plan  # noqa: F401

STATUS = {0: "converged", 1: "maxit", 2: "failed"}
