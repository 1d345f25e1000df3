"""ctypes binding of ``libnrpf.so`` (include/nrpf.h): argument marshalling only.

Every computation runs in the CUDA library; this module converts numpy /
torch objects into plain pointers and sizes.  Importing it fails loudly when
the shared library has not been built.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libnrpf.so")

NRPF_OK = 0
LU_FP64, LU_FP32 = 0, 1
ORDER_AMD, ORDER_NATURAL = 0, 1


class NrpfError(RuntimeError):
    pass


class pf_options(C.Structure):
    _fields_ = [("lu_precision", C.c_int), ("ordering", C.c_int), ("dense_frac", C.c_double),
                ("panel", C.c_int), ("max_batch", C.c_int), ("host_only", C.c_int),
                ("order_tries", C.c_int), ("dense_layout", C.c_int)]


class pf_plan_info(C.Structure):
    _fields_ = [("n", C.c_int), ("m", C.c_int), ("n_pv", C.c_int), ("n_pq", C.c_int),
                ("n_slack", C.c_int), ("nnz_ybus", C.c_int64), ("nnz_j", C.c_int64),
                ("nnz_lu", C.c_int64), ("sparse_cols", C.c_int), ("dense_dim", C.c_int),
                ("dense_pad", C.c_int), ("lu_levels", C.c_int), ("fwd_levels", C.c_int),
                ("bwd_levels", C.c_int), ("lu_fma", C.c_double), ("solve_fma", C.c_double),
                ("capacity", C.c_int), ("lu_precision", C.c_int), ("panel", C.c_int),
                ("order_seed", C.c_int), ("order_key", C.c_int), ("dense_layout", C.c_int)]


NKCLASSES = 16


class pf_profile(C.Structure):
    _fields_ = [("launches", C.c_int64 * NKCLASSES), ("timed", C.c_int64 * NKCLASSES),
                ("ms", C.c_double * NKCLASSES)]


EXPORTS = ["pf_options_default", "pf_ybus_from_branches", "pf_plan_create", "pf_plan_get_info",
           "pf_plan_get_pattern", "pf_solve_batch", "pf_solve_batch_host", "pf_solve_batch_y", "pf_ybus_values", "pf_plan_set_branches", "pf_solve_batch_outages", "pf_branch_flows", "pf_solve_pivoting_host", "pf_retry_failed", "pf_solve_batch_cpu", "pf_stage_mismatch", "pf_stage_factor",
           "pf_stage_linear_solve", "pf_profile_start", "pf_profile_read", "pf_kernel_class_name",
           "pf_fma_peak", "pf_stage_mismatch_noalloc", "pf_multi_create", "pf_multi_solve",
           "pf_multi_set_config", "pf_multi_get_config", "pf_multi_set_scenarios", "pf_multi_get_scenarios", "pf_multi_autotune", "pf_multi_destroy",
           "pf_mlp_create", "pf_mlp_set_norm", "pf_mlp_fit_norm", "pf_mlp_params", "pf_mlp_grads",
           "pf_mlp_predict", "pf_mlp_train_step", "pf_mlp_error", "pf_mlp_destroy", "pf_gemm_bf16",
           "pf_gemm_set_variant",
           "pf_warmstart_features", "pf_warmstart_targets", "pf_warmstart_v0", "pf_warmstart_screen",
           "pf_plan_destroy", "pf_status_str"]


def _load():
    if not os.path.exists(LIB_PATH):
        raise NrpfError(f"{LIB_PATH} is missing: build it with "
                        "`python paper_2101_02270_gb300/build.py` (no CPU fallback exists)")
    lib = C.CDLL(LIB_PATH)
    P, I, D, I64 = C.c_void_p, C.c_int, C.c_double, C.c_int64
    lib.pf_options_default.argtypes = [C.POINTER(pf_options)]
    lib.pf_ybus_from_branches.argtypes = [I, I, P, P, P, P, P, P, P, P, P, I64, C.POINTER(I64)]
    lib.pf_plan_create.argtypes = [I, P, P, P, P, P, C.POINTER(pf_options), C.POINTER(C.c_void_p)]
    lib.pf_plan_get_info.argtypes = [P, C.POINTER(pf_plan_info)]
    lib.pf_plan_get_pattern.argtypes = [P, P, P, P, C.POINTER(I64)]
    lib.pf_solve_batch.argtypes = [P, I, P, P, D, I, P, P, P, P]
    lib.pf_solve_batch_host.argtypes = [P, I, P, P, D, I, P, P, P, I, P]
    lib.pf_solve_batch_y.argtypes = [P, I, P, P, P, D, I, P, P, P, P]
    lib.pf_ybus_values.argtypes = [I, I, P, P, P, P, P, I, P, P, P, P]
    lib.pf_plan_set_branches.argtypes = [P, I, P, P, P, P, P]
    lib.pf_solve_batch_outages.argtypes = [P, I, P, I, P, P, D, I, P, P, P, P]
    lib.pf_branch_flows.argtypes = [I, I, P, P, P, P, P, I, P, P, P, P, P]
    lib.pf_solve_pivoting_host.argtypes = [P, I, P, P, D, I, P, P, P]
    lib.pf_solve_batch_cpu.argtypes = [P, I, P, P, D, I, P, P, P, I]
    lib.pf_retry_failed.argtypes = [P, I, P, P, D, I, P, P, P, C.POINTER(I), P]
    lib.pf_stage_mismatch.argtypes = [P, I, P, P, P, P, P]
    lib.pf_stage_factor.argtypes = [P, I, P, I, P, P]
    lib.pf_stage_linear_solve.argtypes = [P, I, P, P, P, P]
    lib.pf_profile_start.argtypes = [P, C.c_uint32]
    lib.pf_profile_read.argtypes = [P, C.POINTER(pf_profile)]
    lib.pf_kernel_class_name.argtypes = [I]
    lib.pf_kernel_class_name.restype = C.c_char_p
    lib.pf_fma_peak.argtypes = [C.POINTER(D), C.POINTER(D), P]
    lib.pf_stage_mismatch_noalloc.argtypes = [P, I, P, P, P, P, P]
    lib.pf_multi_create.argtypes = [I, P, P, C.POINTER(C.c_void_p)]
    lib.pf_multi_solve.argtypes = [P, P, P, D, I, P, P, P, P]
    lib.pf_multi_set_config.argtypes = [P, I, I]
    lib.pf_multi_get_config.argtypes = [P, C.POINTER(I), C.POINTER(I), C.POINTER(I64), C.POINTER(I)]
    lib.pf_multi_autotune.argtypes = [P, P, P, D, I, P, P, P, P, C.POINTER(D)]
    lib.pf_multi_set_scenarios.argtypes = [P, I, I]
    lib.pf_multi_get_scenarios.argtypes = [P, C.POINTER(I), C.POINTER(I), C.POINTER(I64), C.POINTER(I)]
    lib.pf_multi_destroy.argtypes = [P]
    lib.pf_multi_destroy.restype = None
    lib.pf_mlp_create.argtypes = [I, I, I, I, I, C.c_uint64, C.POINTER(C.c_void_p)]
    lib.pf_mlp_set_norm.argtypes = [P, P, P, P, P]
    lib.pf_mlp_fit_norm.argtypes = [P, I64, P, P, P]
    lib.pf_mlp_params.argtypes = [P, I, P]
    lib.pf_mlp_grads.argtypes = [P, P]
    lib.pf_mlp_predict.argtypes = [P, I, P, P, P]
    lib.pf_mlp_train_step.argtypes = [P, I, P, P, C.c_float, C.c_float, I, P, P]
    lib.pf_mlp_error.argtypes = [P]
    lib.pf_mlp_destroy.argtypes = [P]
    lib.pf_mlp_destroy.restype = None
    lib.pf_gemm_bf16.argtypes = [P, P, P, I, I, I, I, P, P]
    lib.pf_gemm_set_variant.argtypes = [I]
    lib.pf_warmstart_features.argtypes = [I, I, P, P, P]
    lib.pf_warmstart_targets.argtypes = [I, I, P, I, P, P, P]
    lib.pf_warmstart_v0.argtypes = [I, I, P, P, I, P, P, P, P]
    lib.pf_warmstart_screen.argtypes = [I, I, P, P, C.c_double, P, P]
    lib.pf_plan_destroy.argtypes = [P]
    lib.pf_plan_destroy.restype = None
    lib.pf_status_str.argtypes = [I]
    lib.pf_status_str.restype = C.c_char_p
    return lib


lib = _load()


def check(rc: int, what: str = "") -> None:
    if rc != NRPF_OK:
        raise NrpfError(f"{what}: {lib.pf_status_str(rc).decode()} ({rc})")


def _np_ptr(a: np.ndarray):
    return C.c_void_p(a.ctypes.data)


def ybus_from_branches(n, f, t, r, x, b):
    """Ybus in CRS from branch data (pi model), computed by the library on the host."""
    f = np.ascontiguousarray(f, np.int32)
    t = np.ascontiguousarray(t, np.int32)
    r = np.ascontiguousarray(r, np.float64)
    x = np.ascontiguousarray(x, np.float64)
    b = np.ascontiguousarray(b, np.float64)
    nbr = f.shape[0]
    cap = n + 2 * nbr
    rowptr = np.zeros(n + 1, np.int32)
    colidx = np.zeros(cap, np.int32)
    yre = np.zeros(cap)
    yim = np.zeros(cap)
    nnz = C.c_int64(0)
    check(lib.pf_ybus_from_branches(n, nbr, _np_ptr(f), _np_ptr(t), _np_ptr(r), _np_ptr(x), _np_ptr(b),
                                    _np_ptr(rowptr), _np_ptr(colidx), _np_ptr(yre), _np_ptr(yim), cap,
                                    C.byref(nnz)), "pf_ybus_from_branches")
    k = nnz.value
    return rowptr, colidx[:k].copy(), yre[:k].copy(), yim[:k].copy()


def ybus_values(n, f, t, r, x, b, rowptr, colidx, in_service=None):
    """Ybus values [B, nnz] complex128 of B branch-status cases on a given CRS
    pattern (in_service [B, nbr] bool; None = one case, all in service),
    computed by the library on the host."""
    f = np.ascontiguousarray(f, np.int32)
    t = np.ascontiguousarray(t, np.int32)
    r = np.ascontiguousarray(r, np.float64)
    x = np.ascontiguousarray(x, np.float64)
    b = np.ascontiguousarray(b, np.float64)
    rowptr = np.ascontiguousarray(rowptr, np.int32)
    colidx = np.ascontiguousarray(colidx, np.int32)
    nbr = f.shape[0]
    ins = None if in_service is None else np.ascontiguousarray(in_service, np.uint8).reshape(-1, nbr)
    B = 1 if ins is None else ins.shape[0]
    y = np.zeros((B, int(rowptr[n])), np.complex128)
    check(lib.pf_ybus_values(n, nbr, _np_ptr(f), _np_ptr(t), _np_ptr(r), _np_ptr(x), _np_ptr(b), B,
                             None if ins is None else _np_ptr(ins), _np_ptr(rowptr), _np_ptr(colidx),
                             _np_ptr(y)), "pf_ybus_values")
    return y


def fma_peak(stream=None):
    """(fp64, fp32) FMA throughput of the current device in TFLOP/s."""
    a, b = C.c_double(0), C.c_double(0)
    check(lib.pf_fma_peak(C.byref(a), C.byref(b), stream), "pf_fma_peak")
    return a.value, b.value
