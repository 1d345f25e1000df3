"""Python face of the batched Newton-Raphson library: a plan object whose
methods pass torch CUDA tensors (device memory, the caller's stream) to the C
ABI.  No arithmetic of the method happens here."""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import _lib
from ._lib import check, lib

_PREC = {"fp64": _lib.LU_FP64, "fp32": _lib.LU_FP32}
_ORDER = {"amd": _lib.ORDER_AMD, "natural": _lib.ORDER_NATURAL}
# dense-block storage: "auto" (instance-major for large FP32 blocks),
# "interleaved", "instance_major"
_LAYOUT = {"auto": 0, "interleaved": 1, "instance_major": 2}
KERNEL_CLASSES = [lib.pf_kernel_class_name(i).decode() for i in range(16)]


def _dptr(t: torch.Tensor) -> C.c_void_p:
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return C.c_void_p(t.data_ptr())


def _hptr(t: torch.Tensor) -> C.c_void_p:
    if t.device.type != "cpu":
        raise ValueError("expected a host tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return C.c_void_p(t.data_ptr())


def _stream() -> C.c_void_p:
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


class Plan:
    """Symbolic plan for one Ybus sparsity pattern (pf_plan_create)."""

    def __init__(self, n, rowptr, colidx, y_re, y_im, bus_type, lu_precision="fp64",
                 ordering="amd", dense_frac=0.0, panel=0, max_batch=0, host_only=False,
                 order_tries=0, dense_layout="auto"):
        self.n = int(n)
        self._rowptr = np.ascontiguousarray(rowptr, np.int32)
        self._colidx = np.ascontiguousarray(colidx, np.int32)
        self._yre = np.ascontiguousarray(y_re, np.float64)
        self._yim = np.ascontiguousarray(y_im, np.float64)
        self._bt = np.ascontiguousarray(bus_type, np.int8)
        opt = _lib.pf_options()
        lib.pf_options_default(C.byref(opt))
        opt.lu_precision = _PREC[lu_precision]
        opt.ordering = _ORDER[ordering]
        opt.dense_frac = float(dense_frac)
        opt.panel = int(panel)
        opt.max_batch = int(max_batch)
        opt.host_only = int(bool(host_only))
        opt.order_tries = int(order_tries)
        opt.dense_layout = _LAYOUT[dense_layout]
        h = C.c_void_p()
        check(lib.pf_plan_create(self.n, _lib._np_ptr(self._rowptr), _lib._np_ptr(self._colidx),
                                 _lib._np_ptr(self._yre), _lib._np_ptr(self._yim), _lib._np_ptr(self._bt),
                                 C.byref(opt), C.byref(h)), "pf_plan_create")
        self._h = h
        self.lu_precision = lu_precision

    @classmethod
    def from_branches(cls, n, f, t, r, x, b, bus_type, **kw):
        rowptr, colidx, yre, yim = _lib.ybus_from_branches(n, f, t, r, x, b)
        plan = cls(n, rowptr, colidx, yre, yim, bus_type, **kw)
        plan._branches = (f, t, r, x, b)
        return plan

    def ybus_values(self, in_service=None) -> np.ndarray:
        """Ybus values [B, nnz] complex128 on this plan's pattern for B
        branch-status cases (in_service [B, nbr] bool); the plan must come
        from from_branches."""
        f, t, r, x, b = self._branches
        return _lib.ybus_values(self.n, f, t, r, x, b, self._rowptr, self._colidx, in_service)

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib.pf_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    @property
    def info(self) -> dict:
        inf = _lib.pf_plan_info()
        check(lib.pf_plan_get_info(self._h, C.byref(inf)), "pf_plan_get_info")
        return {k: getattr(inf, k) for k, _ in _lib.pf_plan_info._fields_}

    def pattern(self):
        """(pos_of_unknown [m], colptr [m+1], rowidx [nnz]) of A = P J P^T."""
        m = self.info["m"]
        nnz = C.c_int64(0)
        check(lib.pf_plan_get_pattern(self._h, None, None, None, C.byref(nnz)), "pattern")
        pos = np.zeros(m, np.int32)
        colptr = np.zeros(m + 1, np.int64)
        rowidx = np.zeros(max(nnz.value, 1), np.int32)
        check(lib.pf_plan_get_pattern(self._h, _lib._np_ptr(pos), _lib._np_ptr(colptr),
                                      _lib._np_ptr(rowidx), C.byref(nnz)), "pattern")
        return pos, colptr, rowidx[:nnz.value]

    # ---- solves (device tensors, caller's current stream) ----
    def solve(self, sbus: torch.Tensor, v0: torch.Tensor, tol: float = 1e-8, maxit: int = 10,
              out=None):
        """Newton-Raphson for a batch: sbus, v0 complex128 [B, n] on the GPU.
        Returns (v [B, n] complex128, iters [B] int32, status [B] uint8)."""
        B = sbus.shape[0]
        self._check_bn(sbus, B)
        self._check_bn(v0, B)
        dev = sbus.device
        if out is None:
            v = torch.empty((B, self.n), dtype=torch.complex128, device=dev)
            iters = torch.empty(B, dtype=torch.int32, device=dev)
            status = torch.empty(B, dtype=torch.uint8, device=dev)
        else:
            v, iters, status = out
        check(lib.pf_solve_batch(self._h, B, _dptr(sbus), _dptr(v0), float(tol), int(maxit), _dptr(v),
                                 _dptr(iters), _dptr(status), _stream()), "pf_solve_batch")
        return v, iters, status

    def solve_pivoting_host(self, sbus: np.ndarray, v0: np.ndarray, tol: float = 1e-8, maxit: int = 10):
        """Newton-Raphson on the host cores with a pivoting sparse LU
        (pf_solve_pivoting_host): numpy complex128 [B, n] in, numpy
        (v, iters, status) out.  Works on host-only plans."""
        S = np.ascontiguousarray(sbus, np.complex128)
        V0 = np.ascontiguousarray(v0, np.complex128)
        B = S.shape[0]
        if S.shape != (B, self.n) or V0.shape != (B, self.n):
            raise ValueError(f"expected complex128 [{B}, {self.n}]")
        v = np.empty_like(S)
        it = np.empty(B, np.int32)
        st = np.empty(B, np.uint8)
        check(lib.pf_solve_pivoting_host(self._h, B, _lib._np_ptr(S), _lib._np_ptr(V0), float(tol), int(maxit),
                                         _lib._np_ptr(v), _lib._np_ptr(it), _lib._np_ptr(st)), "pf_solve_pivoting_host")
        return v, it, st

    def solve_cpu(self, sbus: np.ndarray, v0: np.ndarray, tol: float = 1e-8, maxit: int = 10, threads: int = 0):
        """Batched Newton-Raphson on the host cores (pf_solve_batch_cpu): numpy
        complex128 [B, n] in, numpy (v, iters, status) out.  Works on host-only
        plans."""
        S = np.ascontiguousarray(sbus, np.complex128)
        V0 = np.ascontiguousarray(v0, np.complex128)
        B = S.shape[0]
        if S.shape != (B, self.n) or V0.shape != (B, self.n):
            raise ValueError(f"expected complex128 [{B}, {self.n}]")
        v = np.empty_like(S)
        it = np.empty(B, np.int32)
        st = np.empty(B, np.uint8)
        check(lib.pf_solve_batch_cpu(self._h, B, _lib._np_ptr(S), _lib._np_ptr(V0), float(tol), int(maxit),
                                     _lib._np_ptr(v), _lib._np_ptr(it), _lib._np_ptr(st), int(threads)),
              "pf_solve_batch_cpu")
        return v, it, st

    def retry_failed(self, sbus: torch.Tensor, v0: torch.Tensor, out, tol: float = 1e-8, maxit: int = 10) -> int:
        """Second chance (pf_retry_failed): re-solve with the pivoting host
        solver every instance of a finished solve (device arrays sbus, v0 and
        out = (v, iters, status)) whose status is 2; returns how many."""
        B = sbus.shape[0]
        self._check_bn(sbus, B)
        self._check_bn(v0, B)
        v, iters, status = out
        n = C.c_int(0)
        check(lib.pf_retry_failed(self._h, B, _dptr(sbus), _dptr(v0), float(tol), int(maxit), _dptr(v),
                                  _dptr(iters), _dptr(status), C.byref(n), _stream()), "pf_retry_failed")
        return n.value

    def branch_flows(self, v: torch.Tensor, in_service: torch.Tensor = None):
        """Power entering every branch at its from and to ends (pf_branch_flows)
        for solved voltages v complex128 [B, n] on the GPU; in_service [B, nbr]
        bool/uint8 on the GPU or None.  The plan must come from from_branches.
        Returns (sf, st) complex128 [B, nbr]."""
        B = v.shape[0]
        self._check_bn(v, B)
        if getattr(self, "_dev_branches", None) is None or self._dev_branches[0].device != v.device:
            f, t, r, x, b = self._branches
            self._dev_branches = tuple(torch.from_numpy(np.ascontiguousarray(a, dt)).to(v.device)
                                       for a, dt in ((f, np.int32), (t, np.int32), (r, np.float64),
                                                     (x, np.float64), (b, np.float64)))
        f, t, r, x, b = self._dev_branches
        nbr = f.shape[0]
        ins = None
        if in_service is not None:
            if in_service.shape != (B, nbr):
                raise ValueError(f"in_service must be [{B}, {nbr}]")
            ins = in_service.to(torch.uint8).contiguous()
        sf = torch.empty((B, nbr), dtype=torch.complex128, device=v.device)
        st = torch.empty((B, nbr), dtype=torch.complex128, device=v.device)
        check(lib.pf_branch_flows(self.n, nbr, _dptr(f), _dptr(t), _dptr(r), _dptr(x), _dptr(b), B,
                                  None if ins is None else _dptr(ins), _dptr(v), _dptr(sf), _dptr(st), _stream()),
              "pf_branch_flows")
        return sf, st

    def solve_outages(self, outages: torch.Tensor, sbus: torch.Tensor, v0: torch.Tensor, tol: float = 1e-8,
                      maxit: int = 10, out=None):
        """Newton-Raphson for branch-outage cases (pf_solve_batch_outages):
        outages int32 [B, k] on the GPU (branch indices, -1 = none); each
        instance's admittances are the base ones minus its outaged branches,
        built on the device.  The plan must come from from_branches."""
        B = sbus.shape[0]
        self._check_bn(sbus, B)
        self._check_bn(v0, B)
        if outages.dtype != torch.int32 or outages.dim() != 2 or outages.shape[0] != B:
            raise ValueError(f"outages must be int32 [{B}, k]")
        if not getattr(self, "_branches_set", False):
            f, t, r, x, b = (np.ascontiguousarray(a, dt) for a, dt in zip(
                self._branches, (np.int32, np.int32, np.float64, np.float64, np.float64)))
            check(lib.pf_plan_set_branches(self._h, f.shape[0], _lib._np_ptr(f), _lib._np_ptr(t), _lib._np_ptr(r),
                                           _lib._np_ptr(x), _lib._np_ptr(b)), "pf_plan_set_branches")
            self._branches_set = True
        dev = sbus.device
        if out is None:
            v = torch.empty((B, self.n), dtype=torch.complex128, device=dev)
            iters = torch.empty(B, dtype=torch.int32, device=dev)
            status = torch.empty(B, dtype=torch.uint8, device=dev)
        else:
            v, iters, status = out
        outages = outages.contiguous()
        check(lib.pf_solve_batch_outages(self._h, B, _dptr(outages), outages.shape[1], _dptr(sbus), _dptr(v0),
                                         float(tol), int(maxit), _dptr(v), _dptr(iters), _dptr(status), _stream()),
              "pf_solve_batch_outages")
        return v, iters, status

    def solve_y(self, ybus: torch.Tensor, sbus: torch.Tensor, v0: torch.Tensor, tol: float = 1e-8,
                maxit: int = 10, out=None):
        """Newton-Raphson with per-instance admittances on this plan's pattern
        (pf_solve_batch_y): ybus complex128 [B, nnz] on the GPU in the
        pattern's CRS order, sbus / v0 complex128 [B, n] on the GPU."""
        B = sbus.shape[0]
        self._check_bn(sbus, B)
        self._check_bn(v0, B)
        nnz = int(self._rowptr[self.n])
        if ybus.dtype != torch.complex128 or ybus.shape != (B, nnz):
            raise ValueError(f"expected complex128 [{B}, {nnz}], got {ybus.dtype} {tuple(ybus.shape)}")
        dev = sbus.device
        if out is None:
            v = torch.empty((B, self.n), dtype=torch.complex128, device=dev)
            iters = torch.empty(B, dtype=torch.int32, device=dev)
            status = torch.empty(B, dtype=torch.uint8, device=dev)
        else:
            v, iters, status = out
        check(lib.pf_solve_batch_y(self._h, B, _dptr(ybus), _dptr(sbus), _dptr(v0), float(tol), int(maxit),
                                   _dptr(v), _dptr(iters), _dptr(status), _stream()), "pf_solve_batch_y")
        return v, iters, status

    def solve_host(self, sbus: torch.Tensor, v0: torch.Tensor, tol: float = 1e-8, maxit: int = 10,
                   out=None, chunk: int = 0):
        """Newton-Raphson for a batch in host memory (complex128 [B, n] CPU
        tensors, page-locked for overlapped copies): the batch is solved in
        chunks whose copies overlap the neighbouring chunks' solves
        (pf_solve_batch_host).  Ordered on the current stream; synchronise it
        before reading the outputs.  Returns host (v, iters, status)."""
        B = sbus.shape[0]
        for t in (sbus, v0):
            if t.device.type != "cpu" or t.dtype != torch.complex128 or t.shape != (B, self.n) \
                    or not t.is_contiguous():
                raise ValueError(f"expected contiguous complex128 [{B}, {self.n}] host tensors")
        if out is None:
            pin = sbus.is_pinned()
            v = torch.empty((B, self.n), dtype=torch.complex128, pin_memory=pin)
            iters = torch.empty(B, dtype=torch.int32, pin_memory=pin)
            status = torch.empty(B, dtype=torch.uint8, pin_memory=pin)
        else:
            v, iters, status = out
        check(lib.pf_solve_batch_host(self._h, B, _hptr(sbus), _hptr(v0), float(tol), int(maxit), _hptr(v),
                                      _hptr(iters), _hptr(status), int(chunk), _stream()), "pf_solve_batch_host")
        return v, iters, status

    def stage_mismatch(self, sbus, v):
        B = v.shape[0]
        self._check_bn(sbus, B)
        self._check_bn(v, B)
        m = self.info["m"]
        F = torch.empty((B, m), dtype=torch.float64, device=v.device)
        norm = torch.empty(B, dtype=torch.float64, device=v.device)
        check(lib.pf_stage_mismatch(self._h, B, _dptr(sbus), _dptr(v), _dptr(F), _dptr(norm), _stream()),
              "pf_stage_mismatch")
        return F, norm

    def stage_factor(self, v, factor=True):
        B = v.shape[0]
        self._check_bn(v, B)
        nnz = C.c_int64(0)
        check(lib.pf_plan_get_pattern(self._h, None, None, None, C.byref(nnz)), "pattern")
        lu = torch.empty((B, nnz.value), dtype=torch.float64, device=v.device)
        check(lib.pf_stage_factor(self._h, B, _dptr(v), int(bool(factor)), _dptr(lu), _stream()),
              "pf_stage_factor")
        return lu

    def stage_linear_solve(self, v, rhs):
        B = v.shape[0]
        self._check_bn(v, B)
        m = self.info["m"]
        if rhs.shape != (B, m) or rhs.dtype != torch.float64:
            raise ValueError("rhs must be float64 [B, m]")
        dx = torch.empty((B, m), dtype=torch.float64, device=v.device)
        check(lib.pf_stage_linear_solve(self._h, B, _dptr(v), _dptr(rhs), _dptr(dx), _stream()),
              "pf_stage_linear_solve")
        return dx

    # ---- launch accounting ----
    def profile_start(self, time_classes=()):
        """Reset launch counters; the named kernel classes get CUDA-event timing."""
        mask = 0
        for c in time_classes:
            mask |= 1 << KERNEL_CLASSES.index(c)
        check(lib.pf_profile_start(self._h, mask), "pf_profile_start")

    def profile_read(self) -> dict:
        """{class: (launches, timed launches, summed ms)} since profile_start."""
        pr = _lib.pf_profile()
        check(lib.pf_profile_read(self._h, C.byref(pr)), "pf_profile_read")
        return {c: (pr.launches[i], pr.timed[i], pr.ms[i]) for i, c in enumerate(KERNEL_CLASSES)}

    def _check_bn(self, t, B):
        if t.dtype != torch.complex128 or t.shape != (B, self.n):
            raise ValueError(f"expected complex128 [{B}, {self.n}], got {t.dtype} {tuple(t.shape)}")


class MultiPlan:
    """Uneven batch: several plans (no dense block) with their own scenario
    counts, solved by one persistent, graph-captured launch (pf_multi_*)."""

    def __init__(self, plans, batches):
        self.plans = list(plans)
        self.batches = [int(b) for b in batches]
        arr = (C.c_void_p * len(self.plans))(*[p._h.value for p in self.plans])
        bat = np.ascontiguousarray(self.batches, np.int32)
        h = C.c_void_p()
        check(lib.pf_multi_create(len(self.plans), arr, _lib._np_ptr(bat), C.byref(h)), "pf_multi_create")
        self._h = h
        self._keep = (arr, bat)
        self.total = int(sum(self.batches))
        self.sizes = [p.n for p in self.plans]

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib.pf_multi_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _outs(self, sbus):
        dev = sbus.device
        return (torch.empty_like(sbus), torch.empty(self.total, dtype=torch.int32, device=dev),
                torch.empty(self.total, dtype=torch.uint8, device=dev))

    def solve(self, sbus, v0, tol=1e-8, maxit=10, out=None):
        """sbus, v0: complex128 1-D tensors, the [B_f, n_f] blocks concatenated."""
        v, it, st = out if out is not None else self._outs(sbus)
        check(lib.pf_multi_solve(self._h, _dptr(sbus), _dptr(v0), float(tol), int(maxit), _dptr(v), _dptr(it),
                                 _dptr(st), _stream()), "pf_multi_solve")
        return v, it, st

    def autotune(self, sbus, v0, tol=1e-8, maxit=10):
        v, it, st = self._outs(sbus)
        ms = C.c_double(0)
        check(lib.pf_multi_autotune(self._h, _dptr(sbus), _dptr(v0), float(tol), int(maxit), _dptr(v), _dptr(it),
                                    _dptr(st), _stream(), C.byref(ms)), "pf_multi_autotune")
        return {**self.config, "ms": ms.value}

    def set_config(self, warps, blocks_per_sm):
        check(lib.pf_multi_set_config(self._h, int(warps), int(blocks_per_sm)), "pf_multi_set_config")

    def set_scenarios(self, per_item, use_smem=True):
        """Scenarios per work item (power of two <= 32) and whether item
        states that fit go to shared memory."""
        check(lib.pf_multi_set_scenarios(self._h, int(per_item), int(bool(use_smem))), "pf_multi_set_scenarios")

    @property
    def config(self):
        w, b, n, i = C.c_int(0), C.c_int(0), C.c_int64(0), C.c_int(0)
        check(lib.pf_multi_get_config(self._h, C.byref(w), C.byref(b), C.byref(n), C.byref(i)), "config")
        s, u, sb, si = C.c_int(0), C.c_int(0), C.c_int64(0), C.c_int(0)
        check(lib.pf_multi_get_scenarios(self._h, C.byref(s), C.byref(u), C.byref(sb), C.byref(si)), "scenarios")
        return {"warps": w.value, "blocks_per_sm": b.value, "instances": n.value, "items": i.value,
                "scenarios_per_item": s.value, "shared_memory": bool(u.value), "smem_bytes": sb.value,
                "smem_items": si.value}
