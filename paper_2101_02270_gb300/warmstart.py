"""Learned warm start: an MLP trained on the solver's own solutions proposes
the start voltages, Newton-Raphson then runs from them to the same tolerance,
and instances that fail from the guess are re-solved from flat start.
Every numeric step runs in the library (pf_mlp_*, pf_warmstart_*,
pf_solve_batch); this module only orchestrates calls and owns the tensors."""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import _lib
from ._lib import check, lib
from .solver import _dptr, _stream


class MLP:
    """pf_mlp: 3-layer GELU network with BF16 tensor-core GEMMs."""

    def __init__(self, nin, nh1, nh2, nout, bmax, seed=0):
        self.shape = (nin, nh1, nh2, nout)
        self.bmax = bmax
        h = C.c_void_p()
        check(lib.pf_mlp_create(nin, nh1, nh2, nout, bmax, C.c_uint64(seed), C.byref(h)), "pf_mlp_create")
        self._h = h

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib.pf_mlp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _host_arrays(self):
        nin, nh1, nh2, nout = self.shape
        shapes = [(nh1, nin), (nh1,), (nh2, nh1), (nh2,), (nout, nh2), (nout,)]
        return [np.zeros(s, np.float32) for s in shapes]

    def params(self):
        arrs = self._host_arrays()
        ptrs = (C.c_void_p * 6)(*[a.ctypes.data for a in arrs])
        check(lib.pf_mlp_params(self._h, 0, ptrs), "pf_mlp_params")
        return arrs

    def set_params(self, arrs):
        arrs = [np.ascontiguousarray(a, np.float32) for a in arrs]
        ptrs = (C.c_void_p * 6)(*[a.ctypes.data for a in arrs])
        check(lib.pf_mlp_params(self._h, 1, ptrs), "pf_mlp_params")

    def grads(self):
        arrs = self._host_arrays()
        ptrs = (C.c_void_p * 6)(*[a.ctypes.data for a in arrs])
        check(lib.pf_mlp_grads(self._h, ptrs), "pf_mlp_grads")
        return arrs

    def set_norm(self, mux, sdx, muy, sdy):
        a = [np.ascontiguousarray(v, np.float32) for v in (mux, sdx, muy, sdy)]
        check(lib.pf_mlp_set_norm(self._h, *[_lib._np_ptr(v) for v in a]), "pf_mlp_set_norm")

    def fit_norm(self, X, T):
        check(lib.pf_mlp_fit_norm(self._h, X.shape[0], _dptr(X), _dptr(T), _stream()), "pf_mlp_fit_norm")

    def predict(self, X):
        Y = torch.empty((X.shape[0], self.shape[3]), dtype=torch.float32, device=X.device)
        check(lib.pf_mlp_predict(self._h, X.shape[0], _dptr(X), _dptr(Y), _stream()), "pf_mlp_predict")
        return Y

    def train_step(self, X, T, lr=1e-3, wd=0.0, update=True, loss=None):
        if loss is None:
            loss = torch.zeros(1, dtype=torch.float32, device=X.device)
        check(lib.pf_mlp_train_step(self._h, X.shape[0], _dptr(X), _dptr(T), float(lr), float(wd), int(update),
                                    _dptr(loss), _stream()), "pf_mlp_train_step")
        return loss

    def error(self):
        return lib.pf_mlp_error(self._h)

    # ---- checkpoint / resume (weights and standardisation; the optimiser
    # state restarts) ----
    def save(self, path, norm=None):
        arrs = self.params()
        extra = {} if norm is None else {f"norm{i}": np.asarray(v, np.float32) for i, v in enumerate(norm)}
        np.savez(path, shape=np.array(self.shape), **{f"p{i}": a for i, a in enumerate(arrs)}, **extra)

    def load(self, path):
        z = np.load(path)
        if tuple(int(v) for v in z["shape"]) != tuple(self.shape):
            raise ValueError(f"checkpoint shape {tuple(z['shape'])} != network {self.shape}")
        self.set_params([z[f"p{i}"] for i in range(6)])
        if "norm0" in z:
            self.set_norm(*[z[f"norm{i}"] for i in range(4)])


def gemm_bf16(A, B, variant=1):
    """C = A B^T on the tensor cores (A [M,K], B [N,K] bfloat16 CUDA tensors).
    variant 0: one-stage kernel; 1: TMA-pipelined kernel."""
    M, K = A.shape
    N = B.shape[0]
    Cm = torch.empty((M, N), dtype=torch.float32, device=A.device)
    err = torch.zeros(1, dtype=torch.int32, device=A.device)
    check(lib.pf_gemm_bf16(_dptr(A), _dptr(B), _dptr(Cm), M, N, K, int(variant), _dptr(err), _stream()),
          "pf_gemm_bf16")
    return Cm, err


class WarmStart:
    """Solver + network for one grid: features, targets, guesses, solves."""

    def __init__(self, plan, bus_type, mlp: MLP):
        self.plan = plan
        self.n = plan.n
        bt = np.asarray(bus_type, np.int8)
        ns = np.flatnonzero(bt != 3)
        nsidx = -np.ones(self.n, np.int32)
        nsidx[ns] = np.arange(ns.size, dtype=np.int32)
        self.nns = int(ns.size)
        self.nsidx = torch.from_numpy(nsidx).cuda()
        self.bt = torch.from_numpy(bt).cuda()
        self.mlp = mlp
        assert mlp.shape[0] == 2 * self.n and mlp.shape[3] == 2 * self.nns

    def features(self, sbus):
        X = torch.empty((sbus.shape[0], 2 * self.n), dtype=torch.float32, device=sbus.device)
        check(lib.pf_warmstart_features(self.n, sbus.shape[0], _dptr(sbus), _dptr(X), _stream()), "features")
        return X

    def targets(self, V):
        T = torch.empty((V.shape[0], 2 * self.nns), dtype=torch.float32, device=V.device)
        check(lib.pf_warmstart_targets(self.n, V.shape[0], _dptr(self.nsidx), self.nns, _dptr(V), _dptr(T),
                                       _stream()), "targets")
        return T

    def guess(self, sbus, v_flat):
        Y = torch.empty((sbus.shape[0], 2 * self.nns), dtype=torch.float32, device=sbus.device)
        X = self.features(sbus)
        for b0 in range(0, sbus.shape[0], self.mlp.bmax):
            b1 = min(sbus.shape[0], b0 + self.mlp.bmax)
            Y[b0:b1] = self.mlp.predict(X[b0:b1])
        V0 = torch.empty_like(v_flat)
        check(lib.pf_warmstart_v0(self.n, sbus.shape[0], _dptr(self.nsidx), _dptr(self.bt), self.nns, _dptr(Y),
                                  _dptr(v_flat), _dptr(V0), _stream()), "v0")
        return V0

    def screen(self, v, status, vmin=None):
        """redo [B] (bool, device): instances whose warm-started result is not
        taken: status != 0, a non-finite voltage, or a magnitude below vmin
        p.u. (a low-voltage root of the power-flow equations)."""
        vmin = self.vmin if vmin is None else vmin
        redo = torch.empty(v.shape[0], dtype=torch.uint8, device=v.device)
        check(lib.pf_warmstart_screen(self.n, v.shape[0], _dptr(v), _dptr(status), float(vmin), _dptr(redo),
                                      _stream()), "pf_warmstart_screen")
        return redo.bool()

    # Magnitude floor of the screen.  Operating points of the workloads here
    # stay above 0.8 p.u. (their load scale is chosen so); the low-voltage
    # roots reached from bad guesses sit at a few hundredths of a p.u.
    vmin = 0.5

    def solve(self, sbus, v_flat, tol=1e-8, maxit=10):
        """NR from the network's guess; instances whose result fails the
        screen (no convergence, or a low-voltage root) are re-solved from flat
        start, whose result is taken as it is.  Returns (v, iters, status,
        fallback) with iters counting the updates of the run that produced v."""
        V0 = self.guess(sbus, v_flat)
        v, it, st = self.plan.solve(sbus, V0, tol, maxit)
        fb = self.screen(v, st)
        bad = torch.nonzero(fb).flatten()
        if bad.numel():
            v2, it2, st2 = self.plan.solve(sbus[bad].contiguous(), v_flat[bad].contiguous(), tol, maxit)
            v[bad], it[bad], st[bad] = v2, it2, st2
        return v, it, st, fb
