#!/usr/bin/env python
"""Benchmark: Newton-Raphson AC power flows per second on one GB300.

A step is one pf_solve_batch over the whole batch of the workload (every NR
iteration: mismatch + Jacobian refill, sparse + dense LU refactor, FS/BS,
update, until max|F| < 1e-8 p.u. or maxit) with inputs resident in HBM.
Default workload: the 9,000-bus meshed synthetic grid, 10,000 load scenarios,
the mixed-precision form (LU refactor and FS/BS in FP32; mismatch, update and
convergence test in FP64), flat start, tol 1e-8, maxit 10.  The same line
carries the 2,000-bus workload in plain FP64 and with FP32 LU, the learned
warm start, and plain FP64 on a subset of the 9,000-bus batch, each with its
own oracle comparison (``--config`` / ``--lu`` select a single workload).
Prints one JSON line.

Multi-GPU (torchrun): every rank solves its own batch (weak scaling, no data
exchange); barrier + max-over-ranks timing.
``--impl reference`` times the CPU FP64 oracle on the host cores instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import gridgen  # noqa: E402

METRIC = "NR power flows/sec at 1e-8 p.u. mismatch on 1 GB300; % of HBM roofline"
UNIT = "flows/s"
TOL = 1e-8
MAXIT = 10
# Peaks: HBM copy bandwidth from the pool's measurement file; FP64 / FP32 FMA
# throughput measured live by pf_fma_peak (independent FMA chains on every SM).
HBM_FALLBACK_GBS = 6800.0
# DRAM bytes (read + write) of one k_dense_update launch per instance and per
# trailing-matrix entry r^2, from the ncu capture summarised in
# profiles/dense_update_fp64_mesh2000.md (batch 640, panel 8, r = 200).
DENSE_UPDATE_DRAM_B_PER_R2 = 14.3


def measured_hbm():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except Exception:
        return HBM_FALLBACK_GBS, "fallback"


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="mesh9000_b10k",
                    choices=list(gridgen.CONFIGS) + ["feeders256x100", "warmstart2000", "n1_2000"])
    ap.add_argument("--train-samples", type=int, default=200000)
    ap.add_argument("--train-steps", type=int, default=3000)
    ap.add_argument("--batch", type=int, default=0, help="override the batch size (0 = the workload's)")
    ap.add_argument("--lu", default=None, choices=["fp64", "fp32"],
                    help="LU precision (default: fp32 for the 9,000-bus workload, fp64 otherwise)")
    ap.add_argument("--maxit", type=int, default=MAXIT)
    ap.add_argument("--dense-frac", type=float, default=0.0, help="0 = the library's default for the precision")
    ap.add_argument("--panel", type=int, default=0, help="0 = the library's default for the precision")
    ap.add_argument("--dense-layout", default="auto", choices=["auto", "interleaved", "instance_major"],
                    help="storage of the dense block (auto: instance-major for large FP32 blocks)")
    ap.add_argument("--chunk", type=int, default=0,
                    help="instances per chunk of the end-to-end host solve (0 = about a quarter of the batch)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-oracle", action="store_true",
                    help="skip the oracle comparison of the GPU results (profiling runs)")
    ap.add_argument("--no-extras", action="store_true",
                    help="default workload only: skip the 2,000-bus, warm-start and FP64-subset keys")
    ap.add_argument("--roofline-steps", type=int, default=0,
                    help="steps of the per-launch-timed roofline pass (0: all K steps, at most 4 on the "
                         "9,000-bus workload)")
    ap.add_argument("--time-all", action="store_true",
                    help="diagnostic: CUDA-event timing of every kernel class (adds two events per launch)")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    return ap.parse_args()


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out = ""
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# CPU oracle (baseline and reference arm)
# ---------------------------------------------------------------------------
# one oracle solve on grids above this size takes longer than the whole CPU
# budget of a bench line (about 100 s on one Grace core for 9,000 buses): the
# sample is then one round of one instance per core, without a calibration run
ORACLE_ROUND_ONLY_BUSES = 4000


def _oracle_cases(task):
    """Oracle Newton solves of instances with their own branch sets (one
    process of the per-instance-admittance sample): (V, iters, status)."""
    from oracle import nrpf
    n, f, t, r, x, b, bus_type, ins, S, V0 = task
    out = []
    for keep, s, v0 in zip(ins, S, V0):
        Y = nrpf.make_ybus(n, f[keep], t[keep], r[keep], x[keep], b[keep])
        out.append(nrpf.newton(Y, s, v0, bus_type, TOL, MAXIT))
    return (np.array([o[0] for o in out]), np.array([o[1] for o in out]), np.array([o[2] for o in out]))


def compare_with_oracle(Vg, itg, stg, Vo, ito, sto):
    """The GPU's results against the FP64 oracle's on the same instances:
    statuses, max |V| and angle differences, Newton-iteration difference
    (GPU minus oracle)."""
    ok = (sto == 0) & (stg == 0)
    Vs = Vg[ok]
    dvm = np.abs(np.abs(Vs) - np.abs(Vo[ok]))
    dth = np.abs(np.angle(Vs * np.conj(Vo[ok])))
    dit = itg[ok].astype(int) - ito[ok].astype(int)
    return {"instances": int(len(sto)), "same_status": bool(np.array_equal(stg, sto)),
            "max_abs_dv": float(np.max(np.abs(Vs - Vo[ok]), initial=0.0)),
            "max_abs_dvm": float(np.max(dvm, initial=0.0)), "max_abs_dtheta": float(np.max(dth, initial=0.0)),
            "max_iter_diff": int(np.max(np.abs(dit), initial=0)),
            "mean_iter_diff": float(np.mean(dit)) if dit.size else 0.0,
            "oracle_iters_mean": float(np.mean(ito)), "tolerance": "|dV| <= 1e-6 p.u., |dtheta| <= 1e-6 rad"}


def oracle_sample(g, S, V0, seconds, cores, ins=None, gpu=None):
    """Time the CPU oracle on a bounded sample of the workload: a first
    calibration run sizes the sample to about `seconds` of work on `cores`
    processes (grids above ORACLE_ROUND_ONLY_BUSES: one round of one instance
    per core).  ins [B, nbr] (optional): per-instance branch sets, each
    instance then gets its own admittance matrix.  gpu = (V, iters, status)
    of the GPU on the whole batch: the sample's oracle results are compared
    with them ("vs_oracle")."""
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")
    from oracle import nrpf
    B = S.shape[0]
    if ins is None:
        Y = nrpf.make_ybus(g.n, g.f, g.t, g.r, g.x, g.b)
        run = lambda k, w: nrpf.newton_batch(Y, S[:k], V0[:k], g.bus_type, TOL, MAXIT, workers=w)
    else:
        import multiprocessing as mp

        def run(k, w):
            if w <= 1 or k < 2:
                return _oracle_cases((g.n, g.f, g.t, g.r, g.x, g.b, g.bus_type, ins[:k], S[:k], V0[:k]))
            parts = np.array_split(np.arange(k), min(w, k))
            tasks = [(g.n, g.f, g.t, g.r, g.x, g.b, g.bus_type, ins[p], S[p], V0[p]) for p in parts]
            with mp.get_context("spawn").Pool(len(tasks)) as pool:
                res = pool.map(_oracle_cases, tasks)
            return tuple(np.concatenate([r[i] for r in res]) for i in range(3))
    if g.n > ORACLE_ROUND_ONLY_BUSES:
        size = min(cores, B)
    else:
        t0 = time.perf_counter()
        run(1, 1)
        t1 = max(time.perf_counter() - t0, 1e-4)
        size = min(B, int(max(cores, min(B, seconds * cores / t1))))
    t0 = time.perf_counter()
    Vo, ito, sto = run(size, cores)
    dt = time.perf_counter() - t0
    conv = int(np.sum(sto == 0))
    what = "instances (own admittance matrix each)" if ins is not None else "scenarios"
    out = {"value": conv / dt, "unit": UNIT, "cores": min(cores, size), "kind": "oracle",
           "sample": f"first {size} of {B} {what}, scipy SuperLU per Newton step, "
                     f"{min(cores, size)} spawn processes, {dt:.1f} s"}
    if gpu is not None:
        Vg, itg, stg = gpu
        out["vs_oracle"] = compare_with_oracle(Vg[:size], itg[:size], stg[:size], Vo, ito, sto)
    return out


def whole_solve_roofline(parts, ms_per_step, kernel):
    """HBM roofline of a solve done by one persistent kernel: algorithmic
    bytes per instance-iteration (LU values written and read once, voltages,
    injections, right-hand side and solution: 2 w nnz_LU + 8 (8 n + 4 m)),
    summed over (plan info, LU bytes per value w, Newton updates of its
    instances), over the step time, against the measured copy bandwidth."""
    hbm, kind = measured_hbm()
    total = sum((2 * w * info["nnz_lu"] + 8 * (8 * info["n"] + 4 * info["m"])) * int(upd)
                for info, w, upd in parts)
    achieved = total / (ms_per_step / 1e3) / 1e9
    return {"bound": "hbm", "kernel": kernel, "achieved": achieved, "peak": hbm, "unit": "GB/s",
            "frac": achieved / hbm, "traffic": None, "peak_kind": f"{kind} HBM copy bandwidth",
            "bytes_per_step": total}


def cpu_batched_sample(pf, g, S, V0, seconds):
    """The library's batched host solver (pf_solve_batch_cpu: instances in
    SIMD lanes, all hardware threads) on a bounded sample of the workload, a
    stronger CPU point than the oracle.  Its own host-only plan with the dense
    cut at 0.3 of the remaining weight."""
    cores = os.cpu_count() or 1
    plan = pf.Plan.from_branches(g.n, g.f, g.t, g.r, g.x, g.b, g.bus_type, host_only=True, dense_frac=0.3)
    k = min(S.shape[0], 2 * 8 * cores)
    t0 = time.perf_counter()
    plan.solve_cpu(S[:k], V0[:k], TOL, MAXIT)
    t1 = max(time.perf_counter() - t0, 1e-3)
    size = int(min(S.shape[0], max(k, k * seconds / t1)))
    t0 = time.perf_counter()
    _, it, st = plan.solve_cpu(S[:size], V0[:size], TOL, MAXIT)
    dt = time.perf_counter() - t0
    plan.close()
    return {"value": int(np.sum(st == 0)) / dt, "unit": UNIT, "cores": cores, "kind": "library host solver",
            "sample": f"first {size} of {S.shape[0]} scenarios, pf_solve_batch_cpu (8 instances per SIMD "
                      f"mini-batch, {cores} threads), {dt:.1f} s"}


def run_reference(args):
    """The CPU FP64 oracle on the host cores, on the same workload and metric
    (each step a bounded sample of the workload)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    name = args.config
    if name == "feeders256x100":
        fs = gridgen.make_feeders()
        scen = gridgen.grids.feeder_scenarios(fs)
        # a sample mixing feeders: every 16th feeder, its scenarios
        cases = [(fs[i], scen[i].sbus(fs[i]), scen[i].v0_flat(fs[i])) for i in range(0, len(fs), 16)]
        batch = sum(sc.batch for sc in scen)
    elif name == "n1_2000":
        g = gridgen.make_grid("mesh2000_b10k")
        _, _, ins, S = gridgen.n1_batch(g)
        cases = [(g, S, np.broadcast_to(g.v_set.astype(np.complex128), S.shape).copy(), ins)]
        batch = int(S.shape[0])
    else:
        gname = "mesh2000_b10k" if name == "warmstart2000" else name
        g = gridgen.make_grid(gname)
        sc = gridgen.config_scenarios(gname, g, batch=args.batch or None)
        cases = [(g, sc.sbus(g), sc.v0_flat(g))]
        batch = int(sc.batch)
    cores = os.cpu_count() or 1
    per_step = max(1.0, 60.0 / max(args.steps + args.warmup, 1))

    def one(seconds):
        vals, last = [], None
        for case in cases:
            last = oracle_sample(*case[:3], seconds / len(cases), cores, *case[3:])
            vals.append(last["value"])
        return statistics.mean(vals), last

    if any(case[0].n > ORACLE_ROUND_ONLY_BUSES for case in cases):
        # a single oracle solve of this grid takes about 100 s on one core:
        # one round of one instance per core stands for the K steps (and the
        # warm-up is the spawn of the processes inside it)
        t0 = time.perf_counter()
        v, last = one(per_step)
        dt = time.perf_counter() - t0
        line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic", "config": {"workload": name, "batch": batch, "tol": TOL, "maxit": MAXIT,
                                                "reference_rounds": 1},
                "cpu_baseline": dict(last, value=v, sample=last["sample"] + "; one round stands for the K steps"),
                "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return
    for _ in range(args.warmup):
        one(min(per_step, 2.0))
    vals = []
    last = None
    t0 = time.perf_counter()
    for _ in range(args.steps):
        v, last = one(per_step)
        vals.append(v)
    dt = time.perf_counter() - t0
    value = statistics.mean(vals)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / max(args.steps, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": name, "batch": batch, "tol": TOL, "maxit": MAXIT},
            "cpu_baseline": dict(last, value=value),
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# multi-rank bookkeeping (weak scaling: every rank solves its own scenarios)
# ---------------------------------------------------------------------------
def rank_scenarios(name, g, rank, batch=None):
    """Scenarios of one rank: the workload's distribution drawn with seed 1 + rank."""
    return gridgen.config_scenarios(name, g, batch=batch, seed=1 + rank)


def combine_ranks(ms, converged, device):
    """Max elapsed time over ranks and the total converged instances of the
    job (value = total / max time); a no-op without a process group."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    c = torch.tensor([float(converged)], dtype=torch.float64, device=device)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(c)
    return float(t.item()), float(c.item())


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
# ncu DRAM bytes over algorithmic bytes of the depth-64 FP32 trailing update
# of the interleaved layout; None: the kernel changed (packed two-wide FMAs)
# after the capture in profiles/dense_update_fp32_mesh2000.md (371.7 MB of
# 419.4 MB), which is not repeated for it.
DENSE_UPDATE_FP32_DRAM_PER_ALG = None

# ncu DRAM bytes (read + write) of one k_im_gemm launch over its algorithmic
# bytes (im_update_bytes), from the capture summarised in
# profiles/im_gemm_mesh9000_b64.md (batch 64, outer panel 8: 739.5 MB
# against 746.6 MB).
IM_GEMM_DRAM_PER_ALG = 0.99

KERNEL_TIMING = ("CUDA events around every dense_update launch on its stream, during a second pass of the "
                 "K timed steps")


def dense_update_launches(ndp, kb):
    """The k_dense_update launches of one dense refactor, each a list of the
    rectangles A[rows, cols] -= L U of depth d it updates, as (rows, cols, d).
    Panels of 4-16: one trailing update per panel.  Two-level panels (32, 64):
    per 16-wide inner step, the outer panel's columns below the step plus, for
    the outer panel's rows below the step, the columns right of the outer panel
    (one L-shaped launch); then one trailing update of depth kb per outer
    panel."""
    out = []
    for k in range(0, ndp, kb):
        if kb <= 16:
            if ndp - k - kb > 0:
                out.append([(ndp - k - kb, ndp - k - kb, kb)])
            continue
        for ki in range(k, k + kb, 16):
            r0, kend = ki + 16, k + kb
            rects = [(ndp - r0, kend - r0, 16), (kend - r0, ndp - kend, 16)]
            rects = [r for r in rects if r[0] > 0 and r[1] > 0]
            if rects:
                out.append(rects)
        if ndp - k - kb > 0:
            out.append([(ndp - k - kb, ndp - k - kb, kb)])
    return out


def dense_update_flop(ndp, kb):
    """Algorithmic flops of the updates of one dense refactor: 2 * rows * cols
    * depth per rectangle."""
    return sum(2 * r * c * d for L in dense_update_launches(ndp, kb) for r, c, d in L)


def dense_update_bytes(ndp, kb, w):
    """Algorithmic bytes of the same updates: each rectangle read and written
    once, its two operand panels read once (w bytes a value)."""
    return sum(w * (2 * r * c + d * (r + c)) for L in dense_update_launches(ndp, kb) for r, c, d in L)


def run_feeders(args):
    """256 radial feeders of 20-400 buses, 100 scenarios each, every feeder
    with its own pattern and plan, solved by one persistent graph-captured
    launch (pf_multi_solve) whose shape the library's autotuner picks."""
    import torch

    import paper_2101_02270_gb300 as pf

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    fs = gridgen.make_feeders()
    scen = gridgen.grids.feeder_scenarios(fs, seed=1 + rank)
    S = np.concatenate([sc.sbus(g).ravel() for g, sc in zip(fs, scen)])
    V0 = np.concatenate([sc.v0_flat(g).ravel() for g, sc in zip(fs, scen)])
    lu = "fp32" if args.lu == "fp64" and not args.lu_explicit else args.lu
    t0 = time.perf_counter()
    plans = [pf.Plan.from_branches(g.n, g.f, g.t, g.r, g.x, g.b, g.bus_type, lu_precision=lu, dense_frac=1.0)
             for g in fs]
    mp = pf.MultiPlan(plans, [sc.batch for sc in scen])
    plan_ms = 1e3 * (time.perf_counter() - t0)
    Sd = torch.from_numpy(S).to(dev)
    Vd = torch.from_numpy(V0).to(dev)
    maxit = args.maxit if args.maxit != MAXIT else 20
    tuned = mp.autotune(Sd, Vd, TOL, maxit)
    out = mp._outs(Sd)
    for _ in range(max(args.warmup, 0)):
        mp.solve(Sd, Vd, TOL, maxit, out=out)
    stream = torch.cuda.current_stream()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.steps):
        mp.solve(Sd, Vd, TOL, maxit, out=out)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    clk = clocks.stop()
    it = out[1].cpu().numpy()
    st = out[2].cpu().numpy()
    conv = int(np.sum(st == 0))
    value = conv * args.steps / (ms / 1e3)
    # end to end from pinned host buffers
    S_h, V_h = torch.from_numpy(S).pin_memory(), torch.from_numpy(V0).pin_memory()
    Vo_h = torch.empty_like(S_h).pin_memory()
    it_h = torch.empty(mp.total, dtype=torch.int32).pin_memory()
    st_h = torch.empty(mp.total, dtype=torch.uint8).pin_memory()
    S2, V2 = torch.empty_like(Sd), torch.empty_like(Vd)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.steps):
        S2.copy_(S_h, non_blocking=True)
        V2.copy_(V_h, non_blocking=True)
        v, i2, s2 = mp.solve(S2, V2, TOL, maxit, out=out)
        Vo_h.copy_(v, non_blocking=True)
        it_h.copy_(i2, non_blocking=True)
        st_h.copy_(s2, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e = int(np.sum(st_h.numpy() == 0)) * args.steps / (e0.elapsed_time(e1) / 1e3)
    nbus = np.array([g.n for g in fs])
    w = 4 if lu == "fp32" else 8
    parts, off = [], 0
    for p_, sc in zip(plans, scen):
        parts.append((p_.info, w, int(it[off:off + sc.batch].sum())))
        off += sc.batch
    roof = whole_solve_roofline(parts, ms / args.steps, "k_multi (the whole persistent solve)")
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64+f32lu" if lu == "fp32" else "f64", "data": "synthetic",
        "config": {"workload": "feeders256x100", "feeders": len(fs), "scenarios_per_feeder": 100,
                   "buses_min": int(nbus.min()), "buses_max": int(nbus.max()), "buses_total": int(nbus.sum()),
                   "lu_precision": lu, "tol": TOL, "maxit": maxit, "load_scale": fs[0].load_scale,
                   "launch": "one persistent kernel per solve, CUDA graph", "autotuned": tuned,
                   "plan_ms": round(plan_ms, 1)},
        "iterations": {"mean": float(it.mean()), "max": int(it.max()), "hist": np.bincount(it).tolist()},
        "converged": conv, "failed": int(np.sum(st == 2)),
        "clocks": clk,
        "e2e": {"value": e2e, "unit": UNIT, "h2d_bytes_per_step": int(2 * S.nbytes),
                "d2h_bytes_per_step": int(S.nbytes + 5 * mp.total)},
        "gpu_launches": 1,
        "roofline": roof,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # the oracle on every 64th feeder's scenarios, the seconds shared out
        picks = list(range(0, len(fs), 64))
        res = [oracle_sample(fs[i], scen[i].sbus(fs[i]), scen[i].v0_flat(fs[i]), args.cpu_seconds / len(picks),
                             os.cpu_count() or 1) for i in picks]
        line["cpu_baseline"] = dict(res[-1], value=float(np.mean([r["value"] for r in res])),
                                    sample=f"feeders {picks}, each: " + res[-1]["sample"])
    if rank == 0:
        print(json.dumps(line), flush=True)
    mp.close()


def run_warmstart(args):
    print(json.dumps(warmstart_measure(args, args.steps, args.warmup)), flush=True)


def warmstart_measure(args, steps, warmup):
    """Learned warm start on the 2,000-bus grid: 200,000 solver-made solutions
    (scenario seeds 2, 3, ...) train the 4000-1024-1024-3998 network; the
    10,000 held-out scenarios (seed 1, the 2,000-bus workload) are then solved
    from its guesses and from flat start, NR to 1e-8 p.u. with fallback (a
    result that did not converge or sits on a low-voltage root is re-solved
    from flat start).  Returns the JSON line as a dict."""
    import torch

    import paper_2101_02270_gb300 as pf
    from paper_2101_02270_gb300 import warmstart as wsm

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
    torch.cuda.set_device(dev)
    g = gridgen.make_grid("mesh2000_b10k")
    plan64 = pf.Plan.from_branches(g.n, g.f, g.t, g.r, g.x, g.b, g.bus_type, max_batch=10000)
    plan32 = pf.Plan.from_branches(g.n, g.f, g.t, g.r, g.x, g.b, g.bus_type, lu_precision="fp32", max_batch=10000)
    nns = int(np.sum(g.bus_type != 3))
    net = wsm.MLP(2 * g.n, 1024, 1024, 2 * nns, bmax=1024, seed=0)
    ws64 = wsm.WarmStart(plan64, g.bus_type, net)
    ws32 = wsm.WarmStart(plan32, g.bus_type, net)
    # ---- training data from the solver itself ----
    t0 = time.perf_counter()
    chunk = 10000
    nchunks = max(1, args.train_samples // chunk)
    Xs, Ts = [], []
    for c in range(nchunks):
        sc = gridgen.config_scenarios("mesh2000_b10k", g, batch=chunk, seed=2 + c)
        S = torch.from_numpy(sc.sbus(g)).to(dev)
        V, it, st = plan32.solve(S, torch.from_numpy(sc.v0_flat(g)).to(dev), TOL, 20)
        ok = st == 0
        Xs.append(ws32.features(S)[ok])
        Ts.append(ws32.targets(V)[ok])
    X = torch.cat(Xs)
    T = torch.cat(Ts)
    del Xs, Ts
    torch.cuda.synchronize()
    gen_s = time.perf_counter() - t0
    # ---- training ----
    net.fit_norm(X, T)
    gen = torch.Generator(device=dev).manual_seed(0)
    loss = None
    t0 = time.perf_counter()
    train_steps = args.train_steps
    for step in range(train_steps):
        lr = 1e-3 * (0.5 * (1 + np.cos(np.pi * step / train_steps))) + 2e-5
        idx = torch.randint(0, X.shape[0], (1024,), device=dev, generator=gen)
        loss = net.train_step(X[idx].contiguous(), T[idx].contiguous(), lr=lr, wd=1e-4)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    final_loss = float(loss.item())
    del X, T
    # ---- held-out evaluation ----
    ho = gridgen.config_scenarios("mesh2000_b10k", g, seed=1)
    S_np, V0_np = ho.sbus(g), ho.v0_flat(g)
    Sh = torch.from_numpy(S_np).to(dev)
    Vh = torch.from_numpy(V0_np).to(dev)
    stream = torch.cuda.current_stream()

    def timed(fn):
        for _ in range(max(warmup, 1)):
            fn()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(steps):
            r = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps, r

    clocks = ClockSampler(dev.index or 0)
    clocks.start()
    time.sleep(0.3)
    ms_flat64, (vf, itf, stf) = timed(lambda: plan64.solve(Sh, Vh, TOL, MAXIT))
    plan64.profile_start([])
    ms_warm64, (vw, itw, stw, fb) = timed(lambda: ws64.solve(Sh, Vh, TOL, MAXIT))
    prof = plan64.profile_read()
    # library launches of the timed warm solves: the plan's (solves, including
    # any flat-start fallback) plus the network's per guess: features, v0 and,
    # per chunk of bmax instances, input scaling + three GEMMs + output scaling
    # (the counters also saw the warm-up calls: scale to the timed ones)
    calls = max(warmup, 1) + steps
    per_call = sum(v[0] for v in prof.values()) / calls + 3 + 5 * -(-S_np.shape[0] // net.bmax)
    launches = int(round(per_call * steps))
    ms_flat32, (vf32, itf32, stf32) = timed(lambda: plan32.solve(Sh, Vh, TOL, 20))
    ms_warm32, (vw32, itw32, stw32, fb32) = timed(lambda: ws32.solve(Sh, Vh, TOL, 20))
    clk = clocks.stop()
    B = S_np.shape[0]
    conv = int((stw == 0).sum().item())
    value = conv / (ms_warm64 / 1e3)
    # end to end: page-locked host scenarios in, warm-started solve, results out
    S_pin = torch.from_numpy(S_np).pin_memory()
    V_pin = torch.from_numpy(V0_np).pin_memory()
    Sd, Vd = torch.empty_like(Sh), torch.empty_like(Vh)
    v_pin = torch.empty((B, g.n), dtype=torch.complex128).pin_memory()
    it_pin = torch.empty(B, dtype=torch.int32).pin_memory()
    st_pin = torch.empty(B, dtype=torch.uint8).pin_memory()

    def e2e():
        Sd.copy_(S_pin, non_blocking=True)
        Vd.copy_(V_pin, non_blocking=True)
        v, it, st, _ = ws64.solve(Sd, Vd, TOL, MAXIT)
        v_pin.copy_(v, non_blocking=True)
        it_pin.copy_(it, non_blocking=True)
        st_pin.copy_(st, non_blocking=True)
        return None

    ms_e2e, _ = timed(e2e)
    e2e_value = int((st_pin == 0).sum()) / (ms_e2e / 1e3)
    dv = float((vw - vf).abs().max().item())
    # the warm-started results against the FP64 oracle's flat-start solutions
    # on sampled held-out scenarios (iteration difference: saved iterations
    # show as negative numbers)
    idx = sample_indices(B)
    vo64 = vs_oracle(g, S_np, V0_np, vw.cpu().numpy(), itw.cpu().numpy(), stw.cpu().numpy(), idx, MAXIT)
    vo32 = vs_oracle(g, S_np, V0_np, vw32.cpu().numpy(), itw32.cpu().numpy(), stw32.cpu().numpy(), idx, MAXIT)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": steps, "warmup": warmup,
        "ms_per_step": ms_warm64, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64 (NR) + bf16 (MLP)", "data": "synthetic",
        "config": {"workload": "warmstart2000", "buses": g.n, "held_out": B, "train_samples": nchunks * chunk,
                   "train_steps": train_steps, "mlp": [2 * g.n, 1024, 1024, 2 * nns], "tol": TOL},
        "warm_fp64": {"flows_s": value, "ms": ms_warm64, "iters_mean": float(itw.float().mean()),
                      "fallbacks": int(fb.sum()), "converged": conv},
        "flat_fp64": {"flows_s": int((stf == 0).sum()) / (ms_flat64 / 1e3), "ms": ms_flat64,
                      "iters_mean": float(itf.float().mean())},
        "warm_fp32lu": {"flows_s": int((stw32 == 0).sum()) / (ms_warm32 / 1e3), "ms": ms_warm32,
                        "iters_mean": float(itw32.float().mean()), "fallbacks": int(fb32.sum()),
                        "vs_oracle": vo32},
        "flat_fp32lu": {"flows_s": int((stf32 == 0).sum()) / (ms_flat32 / 1e3), "ms": ms_flat32,
                        "iters_mean": float(itf32.float().mean())},
        "max_dv_warm_vs_flat": dv, "vs_oracle": vo64,
        "training": {"generate_s": round(gen_s, 2), "train_s": round(train_s, 2), "final_loss": final_loss},
        "clocks": clk, "gpu_launches": launches,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(2 * S_pin.nbytes),
                "d2h_bytes_per_step": int(v_pin.nbytes + it_pin.nbytes + st_pin.nbytes)},
        "roofline": whole_solve_roofline([(plan64.info, 8, int(itw.sum()))], ms_warm64,
                                         "the warm-started FP64 solve (its dense update is FP64-bound)"),
    }
    if not args.no_cpu_baseline and args.config == "warmstart2000":
        line["cpu_baseline"] = oracle_sample(g, S_np, V0_np, args.cpu_seconds, os.cpu_count() or 1)
        line["cpu_baseline"]["sample"] += " (flat start: the oracle has no network)"
    plan64.close()
    plan32.close()
    net.close()
    torch.cuda.empty_cache()
    return line


def run_small(args):
    """30-bus meshed grid, 64 scenarios: a latency case.  Solved by the fused
    persistent kernel (pf_multi_*, one graph launch, pure sparse plan) and,
    for comparison, by the multi-kernel pf_solve_batch path."""
    import torch

    import paper_2101_02270_gb300 as pf

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
    torch.cuda.set_device(dev)
    name = args.config
    g = gridgen.make_grid(name)
    sc = gridgen.config_scenarios(name, g, batch=args.batch or None)
    S_np, V0_np = sc.sbus(g), sc.v0_flat(g)
    B = S_np.shape[0]
    plan = pf.Plan.from_branches(g.n, g.f, g.t, g.r, g.x, g.b, g.bus_type, lu_precision=args.lu, dense_frac=1.0)
    mp = pf.MultiPlan([plan], [B])
    Sd = torch.from_numpy(S_np.ravel()).to(dev)
    Vd = torch.from_numpy(V0_np.ravel()).to(dev)
    tuned = mp.autotune(Sd, Vd, TOL, args.maxit)
    out = mp._outs(Sd)
    stream = torch.cuda.current_stream()
    plan_mk = pf.Plan.from_branches(g.n, g.f, g.t, g.r, g.x, g.b, g.bus_type, lu_precision=args.lu)
    S2 = torch.from_numpy(S_np).to(dev)
    V2 = torch.from_numpy(V0_np).to(dev)

    def timed(fn):
        for _ in range(max(args.warmup, 3)):
            fn()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(args.steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / args.steps

    clocks = ClockSampler(dev.index or 0)
    clocks.start()
    time.sleep(0.3)
    ms = timed(lambda: mp.solve(Sd, Vd, TOL, args.maxit, out=out))
    ms_mk = timed(lambda: plan_mk.solve(S2, V2, TOL, args.maxit))
    clk = clocks.stop()
    it = out[1].cpu().numpy()
    st = out[2].cpu().numpy()
    conv = int(np.sum(st == 0))
    # end to end from pinned host memory through the fused path
    S_h, V_h = torch.from_numpy(S_np.ravel()).pin_memory(), torch.from_numpy(V0_np.ravel()).pin_memory()
    Vo = torch.empty_like(S_h).pin_memory()
    Sx, Vx = torch.empty_like(Sd), torch.empty_like(Vd)

    def e2e():
        Sx.copy_(S_h, non_blocking=True)
        Vx.copy_(V_h, non_blocking=True)
        v, i2, s2 = mp.solve(Sx, Vx, TOL, args.maxit, out=out)
        Vo.copy_(v, non_blocking=True)
    ms_e2e = timed(e2e)
    line = {
        "metric": METRIC, "value": conv / (ms / 1e3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if args.lu == "fp64" else "f64+f32lu", "data": "synthetic",
        "config": {"workload": name, "batch": B, "buses": g.n, "lu_precision": args.lu, "tol": TOL,
                   "maxit": args.maxit, "path": "fused persistent kernel, CUDA graph", "autotuned": tuned},
        "latency_us": 1e3 * ms, "multi_kernel_path_ms": ms_mk,
        "iterations": {"mean": float(it.mean()), "hist": np.bincount(it).tolist()}, "converged": conv,
        "clocks": clk, "e2e": {"value": conv / (ms_e2e / 1e3), "unit": UNIT, "h2d_bytes_per_step": int(2 * S_h.nbytes),
                               "d2h_bytes_per_step": int(S_h.nbytes)},
        "gpu_launches": 1,
        "roofline": whole_solve_roofline([(plan.info, 8 if args.lu == "fp64" else 4, int(it.sum()))], ms,
                                         "k_multi (the whole persistent solve)"),
    }
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = oracle_sample(g, S_np, V0_np, args.cpu_seconds, os.cpu_count() or 1)
    print(json.dumps(line), flush=True)


def vs_oracle(g, S, V0, Vg, itg, stg, idx, maxit):
    """The GPU's results on the sampled instances idx against the FP64 oracle
    (oracle/nrpf.py), each re-solved from the same start in spawn processes."""
    from oracle import nrpf
    idx = np.asarray(idx)
    Y = nrpf.make_ybus(g.n, g.f, g.t, g.r, g.x, g.b)
    cores = os.cpu_count() or 1
    Vo, ito, sto = nrpf.newton_batch(Y, S[idx], V0[idx], g.bus_type, TOL, maxit, workers=min(len(idx), cores))
    out = compare_with_oracle(Vg[idx], itg[idx], stg[idx], Vo, ito, sto)
    out["sample"] = "instances " + ",".join(str(int(i)) for i in idx)
    return out


def sample_indices(B, k=8, seed=0):
    """First, middle and last instance plus seeded random ones."""
    pick = {0, B // 2, B - 1}
    rng = np.random.default_rng(seed)
    while len(pick) < min(k, B):
        pick.add(int(rng.integers(B)))
    return sorted(pick)


def dense_update_launches_im(ndp):
    """The k_im_gemm launches of one instance-major dense refactor, each a list
    of (rows, columns, depth) pieces.  Left-looking by outer panels of 128:
    before panel j (at kj = 128 j, j > 0) is factorised, its block column and
    row take depth kj (rows [kj, ndp) x columns [kj, kj+c) and rows [kj, kj+c)
    x columns [kj+128, ndp), c = min(128, ndp-kj)) (the second 64-wide step's
    left-looking products are counted with the diagonal and panel kernels)."""
    out = []
    for kj in range(128, ndp, 128):
        c = min(128, ndp - kj)
        out.append([(ndp - kj, c, kj), (c, max(0, ndp - kj - 128), kj)])
    return out


def im_update_bytes(ndp, kj):
    """Algorithmic bytes of the k_im_gemm launch of outer panel kj, per
    instance: its block column and row read and written once (8 B per entry)
    and the operands L(kj:, :kj) and U(:kj, kj:) read once (4 B each)."""
    c = min(128, ndp - kj)
    entries = (ndp - kj) * c + c * max(0, ndp - kj - 128)
    return 8 * entries + 8 * kj * (ndp - kj)


def measure_mesh(args, pf, name, lu, steps, warmup, dev, rank=0, world=1, with_cpu=True, batch=None,
                 roof_steps=None, e2e=True):
    """One meshed-grid workload: K timed pf_solve_batch steps (graph-ended
    Newton loop, inputs in HBM), a per-launch-timed pass for the dominant
    kernel's roofline, the end-to-end rate through pf_solve_batch_host, the
    oracle comparison on sampled instances and (optionally) the CPU
    baselines.  Returns the JSON line as a dict."""
    import ctypes as C

    import torch
    import torch.distributed as dist

    from paper_2101_02270_gb300.solver import KERNEL_CLASSES

    n1 = name == "n1_2000"  # static N-1: every connected single outage x load levels
    g = gridgen.make_grid("mesh2000_b10k" if n1 else name)
    ins = None
    if n1:
        # rank r scales the load levels by (1 + 0.01 r) (weak scaling)
        _, _, ins, S_np = gridgen.n1_batch(g, levels=tuple(l * (1 + 0.01 * rank) for l in gridgen.N1_LEVELS))
        V0_np = np.broadcast_to(g.v_set.astype(np.complex128), S_np.shape).copy()
    else:
        sc = rank_scenarios(name, g, rank, batch=batch or args.batch or None)
        S_np, V0_np = sc.sbus(g), sc.v0_flat(g)
    B = S_np.shape[0]
    S = torch.from_numpy(S_np).to(dev)
    V0 = torch.from_numpy(V0_np).to(dev)
    t0 = time.perf_counter()
    plan = pf.Plan.from_branches(g.n, g.f, g.t, g.r, g.x, g.b, g.bus_type, lu_precision=lu,
                                 dense_frac=args.dense_frac, panel=args.panel, max_batch=B,
                                 dense_layout=args.dense_layout if lu == "fp32" else "auto")
    plan_ms = 1e3 * (time.perf_counter() - t0)
    out_np = np.argmin(ins, axis=1).astype(np.int32)[:, None] if n1 else None
    Od = torch.from_numpy(out_np).to(dev) if n1 else None
    info = plan.info
    im = info["dense_layout"] == 2
    fp64_peak, fp32_peak = pf._lib.fma_peak(C.c_void_p(torch.cuda.current_stream().cuda_stream))
    out = (torch.empty((B, g.n), dtype=torch.complex128, device=dev),
           torch.empty(B, dtype=torch.int32, device=dev), torch.empty(B, dtype=torch.uint8, device=dev))
    stream = torch.cuda.current_stream()

    def step():
        if n1:
            return plan.solve_outages(Od, S, V0, TOL, args.maxit, out=out)
        return plan.solve(S, V0, TOL, args.maxit, out=out)

    for _ in range(max(warmup, 0)):
        step()
    torch.cuda.synchronize()

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    clocks = ClockSampler(dev.index or 0)
    clocks.start()
    time.sleep(0.3)
    plan.profile_start([])  # launch counts only: the Newton loop runs as a graph
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    e0.record(stream)
    for _ in range(steps):
        step()
    e1.record(stream)
    barrier()
    ms = e0.elapsed_time(e1)
    counts = plan.profile_read()
    clk = clocks.stop()
    # per-kernel device times: timed steps again with CUDA events around
    # every launch of the timed classes, on the launch stream (the loop then
    # ends from the host; the kernels and their work are the same)
    rsteps = steps if roof_steps is None else max(1, min(steps, roof_steps))
    plan.profile_start(KERNEL_CLASSES if args.time_all else ["dense_update"])
    for _ in range(rsteps):
        step()
    prof = plan.profile_read()
    plan.profile_start([])  # per-launch timing off again: later solves run the graph loop
    iters = out[1].cpu().numpy()
    status = out[2].cpu().numpy()
    Vg = out[0].cpu().numpy()
    conv = int(np.sum(status == 0))
    ms_max, conv_all = combine_ranks(ms, conv, dev)
    value = conv_all * steps / (ms_max / 1e3)
    launches = int(sum(v[0] for v in counts.values()))

    # ---- end to end through the public API with host buffers ----
    # (pf_solve_batch_host: chunks of the batch copied in and out on the
    # plan's copy streams while the neighbouring chunks are solved)
    e2e_line = None
    if e2e:
        S_h = torch.from_numpy(S_np).pin_memory()
        V0_h = torch.from_numpy(V0_np).pin_memory()
        V_h = torch.empty((B, g.n), dtype=torch.complex128).pin_memory()
        it_h = torch.empty(B, dtype=torch.int32).pin_memory()
        st_h = torch.empty(B, dtype=torch.uint8).pin_memory()
        if n1:
            # the outage lists travel with the injections: copies in, solve, copies out
            O_h = torch.from_numpy(out_np).pin_memory()
            Sd, Vd, Odd = torch.empty_like(S), torch.empty_like(V0), torch.empty_like(Od)

            def e2e_step():
                Odd.copy_(O_h, non_blocking=True)
                Sd.copy_(S_h, non_blocking=True)
                Vd.copy_(V0_h, non_blocking=True)
                v, it, st = plan.solve_outages(Odd, Sd, Vd, TOL, args.maxit, out=out)
                V_h.copy_(v, non_blocking=True)
                it_h.copy_(it, non_blocking=True)
                st_h.copy_(st, non_blocking=True)
        else:
            def e2e_step():
                plan.solve_host(S_h, V0_h, TOL, args.maxit, out=(V_h, it_h, st_h), chunk=args.chunk)
        e2e_step()  # staging warm-up
        barrier()
        e0.record(stream)
        for _ in range(steps):
            e2e_step()
        e1.record(stream)
        barrier()
        ms_e2e, conv_e2e = combine_ranks(e0.elapsed_time(e1), int(np.sum(st_h.numpy() == 0)), dev)
        e2e_line = {"value": conv_e2e * steps / (ms_e2e / 1e3), "unit": UNIT,
                    "h2d_bytes_per_step": 2 * B * g.n * 16 + (out_np.nbytes if n1 else 0),
                    "d2h_bytes_per_step": B * g.n * 16 + B * 4 + B,
                    "api": ("pf_solve_batch_outages after page-locked host copies of the outage lists and injections"
                            if n1 else "pf_solve_batch_host (page-locked host buffers, copies overlapped across calls)")}

    # ---- roofline of the dominant kernel (dense trailing update) ----
    w = 8 if lu == "fp64" else 4
    ndp = info["dense_pad"]
    kb = info["panel"]
    refactors = int(iters.sum()) * rsteps  # one refactor per Newton update per instance
    du = prof["dense_update"]
    hbm, hbm_kind = measured_hbm()
    timing = (f"CUDA events around every dense_update launch on its stream, during a second pass of {rsteps} of "
              f"the {steps} timed steps")
    if im:
        du_flop = sum(2 * r * c * d for L in dense_update_launches_im(ndp) for r, c, d in L) * refactors
        achieved = du_flop / (du[2] / 1e3) / 1e12 if du[2] > 0 else None
        alg = [im_update_bytes(ndp, kj) for kj in range(128, ndp, 128)]
        roof = {"bound": "alu", "kernel": "dense_update (k_im_gemm, FP32 CTA-tiled product)", "achieved": achieved,
                "peak": fp32_peak, "unit": "TFLOP/s", "frac": (achieved / fp32_peak) if achieved else None,
                "traffic": (IM_GEMM_DRAM_PER_ALG * B * sum(alg) / len(alg)
                            if alg and IM_GEMM_DRAM_PER_ALG is not None else None),
                "traffic_kind": "ncu DRAM bytes over algorithmic bytes of one launch of a batch-64 capture, times "
                                "the batch and the mean algorithmic bytes of the refactor's launches",
                "peak_kind": "measured FP32 FMA-chain throughput (pf_fma_peak)",
                "launches": du[0], "ms_total": du[2], "timing": timing,
                "algorithmic_bytes": "per launch and instance: the panel's block column and row read and "
                                     "written once, the operands L(kj:, :kj) and U(:kj, kj:) read once"}
    elif lu == "fp64":
        du_flop = dense_update_flop(ndp, kb) * refactors
        achieved = du_flop / (du[2] / 1e3) / 1e12 if du[2] > 0 else None
        r2 = [(ndp - k - kb) ** 2 for k in range(0, ndp, kb) if ndp - k - kb > 0]
        traffic = (DENSE_UPDATE_DRAM_B_PER_R2 * B * sum(r2) / len(r2) if r2 and kb == 8 else None)
        roof = {"bound": "alu", "kernel": "dense_update", "achieved": achieved, "peak": fp64_peak,
                "unit": "TFLOP/s", "frac": (achieved / fp64_peak) if achieved else None, "traffic": traffic,
                "peak_kind": "measured FP64 FMA-chain throughput (pf_fma_peak)",
                "traffic_kind": "ncu DRAM bytes per average active launch, scaled from a batch-640 capture",
                "launches": du[0], "ms_total": du[2], "timing": timing}
    else:
        du_flop = dense_update_flop(ndp, kb) * refactors
        achieved = du_flop / (du[2] / 1e3) / 1e12 if du[2] > 0 else None
        du_bytes = dense_update_bytes(ndp, kb, w) * refactors
        active_launches = len(dense_update_launches(ndp, kb)) * int(iters.max()) * rsteps
        gbs = du_bytes / (du[2] / 1e3) / 1e9 if du[2] > 0 else None
        roof = {"bound": "hbm", "kernel": "dense_update", "achieved": gbs, "peak": hbm, "unit": "GB/s",
                "frac": (gbs / hbm) if gbs else None,
                "traffic": (DENSE_UPDATE_FP32_DRAM_PER_ALG * du_bytes / max(active_launches, 1)
                            if DENSE_UPDATE_FP32_DRAM_PER_ALG is not None else None),
                "traffic_kind": "ncu DRAM bytes / algorithmic bytes of a batch-640 depth-64 capture, times the "
                                "algorithmic bytes per launch",
                "peak_kind": f"{hbm_kind} HBM copy bandwidth", "fp32_tflops": achieved, "fp32_peak_tflops": fp32_peak,
                "launches": du[0], "ms_total": du[2], "timing": timing}
    # whole-step HBM roofline (metric's second half): algorithmic bytes per
    # instance-iteration = LU written once and read once + voltages, injections,
    # rhs and solution
    nnz_lu = info["nnz_lu"]
    bmin = 2 * w * nnz_lu + 8 * (8 * g.n + 4 * info["m"])
    step_bytes = bmin * int(iters.sum())
    hbm_pct = 100.0 * (step_bytes * steps / (ms_max / 1e3) / 1e9) / hbm

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": steps,
        "warmup": warmup, "ms_per_step": ms_max / steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64" if lu == "fp64" else "f64+f32lu",
        "data": "synthetic",
        "config": {"workload": name, "batch_per_gpu": B, "buses": g.n, "branches": g.n_branch,
                   "unknowns": info["m"], "lu_precision": lu, "tol": TOL, "maxit": args.maxit,
                   "load_scale": g.load_scale, "dense_block": info["dense_dim"], "dense_pad": ndp, "panel": kb,
                   "dense_layout": "instance-major" if im else "interleaved",
                   "parallelism": f"instances split over {world} GPU(s)",
                   "l2": f"working set > L2: LU workspace {nnz_lu * w * B / 1e9:.1f} GB per GPU",
                   "plan_ms": round(plan_ms, 1)},
        "iterations": {"mean": float(iters.mean()), "max": int(iters.max()),
                       "hist": np.bincount(iters).tolist()},
        "converged": conv, "failed": int(np.sum(status == 2)),
        "roofline": roof,
        "hbm_roofline": {"algorithmic_bytes_per_instance_iteration": bmin,
                         "achieved_gbs": step_bytes * steps / (ms_max / 1e3) / 1e9,
                         "peak_gbs": hbm, "peak_kind": hbm_kind, "pct": hbm_pct},
        "kernel_ms": {k: round(v[2], 3) for k, v in prof.items() if v[1] > 0},
        "clocks": clk,
        "gpu_launches": launches,
    }
    if e2e_line is not None:
        line["e2e"] = e2e_line
    if n1:
        line["config"].update({"contingencies": int(B // len(gridgen.N1_LEVELS)),
                               "load_levels": list(gridgen.N1_LEVELS),
                               "case": "every single-branch outage that keeps the grid connected, per-instance "
                                       "admittances built on the device from the base values and the outaged "
                                       "branch (pf_solve_batch_outages), one injection profile per load level"})
    if rank == 0 and world == 1:
        if with_cpu and not args.no_cpu_baseline:
            # the timed oracle sample is also the oracle comparison
            cb = oracle_sample(g, S_np, V0_np, args.cpu_seconds, os.cpu_count() or 1, ins, gpu=(Vg, iters, status))
            line["vs_oracle"] = dict(cb.pop("vs_oracle"), sample=cb["sample"].split(",")[0])
            line["cpu_baseline"] = cb
            if not n1 and g.n <= 2000:
                line["cpu_batched"] = cpu_batched_sample(pf, g, S_np, V0_np, args.cpu_seconds)
        elif not n1 and not args.no_oracle:
            line["vs_oracle"] = vs_oracle(g, S_np, V0_np, Vg, iters, status, sample_indices(B), args.maxit)
    plan.close()
    del S, V0, out
    torch.cuda.empty_cache()
    return line


def summary(line):
    """The keys of a workload's line kept when it rides along as an extra."""
    keep = ("value", "unit", "ms_per_step", "steps", "warmup", "dtype", "config", "iterations", "converged", "failed",
            "roofline", "hbm_roofline", "e2e", "vs_oracle", "cpu_baseline", "cpu_batched", "gpu_launches", "clocks")
    return {k: line[k] for k in keep if k in line}


def run_ours(args):
    import torch
    import torch.distributed as dist

    import paper_2101_02270_gb300 as pf

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    big = args.config == "mesh9000_b10k"
    roof = args.roofline_steps or (4 if big else None)
    line = measure_mesh(args, pf, args.config, args.lu, args.steps, args.warmup, dev, rank, world, roof_steps=roof)
    if big and rank == 0 and world == 1 and not args.no_extras:
        # plain FP64 on the first 320 instances of the same batch: the
        # iteration and accuracy change of the FP32 LU, and its speed-up
        sub = measure_mesh(args, pf, "mesh9000_b10k", "fp64", 1, 1, dev, with_cpu=False, batch=320, e2e=False)
        line["fp64_subset"] = summary(sub)
        extra_steps, extra_warm = min(args.steps, 10), min(args.warmup, 3)
        line["extras"] = {
            "mesh2000_b10k_fp64": summary(measure_mesh(args, pf, "mesh2000_b10k", "fp64", extra_steps, extra_warm, dev)),
            "mesh2000_b10k_fp32lu": summary(measure_mesh(args, pf, "mesh2000_b10k", "fp32", extra_steps, extra_warm,
                                                         dev, with_cpu=False)),
            "warmstart2000": warmstart_measure(args, extra_steps, extra_warm),
        }
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def main():
    args = parse_args()
    args.lu_explicit = args.lu is not None
    if args.lu is None:
        args.lu = "fp32" if args.config == "mesh9000_b10k" else "fp64"
    if args.impl == "reference":
        run_reference(args)
    elif args.config == "feeders256x100":
        run_feeders(args)
    elif args.config == "warmstart2000":
        run_warmstart(args)
    elif args.config == "mesh30_b64":
        run_small(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
