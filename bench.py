#!/usr/bin/env python3
"""Benchmark of the non-polynomial RBF-ENO/WENO finite-volume hot path on one GB300 per rank.

Headline (one "step" = one whole solve of the batch): 4096 periodic Burgers instances on
[0, 2 pi], N log-uniform in [64, 8192] (seeded), u0 = 1 + four Fourier modes + up to two
jumps, Gaussian perturbation with the monotone switch, Lax-Friedrichs flux, TVD-RK3 at CFL 0.5,
run past shock formation to T = 1.5.  Float state, candidates, weights and flux; the shape
parameter in FP64; switch and ENO decisions certified equal to their FP64 evaluation.  Each
instance keeps its own dt; every instance fits in shared memory, so the batch runs in the
resident whole-solve kernel (four size classes on side streams).

The same JSON line carries one block per other workload (rank 0, N = 1):
  advection_fp64_n200    linear advection of sin(pi x), FP64, N = 200, CFL 0.5, T = 2, with the
                         convergence sweep N = 25..400 and the solve latency;
  euler1d_component      512 transmissive 1D Euler instances, N log-uniform in [256, 65536],
                         Riemann and Shu-Osher-type data, to their end times (work-queue kernel);
  euler1d_characteristic the same batch characteristic-wise (to a fraction of the end times);
  euler2d                periodic 2D Euler squares 256^2 .. 2048^2 (2^24 cells per size),
                         vortex and four-quadrant data, 100 RK3 steps (work-queue kernel);
  serving                a Poisson request stream served with continuous batching.
Each block has its roofline on the algorithmic HBM bytes of a cell-update, and the FP64
oracle timed on the host cores on a bounded sample, whose results also give the block's L1 /
L_inf difference from the oracle.

`--impl reference` times the FP64 CPU oracle instead, on a bounded sample of the headline
workload.
"""
from __future__ import annotations

import argparse
import ctypes
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_1602_00182_gb300 import inputs as I  # noqa: E402

WORKLOAD = ("batched 1D Burgers u_t+(u^2/2)_x=0 on [0,2pi], periodic: 4096 instances, N log-uniform [64,8192], "
            "u0=1+4 Fourier modes+<=2 jumps, RBF-WENO5 Gaussian + monotone switch, LF flux, TVD-RK3 CFL 0.5 to T=1.5")
T_END = 1.5
CFL = 0.5
SAMPLE_STRIDE = 64     # cpu sample: every 64th instance of the N-sorted batch
SAMPLE_STEPS = 20      # RK3 steps per sampled instance
FLUSH_BYTES = 256 * 1024 * 1024  # > L2 (129 MB)
MIXED_GUARD = 8.0 * 2.0 ** -24  # the mixed path's automatic round-off guard, given to the oracle

# Algorithmic HBM bytes of one cell-update (one cell, all fields, one full RK3 step) of the
# per-stage fused design: stage 1 reads u^n and writes u1, stages 2 and 3 read the stage input
# and u^n and write: 8 + 12 + 12 = 32 B per float field, 64 B per double field.
BYTES_SCALAR_F32 = 32
BYTES_EULER1D_F32 = 96
BYTES_EULER2D_F32 = 128
BYTES_SCALAR_F64 = 64
# FP64-pipe instructions of one shape-parameter evaluation in the mixed path with eta_eval 1
# (k = 3): 2 adds (the differences a, b), 2 multiply-adds (numerator, denominator), 1 add
# (eps_M), 1 multiply and 2 multiply-adds (the Newton quotient); the default eta_eval 0 uses none
FP64_OPS_PER_ETA = 8
# FP64 pipe: 2 instructions per clock per SM (1.25 TFLOP/s nominal FP64 over 152 SMs at 2.07 GHz)
FP64_PIPE_PEAK = 2.0 * 152 * 2.07e9


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def roofline_hbm(bytes_per_cu: int, cell_updates: float, seconds: float, kernel: str, traffic=None, **extra):
    """Roofline on the algorithmic bytes: achieved = bytes per cell-update x cell-updates of the
    dominant kernel / its CUDA-event time, against the measured copy bandwidth."""
    peak, src = _peaks()
    achieved = bytes_per_cu * cell_updates / seconds / 1e9 if seconds > 0 else None
    out = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
           "frac": (achieved / peak) if achieved else None, "traffic": traffic, "kernel": kernel,
           "bytes_per_cell_update": bytes_per_cu, "peak_source": f"{src} (hbm_gbs)"}
    out.update(extra)
    return out


# ------------------------------------------------------------------------------- clocks
class Clocks:
    def __init__(self, path):
        self.path = path
        self.proc = None

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                          "-lms", "200"], stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self, gpu_index: int):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9 or not f[0].isdigit() or int(f[0]) != gpu_index:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


class npw_profile(ctypes.Structure):
    _fields_ = [("kernel_launches", ctypes.c_int64), ("stage_launches", ctypes.c_int64), ("stage_ms", ctypes.c_double),
                ("timed_launches", ctypes.c_int64), ("resident_launches", ctypes.c_int64 * 4),
                ("resident_ms", ctypes.c_double * 4)]


class Profiled:
    """npw_profile counters around a region (launch counts, stage-kernel and resident event times)."""

    def __init__(self, lib):
        self.lib = lib
        self.pr = npw_profile()

    def __enter__(self):
        self.lib.npw_profile_reset()
        self.lib.npw_profile_enable(1)
        return self

    def __exit__(self, *a):
        self.lib.npw_profile_read(ctypes.byref(self.pr))
        self.lib.npw_profile_enable(0)


def kernel_source_hash() -> str:
    """sha256 over the device sources (ncu figures are valid only for the sources they were
    taken from)."""
    import hashlib
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1602_00182_gb300", "csrc")
    for f in ("npw_internal.h", "npw_device.cuh", "npw_fast.cuh", "npw_kernels.cuh", "npw_fp32.cu", "npw_queue.inc",
              "npw_queue_fp32.cu"):
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _ncu_traffic(key: str):
    """DRAM bytes per launch of a dominant launch from the committed ncu summary, when it was
    taken from the current kernel sources (null otherwise)."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as fh:
            d = json.load(fh)
        if d.get("kernel_source_sha256") != kernel_source_hash():
            return None
        return d.get(key)
    except Exception:
        return None


def _timed_event(fn, stream, flush):
    """One call between CUDA events on the launching stream, L2 flushed before."""
    import torch
    flush.fill_(1.0)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    r = fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1), r


# ------------------------------------------------------------------------------- headline (C2)
def headline_burgers(args, rank, world, local_rank):
    import torch
    import paper_1602_00182_gb300.npweno as npw

    lib = npw.load()
    dev = torch.device("cuda", local_rank)
    inst = I.burgers_batch(count=args.instances, seed_index=rank_seed(1, rank))
    # largest instances first in the arena (the work list follows the arena order)
    order = sorted(range(len(inst)), key=lambda i: -inst[i].n)
    ns = [inst[i].n for i in order]
    table, total = npw.make_instances(ns, [inst[i].dx for i in order], [args.t_end] * len(order), [CFL] * len(order),
                                      [npw.NPW_BC_PERIODIC] * len(order))
    host0 = np.concatenate([inst[i].u0[0] for i in order]).astype(np.float32)
    params = npw.Params(rbf=npw.NPW_RBF_GA, precision=npw.NPW_FP32_MIXED, eta_eval=args.eta_eval)
    pristine = torch.tensor(host0, device=dev)
    arena = pristine.clone()
    ws = torch.empty(npw.npw_batch_workspace_size(table, 1, params), dtype=torch.uint8, device=dev)
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def one_solve():
        st, stats = npw.npweno_batch_solve(arena, table, 1, npw.NPW_FLUX_BURGERS, params, workspace=ws)
        if st != 0:
            raise RuntimeError(f"batch solve failed with status {st}")
        return stats

    for _ in range(args.warmup):
        arena.copy_(pristine)
        stats = one_solve()
    cell_updates = sum(n * s["steps"] for n, s in zip(ns, stats))

    times = []
    clocks = Clocks(os.path.join(args.out_dir, f"clocks_rank{rank}.csv"))
    with Profiled(lib) as prof, clocks:
        for _ in range(args.steps):
            arena.copy_(pristine)
            flush.fill_(1.0)  # evict the working set from L2 between timed steps
            if world > 1:
                torch.distributed.barrier()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            stats = one_solve()
            e1.record(stream)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
    pr = prof.pr
    tmax, cu_all = job_totals(sum(times), cell_updates * args.steps, world, dev)
    value = cu_all / (tmax / 1e3)
    result_host = arena.cpu().numpy()  # the last timed solve's states (accuracy sample)

    # roofline of the dominant kernel: the resident class n > 4096 (~3/4 of the work)
    big = [k for k, n in enumerate(ns) if n > 4096]
    cu_a = sum(ns[k] * stats[k]["steps"] for k in big) * args.steps
    faces_a = sum((ns[k] + 1) * 3 * stats[k]["steps"] for k in big) * args.steps
    res_s = pr.resident_ms[0] / 1e3
    secondary = {"hbm_bytes_actually_moved": "8 B per cell per solve: the state stays in shared memory"}
    if args.eta_eval == 1 and res_s > 0:
        fp64 = FP64_OPS_PER_ETA * faces_a / res_s / 1e9
        secondary["fp64_pipe"] = {"achieved": fp64, "peak": FP64_PIPE_PEAK / 1e9, "unit": "G FP64-pipe instr/s",
                                  "frac": fp64 / (FP64_PIPE_PEAK / 1e9),
                                  "count": f"{FP64_OPS_PER_ETA} per face and stage (eta), all n+1 faces"}
    else:
        secondary["fp64_pipe"] = "no FP64 instruction on the common path (eta from float pairs)"
    roof = roofline_hbm(BYTES_SCALAR_F32, cu_a, res_s,
                        "solve1d_resident_kernel<BURGERS, 3>, size class n > 4096 (512 threads, 2 CTAs/SM)",
                        traffic=_ncu_traffic("solve1d_resident_burgers_classA_dram_bytes_per_launch"),
                        secondary=secondary,
                        resident_launches=[int(x) for x in pr.resident_launches],
                        resident_ms=[float(x) for x in pr.resident_ms],
                        kernel_source_sha256=kernel_source_hash())

    # decisions of the shape parameter over the batch (the bound is off: the printed eta)
    eta_tot = {k: sum(s["eta"][k] for s in stats) for k in ("switch", "eval", "guard", "bound")}
    faces_tot = eta_tot["switch"] + eta_tot["eval"]

    # end to end through the C ABI with host buffers: H2D of the initial state, the solve,
    # D2H of the result, per step
    pinned_in = torch.from_numpy(host0).pin_memory()
    pinned_out = torch.empty_like(pinned_in).pin_memory()
    e2e_times = []
    for _ in range(args.steps):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        arena.copy_(pinned_in, non_blocking=True)
        one_solve()
        pinned_out.copy_(arena, non_blocking=True)
        torch.cuda.synchronize()
        e2e_times.append(time.perf_counter() - t0)
    e2e_ms, e2e_units = job_totals(1e3 * sum(e2e_times), cell_updates * args.steps, world, dev)
    e2e_value = e2e_units / (e2e_ms / 1e3)

    variants = {}

    def time_variant(pv, label):
        arena.copy_(pristine)
        npw.npweno_batch_solve(arena, table, 1, npw.NPW_FLUX_BURGERS, pv, workspace=ws)
        vt = []
        for _ in range(args.variant_steps):
            arena.copy_(pristine)
            ms, (st, vstats) = _timed_event(
                lambda: npw.npweno_batch_solve(arena, table, 1, npw.NPW_FLUX_BURGERS, pv, workspace=ws), stream, flush)
            vt.append(ms)
        vcu = sum(n * s["steps"] for n, s in zip(ns, vstats))
        variants[label] = {"value": vcu * len(vt) / (sum(vt) / 1e3), "unit": "cell-updates/s",
                           "ms_per_step": sum(vt) / len(vt)}

    if args.variant_steps > 0 and args.eta_eval == 0 and world == 1:
        time_variant(npw.Params(rbf=npw.NPW_RBF_GA, precision=npw.NPW_FP32_MIXED, eta_eval=1),
                     f"eta_eval=1 (eta in FP64, {FP64_OPS_PER_ETA} FP64-pipe instructions per face and stage)")
        time_variant(npw.Params(k=2, rbf=npw.NPW_RBF_GA, precision=npw.NPW_FP32_MIXED, eta_max=1.0),
                     "k=2 RBF-WENO3 Gaussian + switch (Table k2; resident kernels, eta in FP64), |eta| <= 1 "
                     "(the printed k = 2 eta is singular where u crosses zero)")
        # the schemes the paper compares, side by side on the same batch (Sec. 5.2: RBF-ENO costs
        # a little more than ENO and less than WENO)
        for k, sch, name in ((3, npw.NPW_ENO, "ENO3"), (3, npw.NPW_WENO_JS, "WENO-JS5"), (3, npw.NPW_RBF_ENO, "RBF-ENO3"),
                             (2, npw.NPW_ENO, "ENO2"), (2, npw.NPW_WENO_JS, "WENO-JS3"), (2, npw.NPW_RBF_ENO, "RBF-ENO2")):
            rbf_k2 = k == 2 and sch == npw.NPW_RBF_ENO
            time_variant(npw.Params(k=k, scheme=sch, rbf=npw.NPW_RBF_GA, precision=npw.NPW_FP32_MIXED,
                                    eta_max=1.0 if rbf_k2 else 0.0),
                         f"scheme {name}" + (" (Gaussian, switch, |eta| <= 1)" if rbf_k2 else
                                             " (Gaussian, switch)" if sch == npw.NPW_RBF_ENO else ""))

    out = {
        "metric": "cell-updates/s",
        "value": value,
        "unit": "cell-updates/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": tmax / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic (seeded)",
        "impl": "ours",
        "config": {
            "workload": WORKLOAD,
            "instances": len(ns),
            "cells": int(sum(ns)),
            "cell_updates_per_step": int(cell_updates),
            "precision": ("NPW_FP32_MIXED: f32 state, candidates, beta, weights, flux, update; eta "
                          + ("from exact differences as float pairs, double-float quotient" if args.eta_eval == 0
                             else "in FP64") +
                          f" (eta_eval={args.eta_eval}); switch decisions equal to FP64 evaluation; eta as printed "
                          "(no bound)"),
            "l2": "flushed (256 MB write) before every timed step; working set 3 x 4 B x cells",
            "parallelism": f"independent instance batches, one per rank (x{world})",
        },
        "roofline": roof,
        "eta_decisions": {"faces": faces_tot, **eta_tot,
                          "switch_frac": eta_tot["switch"] / faces_tot if faces_tot else None,
                          "bound_frac": eta_tot["bound"] / faces_tot if faces_tot else None,
                          "guard_frac": eta_tot["guard"] / faces_tot if faces_tot else None,
                          "note": "per face and stage over the batch; guard: the float round-off guard of the "
                                  "mixed path; bound: off (the printed eta)"},
        "e2e": {"value": e2e_value, "unit": "cell-updates/s", "h2d_bytes_per_step": int(host0.nbytes),
                "d2h_bytes_per_step": int(host0.nbytes)},
        "gpu_launches": int(pr.kernel_launches),
        "variants": variants,
        "clocks": clocks.summary(local_rank),
    }
    sample = {"order": order, "ns": ns, "host0": host0, "result": result_host, "inst": inst}
    return out, sample


# ------------------------------------------------------------------------------- C1
def block_advection(args):
    """Sec. 5.2 Ex. 1 setting at the configuration's FP64: sin(pi x) on [-1, 1], periodic,
    RBF-WENO5 (multiquadric) with the switch, LF, TVD-RK3 at CFL 0.5 to T = 2 (400 steps at
    N = 200); solve latency and cell-updates/s through npweno_solve, and the convergence sweep
    N = 25..400 against the exact cell averages (the RK3 time error dominates at CFL 0.5)."""
    import torch
    import paper_1602_00182_gb300.npweno as npw
    lib = npw.load()
    p = npw.Params()
    u0, dx = I.advection_sin(200)
    dev_u = torch.empty(200, dtype=torch.float64, device="cuda")
    pristine = torch.tensor(u0, device="cuda")
    ws = torch.empty(npw.npw_workspace_size(200, 1, p), dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    for _ in range(3):
        dev_u.copy_(pristine)
        npw.npweno_solve(dev_u, dx, 2.0, 0.5, npw.NPW_FLUX_ADVECTION, npw.NPW_BC_PERIODIC, p, workspace=ws)
    lat_dev, lat_host = [], []
    with Profiled(lib) as prof:
        for _ in range(20):
            dev_u.copy_(pristine)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            st = npw.npweno_solve(dev_u, dx, 2.0, 0.5, npw.NPW_FLUX_ADVECTION, npw.NPW_BC_PERIODIC, p, workspace=ws)
            e1.record(stream)
            torch.cuda.synchronize()
            lat_host.append(time.perf_counter() - t0)
            lat_dev.append(e0.elapsed_time(e1))
    result = dev_u.cpu().numpy()
    cu = 200 * st["steps"]
    ms = statistics.median(lat_dev)
    stage_s = prof.pr.stage_ms / 1e3
    sweep = {}
    for n in (25, 50, 100, 200, 400):
        un, dxn = I.advection_sin(n)
        g = torch.tensor(un, device="cuda")
        npw.npweno_solve(g, dxn, 2.0, 0.5, npw.NPW_FLUX_ADVECTION, npw.NPW_BC_PERIODIC, p)
        ex, _ = I.advection_sin(n, shift=2.0)
        e = np.abs(g.cpu().numpy() - ex)
        sweep[n] = {"l1": float(e.mean()), "linf": float(e.max())}
    ns = sorted(sweep)
    orders = [float(np.log(sweep[a]["l1"] / sweep[b]["l1"]) / np.log(b / a)) for a, b in zip(ns, ns[1:])]
    return {
        "metric": "cell-updates/s", "value": cu / (ms / 1e3), "unit": "cell-updates/s", "dtype": "f64",
        "latency_ms": {"device_median": ms, "host_median": 1e3 * statistics.median(lat_host),
                       "host_p99": 1e3 * float(np.percentile(lat_host, 99))},
        "config": {"workload": "1D linear advection u_t+u_x=0 on [-1,1], periodic, u0=sin(pi x), N=200, FP64, "
                               "RBF-WENO5 multiquadric + monotone switch, LF, TVD-RK3 CFL 0.5 to T=2",
                   "steps": st["steps"], "cell_updates": cu, "timed_solves": len(lat_dev)},
        "convergence_vs_exact": {"l1_linf": {str(n): sweep[n] for n in ns}, "l1_orders": orders,
                                 "note": "at CFL 0.5 the RK3 time error dominates WENO5's spatial error: order ~3"},
        "roofline": roofline_hbm(BYTES_SCALAR_F64, cu * len(lat_dev), stage_s, "stage1d_kernel<double, ADVECTION>",
                                 note="a latency-bound case: 200 cells, 1200 stage launches per solve"),
        "gpu_launches_per_solve": int(prof.pr.kernel_launches / len(lat_dev)),
    }, {"u0": u0, "dx": dx, "result": result, "steps": st["steps"]}


# ------------------------------------------------------------------------------- C3
def block_euler1d(args, characteristic: int):
    """512 transmissive Euler instances (m = 3), N log-uniform in [256, 65536], Riemann and
    Shu-Osher-type data, through the work-queue kernel (mixed precision; instances that fit in
    shared memory run in the resident kernel beside it), to t_frac x each end time."""
    import torch
    import paper_1602_00182_gb300.npweno as npw
    lib = npw.load()
    inst = I.euler_batch(count=512, seed_index=2)
    t_frac = args.euler_t_frac if not characteristic else args.euler_char_t_frac
    specs = [dict(kind=npw.NPW_FLUX_EULER1D, nx=it.n, dx=it.dx, t_end=t_frac * it.t_end, cfl=CFL, bc=1) for it in inst]
    table, total, offs = npw.make_queue_instances(specs)
    host0 = np.concatenate([it.u0.ravel() for it in inst]).astype(np.float32)
    pristine = torch.tensor(host0, device="cuda")
    arena = pristine.clone()
    # characteristic runs bound |eta| by 1 (the printed eta of a characteristic field blows up at
    # the foot of the Mach-3 shock of the Shu-Osher-type data)
    eta_max = 1.0 if characteristic else 0.0
    p = npw.Params(precision=npw.NPW_FP32_MIXED, characteristic=characteristic, eta_max=eta_max)
    tile = npw.npw_autotune_1d(npw.NPW_FLUX_EULER1D, 3, p)  # later runs with tile_1d = 0 use it
    if args.euler_tile > 0:
        p.tile_1d = tile = args.euler_tile
    elif not characteristic:
        # the library's rule for fused steps: the tuned tile, halved while six arrays of
        # tile + 18 cells x 3 fields exceed 44 KB
        while tile > 256 and 6 * (tile + 18) * 3 * 4 > 44 * 1024:
            tile //= 2
    ws = torch.empty(npw.npw_queue_workspace_size(table, p), dtype=torch.uint8, device="cuda")
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    # warm-up on a short run (graph capture, attributes)
    wtable, _, _ = npw.make_queue_instances([dict(sp, t_end=0.02 * sp["t_end"]) for sp in specs])
    npw.npweno_queue_solve(arena, wtable, p, workspace=ws)
    arena.copy_(pristine)
    clocks = Clocks(os.path.join(args.out_dir, f"clocks_euler1d_{characteristic}.csv"))
    with Profiled(lib) as prof, clocks:
        ms, (st, stats) = _timed_event(lambda: npw.npweno_queue_solve(arena, table, p, workspace=ws), stream, flush)
    if st != 0:
        raise RuntimeError(f"euler1d queue solve failed with status {st}")
    ns = [it.n for it in inst]
    cu = sum(n * s["steps"] for n, s in zip(ns, stats))
    res_limit = 5682  # resident instances (three 3 (n + 6)-float arrays within 200 KiB)
    cu_queue = sum(n * s["steps"] for n, s in zip(ns, stats) if characteristic or n > res_limit)
    stage_s = prof.pr.stage_ms / 1e3
    eta_tot = {k: sum(s["eta"][k] for s in stats) for k in ("switch", "eval", "guard", "bound")}
    kern = ("queue_stage_kernel<float, K=3, characteristic, 1D Euler> (face-based Roe-field body)" if characteristic
            else "queue_stage_kernel_b5<float, K=3, 1D Euler> (fused RK3 step body)")
    return {
        "metric": "cell-updates/s", "value": cu / (ms / 1e3), "unit": "cell-updates/s", "dtype": "f32",
        "ms_per_solve": ms,
        "config": {"workload": ("batched 1D Euler (m=3, gamma=1.4), transmissive: 512 instances, N log-uniform "
                                "[256,65536], Riemann + Shu-Osher-type data, "
                                f"{'characteristic' if characteristic else 'component'}-wise, RBF-WENO5 MQ + switch"
                                f"{', |eta| <= 1' if characteristic else ''}, LF, TVD-RK3 CFL 0.5 to "
                                f"{t_frac} x each end time"),
                   "instances": 512, "cells": int(sum(ns)), "cell_updates": int(cu), "tile_1d": tile,
                   "path": ("npweno_queue_solve: persistent work-queue stage kernel, steps replayed as CUDA graphs"
                            if characteristic else
                            "npweno_queue_solve: persistent work-queue kernel, one fused launch per RK3 step (u^n "
                            "loaded once with a 9-cell halo, three stages in shared memory), steps replayed as CUDA "
                            "graphs; instances with n <= 5682 in the resident kernel beside it"),
                   "l2": "flushed before the timed solve"},
        "roofline": roofline_hbm(BYTES_EULER1D_F32, cu_queue, stage_s, kern,
                                 traffic=None if characteristic else _ncu_traffic("queue_stage_euler1d_dram_bytes_per_launch"),
                                 traffic_unit="bytes per stage launch over the batch's queued items",
                                 stage_launches=int(prof.pr.stage_launches), stage_ms=prof.pr.stage_ms),
        "eta_decisions": eta_tot,
        "gpu_launches": int(prof.pr.kernel_launches),
        "clocks": clocks.summary(0),
    }, {"inst": inst, "host0": host0, "offs": offs, "result": arena.cpu().numpy(), "t_frac": t_frac,
        "characteristic": characteristic, "eta_max": eta_max}


# ------------------------------------------------------------------------------- C4
def block_euler2d(args):
    """2D Euler, dimension by dimension, on periodic squares 256^2, 512^2, 1024^2, 2048^2: per
    size a batch of 2^24 cells (256, 64, 16, 4 squares; vortex and four-quadrant data), ~100 RK3
    steps at CFL 0.5, all squares of a size in one work-queue batch."""
    import torch
    import paper_1602_00182_gb300.npweno as npw
    lib = npw.load()
    p = npw.Params(precision=npw.NPW_FP32_MIXED)
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    sizes = {}
    tot_cu, tot_ms, tot_stage_s, tot_launch = 0, 0.0, 0.0, 0
    for n in args.sizes2d:
        count = max(1, (1 << 24) // (n * n))
        doms = I.euler2d_batch(n, count, seed_index=3)
        specs, fields = [], []
        for U, d in doms:
            rho, mx, my, E = U
            u, v = mx / rho, my / rho
            c = np.sqrt(1.4 * 0.4 * (E - 0.5 * rho * (u * u + v * v)) / rho)
            rate = (np.abs(u) + c).max() / d + (np.abs(v) + c).max() / d
            specs.append(dict(kind=npw.NPW_FLUX_EULER2D, nx=n, ny=n, dx=d, dy=d, t_end=args.steps2d * CFL / rate,
                              cfl=CFL, bc=0))
            fields.append(U.astype(np.float32).ravel())
        table, total, offs = npw.make_queue_instances(specs)
        pristine = torch.tensor(np.concatenate(fields), device="cuda")
        arena = pristine.clone()
        ws = torch.empty(npw.npw_queue_workspace_size(table, p), dtype=torch.uint8, device="cuda")
        wtable, _, _ = npw.make_queue_instances([dict(sp, t_end=0.05 * sp["t_end"]) for sp in specs])
        npw.npweno_queue_solve(arena, wtable, p, workspace=ws)  # warm-up
        arena.copy_(pristine)
        with Profiled(lib) as prof:
            ms, (st, stats) = _timed_event(lambda: npw.npweno_queue_solve(arena, table, p, workspace=ws), stream, flush)
        if st != 0:
            raise RuntimeError(f"euler2d queue solve failed with status {st}")
        cu = n * n * sum(s["steps"] for s in stats)
        sizes[f"{n}^2"] = {"domains": count, "value": cu / (ms / 1e3), "ms_per_solve": ms,
                           "steps": [min(s["steps"] for s in stats), max(s["steps"] for s in stats)],
                           "roofline_frac": roofline_hbm(BYTES_EULER2D_F32, cu, prof.pr.stage_ms / 1e3, "")["frac"]}
        tot_cu += cu
        tot_ms += ms
        tot_stage_s += prof.pr.stage_ms / 1e3
        tot_launch += int(prof.pr.kernel_launches)
        del arena, pristine, ws
    return {
        "metric": "cell-updates/s", "value": tot_cu / (tot_ms / 1e3), "unit": "cell-updates/s", "dtype": "f32",
        "config": {"workload": ("2D Euler dimension by dimension, periodic squares 256^2..2048^2 (2^24 cells per size: "
                                "isentropic vortex + four-quadrant), RBF-WENO5 MQ + switch, one midpoint point per face, "
                                f"~{args.steps2d} RK3 steps at CFL 0.5"),
                   "path": "npweno_queue_solve: all squares of a size in one persistent work-queue batch",
                   "l2": "flushed before every timed solve"},
        "sizes": sizes,
        "roofline": roofline_hbm(BYTES_EULER2D_F32, tot_cu, tot_stage_s,
                                 "queue_stage_kernel_b5<float, K=3, 2D Euler> (phased 2D body, 32 x 8 tiles)",
                                 traffic=_ncu_traffic("queue_stage_euler2d_512_dram_bytes_per_launch"),
                                 traffic_unit="bytes per stage launch, 64 squares of 512^2 (2^24 cells, every size's "
                                              "launch)"),
        "gpu_launches": tot_launch,
    }


def accuracy_run_2d(npw, n=256, steps=5):
    """Two squares of the 2D workload (vortex, four-quadrant) advanced ~steps RK3 steps on the
    GPU (mixed precision); the oracle runs on the same float data in the CPU leg."""
    import torch
    doms = I.euler2d_batch(n, 2, seed_index=3)
    specs, fields, data = [], [], []
    for U, d in doms:
        U32 = U.astype(np.float32)
        rho, mx, my, E = U32.astype(np.float64)
        u, v = mx / rho, my / rho
        c = np.sqrt(1.4 * 0.4 * (E - 0.5 * rho * (u * u + v * v)) / rho)
        rate = (np.abs(u) + c).max() / d + (np.abs(v) + c).max() / d
        t_end = 0.999 * steps * CFL / rate
        specs.append(dict(kind=npw.NPW_FLUX_EULER2D, nx=n, ny=n, dx=d, dy=d, t_end=t_end, cfl=CFL, bc=0))
        fields.append(U32.ravel())
        data.append((U32.astype(np.float64), d, t_end))
    table, total, offs = npw.make_queue_instances(specs)
    arena = torch.tensor(np.concatenate(fields), device="cuda")
    st, stats = npw.npweno_queue_solve(arena, table, npw.Params(precision=npw.NPW_FP32_MIXED))
    a = arena.cpu().numpy().astype(np.float64)
    return [(U, d, t, a[o:o + U.size].reshape(U.shape)) for (U, d, t), o in zip(data, offs)]


# ------------------------------------------------------------------------------- CPU leg (oracle)
def _oracle_task(task):
    """One oracle run of a bounded sample: returns (result, stats, seconds)."""
    import oracle as O
    t0 = time.perf_counter()
    p = O.Params(**task["params"])
    if task.get("ny"):
        r, st = O.solve_2d(task["u0"], task["dx"], task["dy"], task["t_end"], CFL, task["kind"], task["bc"], p,
                           max_steps=task.get("max_steps", -1))
    else:
        r, st = O.solve(task["u0"], task["dx"], task["t_end"], CFL, task["kind"], task["bc"], p,
                        max_steps=task.get("max_steps", -1))
    return r, st, time.perf_counter() - t0


def run_oracle(tasks, cores):
    import multiprocessing as mp
    import oracle as O
    O.build()
    ctx = mp.get_context("spawn")
    t0 = time.perf_counter()
    with ctx.Pool(min(cores, len(tasks))) as pool:
        res = pool.map(_oracle_task, tasks, chunksize=1)
    return res, time.perf_counter() - t0


def cpu_sample(inst, cores: int):
    """The FP64 oracle on the headline's bounded timing sample: every SAMPLE_STRIDE-th instance
    (sorted by N), the first SAMPLE_STEPS RK3 steps each, over spawned processes."""
    import oracle as O
    order = sorted(range(len(inst)), key=lambda i: inst[i].n)
    pick = order[SAMPLE_STRIDE // 2::SAMPLE_STRIDE]
    tasks = [dict(u0=inst[i].u0[0].astype(np.float64), dx=inst[i].dx, t_end=T_END, kind=O.BURGERS, bc=O.PERIODIC,
                  params=dict(rbf=O.GA), max_steps=SAMPLE_STEPS) for i in pick]
    cells = sum(inst[i].n for i in pick) * SAMPLE_STEPS
    _, wall = run_oracle(tasks, cores)
    return cells / wall, wall, (f"{len(pick)} instances (every {SAMPLE_STRIDE}th by N, N={inst[pick[0]].n}.."
                                f"{inst[pick[-1]].n}), first {SAMPLE_STEPS} RK3 steps each, FP64 oracle, "
                                f"{min(cores, len(pick))} spawned processes")


def _errors(got, ref):
    """L1 (mean) and L_inf of the difference, absolute and relative to max |ref|."""
    got, ref = np.asarray(got, dtype=np.float64), np.asarray(ref, dtype=np.float64)
    e = np.abs(got - ref)
    scale = np.abs(ref).max()
    return {"l1": float(e.mean()), "linf": float(e.max()), "l1_rel": float(e.mean() / scale),
            "linf_rel": float(e.max() / scale)}


def _worst(errs):
    return {k: max(e[k] for e in errs) for k in errs[0]} if errs else None


def cpu_leg_headline(sample, cores):
    """Accuracy of the headline against the oracle: the eight smallest instances of the batch,
    solved to T = 1.5 by the oracle from the same float data."""
    import oracle as O
    ns, order, host0, result = sample["ns"], sample["order"], sample["host0"], sample["result"]
    offs = np.concatenate([[0], np.cumsum(ns)])
    pick = sorted(range(len(ns)), key=lambda k: ns[k])[:8]
    tasks = [dict(u0=host0[offs[k]:offs[k + 1]].astype(np.float64), dx=sample["inst"][order[k]].dx, t_end=T_END,
                  kind=O.BURGERS, bc=O.PERIODIC, params=dict(rbf=O.GA, eta_guard=MIXED_GUARD)) for k in pick]
    res, wall = run_oracle(tasks, cores)
    errs = [_errors(result[offs[k]:offs[k + 1]], r) for k, (r, st, sec) in zip(pick, res)]
    return {"vs_oracle": _worst(errs), "sample": f"the 8 smallest instances (N {ns[pick[0]]}..{ns[pick[-1]]}) to T=1.5, "
            "oracle from the same float data (worst over the sample)"}


def cpu_leg_advection(c1, cores):
    import oracle as O
    res, wall = run_oracle([dict(u0=c1["u0"], dx=c1["dx"], t_end=2.0, kind=O.ADVECTION, bc=O.PERIODIC, params={})], 1)
    r, st, sec = res[0]
    return {"cpu_baseline": {"value": 200 * st["steps"] / sec, "unit": "cell-updates/s", "cores": 1, "kind": "oracle",
                             "sample": "the whole N=200 solve (400 steps), one process"},
            "vs_oracle": {**_errors(c1["result"], r), "steps_equal": st["steps"] == c1["steps"]}}


def cpu_leg_euler1d(c3, cores):
    """Accuracy and timing of the oracle on the eight smallest instances of the 1D Euler batch,
    to the same end times, from the same float data."""
    import oracle as O
    inst, host0, offs, result = c3["inst"], c3["host0"], c3["offs"], c3["result"]
    pick = sorted(range(len(inst)), key=lambda k: inst[k].n)[:8]
    params = dict(characteristic=c3["characteristic"], eta_guard=MIXED_GUARD, eta_max=c3["eta_max"])
    tasks = []
    for k in pick:
        it = inst[k]
        tasks.append(dict(u0=host0[offs[k]:offs[k] + 3 * it.n].astype(np.float64).reshape(3, it.n), dx=it.dx,
                          t_end=c3["t_frac"] * it.t_end, kind=O.EULER1D, bc=O.TRANSMISSIVE, params=params))
    res, wall = run_oracle(tasks, cores)
    errs = [_errors(result[offs[k]:offs[k] + 3 * inst[k].n].reshape(3, inst[k].n), r) for k, (r, st, sec)
            in zip(pick, res)]
    cells = sum(inst[k].n * st["steps"] for k, (r, st, sec) in zip(pick, res))
    return {"cpu_baseline": {"value": cells / wall, "unit": "cell-updates/s", "cores": min(cores, len(pick)),
                             "kind": "oracle",
                             "sample": f"the 8 smallest instances (N {inst[pick[0]].n}..{inst[pick[-1]].n}), whole "
                                       f"solves to {c3['t_frac']} x end time, one process each"},
            "vs_oracle": _worst(errs)}


def cpu_leg_euler2d(runs, cores):
    import oracle as O
    tasks = [dict(u0=U, dx=d, dy=d, ny=U.shape[1], t_end=t, kind=O.EULER2D, bc=O.PERIODIC,
                  params=dict(eta_guard=MIXED_GUARD)) for U, d, t, g in runs]
    res, wall = run_oracle(tasks, cores)
    errs = [_errors(g, r) for (U, d, t, g), (r, st, sec) in zip(runs, res)]
    cells = sum(U.shape[1] * U.shape[2] * st["steps"] for (U, d, t, g), (r, st, sec) in zip(runs, res))
    n = runs[0][0].shape[1]
    return {"cpu_baseline": {"value": cells / wall, "unit": "cell-updates/s", "cores": len(tasks), "kind": "oracle",
                             "sample": f"two {n}^2 squares (vortex, four-quadrant), ~5 RK3 steps, one process each"},
            "vs_oracle": _worst(errs)}


# ------------------------------------------------------------------------------- serving
_SERVING_CACHE = {}


def serving_requests(count: int, rate: float, seed: int = 5):
    """Poisson arrivals of mixed requests: periodic Burgers (the batch family, T scaled by
    U(0.1, 1)), transmissive 1D Euler Riemann / Shu-Osher data (n up to 8192) and periodic 2D
    Euler squares (isentropic vortex or four-quadrant data, 128^2 to 1024^2).  The payloads are
    drawn once per (count, seed); the rate only scales the arrival times."""
    key = (count, seed)
    if key not in _SERVING_CACHE:
        g = np.random.Generator(np.random.PCG64(I.SEED_BASE + 50 + seed))
        burg = I.burgers_batch(count=count, seed_index=60 + seed)
        eul = I.euler_batch(count=count, nmin=256, nmax=8192, seed_index=70 + seed)
        gaps, items = [], []
        for k in range(count):
            gaps.append(g.exponential(1.0))
            u = g.uniform()
            if u < 0.4:
                it = burg[k]
                items.append(dict(kind=1, bc=0, m=1, n=it.n, ny=0, dx=it.dx, t_end=1.5 * g.uniform(0.1, 1.0),
                                  u0=it.u0.ravel()))
            elif u < 0.8:
                it = eul[k]
                items.append(dict(kind=2, bc=1, m=3, n=it.n, ny=0, dx=it.dx, t_end=it.t_end * g.uniform(0.1, 1.0),
                                  u0=it.u0.ravel()))
            else:
                n2 = int(g.choice([128, 256, 512, 1024], p=[0.4, 0.3, 0.2, 0.1]))
                U, d = I.euler2d_batch(n2, 2, seed_index=1000 + 100 * seed + k)[k % 2]
                t2 = (0.1 if k % 2 == 0 else 0.02) * g.uniform(0.1, 1.0)  # ~10-80 steps
                items.append(dict(kind=3, bc=0, m=4, n=n2, ny=n2, dx=d, t_end=t2, u0=U))
        _SERVING_CACHE[key] = (np.array(gaps), items)
    gaps, items = _SERVING_CACHE[key]
    arrivals = np.cumsum(gaps) / rate
    return [dict(arrival=float(t), **it) for t, it in zip(arrivals, items)]


def run_serving(npw, reqs, max_steps: int = 32, precision=None):
    """Continuous batching: requests are submitted at their arrival times and stepped together
    (every request in the lane of the server's precision: mixed by default)."""
    p = npw.Params(rbf=npw.NPW_RBF_GA, precision=npw.NPW_FP32_MIXED if precision is None else precision,
                   batch_mode=1, eta_max=SWEEP_ETA_MAX)
    srv = npw.Server(heap_cells=64 * 1024 * 1024, max_slots=512, params=p)
    t0 = time.perf_counter()
    k, done = 0, {}
    while len(done) < len(reqs):
        now = time.perf_counter() - t0
        while k < len(reqs) and reqs[k]["arrival"] <= now:
            r = reqs[k]
            srv.submit(r["u0"], r["kind"], r["bc"], r["dx"], r["t_end"], 0.5, tag=k,
                       dy=r["dx"] if r["ny"] else 0.0)
            k += 1
        act, q = srv.step(max_steps)
        for res in srv.poll():
            done[res["tag"]] = res
        if act == 0 and q == 0 and k < len(reqs):
            time.sleep(max(0.0, reqs[k]["arrival"] - (time.perf_counter() - t0)))
    srv.close()
    lat = np.array([done[i]["done_s"] - reqs[i]["arrival"] for i in range(len(reqs))])
    cells = sum(reqs[i]["n"] * max(reqs[i]["ny"], 1) * done[i]["steps"] for i in range(len(reqs)))
    span = max(done[i]["done_s"] for i in done) - reqs[0]["arrival"]
    ok = all(done[i]["status"] == 0 for i in done)
    return lat, cells / span, ok


def fifo_service_times(npw, reqs):
    """The comparator's service time of every request: the plain FP64 per-instance solve, one
    request at a time (host copy in, solve, host copy out)."""
    import torch
    p = npw.Params(rbf=npw.NPW_RBF_GA, precision=npw.NPW_FP64, eta_max=SWEEP_ETA_MAX)
    svc, cells = [], []
    for r in reqs:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        u = torch.tensor(r["u0"], dtype=torch.float64, device="cuda")
        if r["ny"]:
            st = npw.npweno_solve_2d(u, r["dx"], r["dx"], r["t_end"], 0.5, r["kind"], r["bc"], p)
        else:
            st = npw.npweno_solve(u.view(r["m"], r["n"]), r["dx"], r["t_end"], 0.5, r["kind"], r["bc"], p)
        u.cpu()
        svc.append(time.perf_counter() - t0)
        cells.append(r["n"] * max(r["ny"], 1) * st["steps"])
    return np.array(svc), np.array(cells)


def fifo_latencies(svc, arrivals):
    """Latencies of a first-in first-out server that runs one request at a time: request i
    starts at max(its arrival, the end of request i-1) and takes its service time."""
    lat, end = [], 0.0
    for s, a in zip(svc, arrivals):
        end = max(end, a) + s
        lat.append(end - a)
    return np.array(lat), end


def serving_block(npw, count: int, rates):
    """The request stream at each arrival rate (the same requests; only the arrival times
    scale): the continuous-batching server measured live, and the FP64 first-in first-out
    comparator from its measured per-request service times (it runs one request at a time, so
    its latencies follow from the arrival times and the service times)."""
    q = lambda a, x: float(np.percentile(a, x) * 1e3)
    base = serving_requests(count, rates[0])
    svc, fcells = fifo_service_times(npw, base)
    out = {"requests": count,
           "mix": "0.4 periodic Burgers (N 64..8192, T 0.15..1.5), 0.4 transmissive 1D Euler (N 256..8192), "
                  "0.2 periodic 2D Euler squares (128^2..1024^2, vortex or four-quadrant)",
           "server_mode": "continuous batching, NPW_FP32_MIXED, work-queue kernels specialised per instance shape "
                          "(one stream each; fused RK3 steps for the 1D requests), 32-step rounds; every arm "
                          "drops faces with |eta| > 100",
           "fp64_fifo_mode": "one request at a time, npweno_solve / npweno_solve_2d NPW_FP64; latencies from "
                             "measured service times",
           "fp64_server_mode": "the same continuous-batching server with every request in its FP64 lane: "
                               "batching alone, against the FP64 FIFO",
           "rates": []}
    for rate in rates:
        reqs = serving_requests(count, rate)
        lat, thr, ok = run_serving(npw, reqs)
        lat64, thr64, ok64 = run_serving(npw, reqs, precision=npw.NPW_FP64)
        flat, fend = fifo_latencies(svc, [r["arrival"] for r in reqs])
        out["rates"].append({
            "rate_per_s": rate,
            "server": {"p50_ms": q(lat, 50), "p99_ms": q(lat, 99), "cell_updates_per_s": thr, "all_ok": ok},
            "fp64_server": {"p50_ms": q(lat64, 50), "p99_ms": q(lat64, 99), "cell_updates_per_s": thr64,
                            "all_ok": ok64},
            "fp64_fifo": {"p50_ms": q(flat, 50), "p99_ms": q(flat, 99),
                          "cell_updates_per_s": float(fcells.sum() / (fend - reqs[0]["arrival"]))},
        })
    return out


# ------------------------------------------------------------------------------- serving sweep
FP64_TOL_CLASS = 1e-10   # a request asking for this tolerance takes the server's FP64 lane
FP32_TOL_CLASS = 1e-4    # the float lane's class (npweno.MIXED_TOLERANCE)
SWEEP_FP64_SHARE = 0.1   # share of the sweep's requests in the FP64 class
# the sweep's servers and comparator drop faces with |eta| > 100: with the printed eta a
# four-quadrant square in FP64 goes non-finite from one face whose denominator vanishes
SWEEP_ETA_MAX = 100.0


def sweep_payloads(count: int, seed: int = 7):
    """Payloads of the C5-type stream: each request is, with equal probability, a periodic Burgers
    instance of the batch family (N log-uniform 64..8192, T = 1.5 U(0.1, 1)), a transmissive 1D
    Euler instance (Riemann or Shu-Osher-type data, N log-uniform 256..65536, T = its end time x
    U(0.1, 1)) or a periodic 2D Euler square (vortex or four-quadrant, 128^2..1024^2, T x
    U(0.1, 1) of ~10-80 steps); a tenth ask for FP64 (tolerance 1e-10), the rest for the float
    class (1e-4)."""
    g = np.random.Generator(np.random.PCG64(I.SEED_BASE + 900 + seed))
    burg = I.burgers_batch(count=count, seed_index=910 + seed)
    eul = I.euler_batch(count=count, nmin=256, nmax=65536, seed_index=920 + seed)
    sq = {}
    items = []
    for k in range(count):
        fam = int(g.integers(3))
        tol = FP64_TOL_CLASS if g.uniform() < SWEEP_FP64_SHARE else FP32_TOL_CLASS
        if fam == 0:
            it = burg[k]
            items.append(dict(family="burgers", kind=1, bc=0, m=1, n=it.n, ny=0, dx=it.dx,
                              t_end=1.5 * g.uniform(0.1, 1.0), u0=it.u0.ravel(), tol=tol))
        elif fam == 1:
            it = eul[k]
            items.append(dict(family="euler1d", kind=2, bc=1, m=3, n=it.n, ny=0, dx=it.dx,
                              t_end=it.t_end * g.uniform(0.1, 1.0), u0=it.u0.ravel(), tol=tol))
        else:
            n2 = int(g.choice([128, 256, 512, 1024], p=[0.4, 0.3, 0.2, 0.1]))
            which = int(g.integers(2))
            if n2 not in sq:  # one vortex and one four-quadrant square per size, shared by the requests
                sq[n2] = I.euler2d_batch(n2, 2, seed_index=930 + seed)
            U, d = sq[n2][which]
            t2 = (0.1 if which == 0 else 0.02) * g.uniform(0.1, 1.0)
            items.append(dict(family="euler2d", kind=3, bc=0, m=4, n=n2, ny=n2, dx=d, t_end=t2, u0=U, tol=tol))
    gaps = g.exponential(1.0, size=count)
    return gaps, items


def run_serving_stream(npw, reqs, heap_cells: int, max_slots: int, max_steps: int = 32):
    """The live server on a stream of requests (arrival, payload): each is submitted at its
    arrival time (held on the host while the server's queue is full), the server is stepped in
    rounds of max_steps steps, results are polled; latency = result on the host - arrival."""
    p = npw.Params(rbf=npw.NPW_RBF_GA, precision=npw.NPW_FP32_MIXED, batch_mode=1, eta_max=SWEEP_ETA_MAX)
    srv = npw.Server(heap_cells=heap_cells, max_slots=max_slots, params=p)
    t0 = time.perf_counter()
    k, done, backlog = 0, {}, []
    while len(done) < len(reqs):
        now = time.perf_counter() - t0
        while k < len(reqs) and reqs[k]["arrival"] <= now:
            backlog.append(k)
            k += 1
        while backlog:
            r = reqs[backlog[0]]
            try:
                srv.submit(r["u0"], r["kind"], r["bc"], r["dx"], r["t_end"], 0.5, tag=backlog[0],
                           dy=r["dx"] if r["ny"] else 0.0, tolerance=r["tol"])
            except npw.NpwError as e:
                if e.status != npw.NPW_EBUSY:
                    raise
                break
            backlog.pop(0)
        act, q = srv.step(max_steps)
        for res in srv.poll():
            done[res["tag"]] = res
        if act == 0 and q == 0 and not backlog and k < len(reqs):
            time.sleep(max(0.0, reqs[k]["arrival"] - (time.perf_counter() - t0)))
    srv.close()
    return done


def fifo_per_step_model(npw, items, per_family: int = 12, probe_steps: int = 40):
    """The FP64 first-in first-out comparator's service time: for a sample of each family's
    requests (spread over their sizes), the FP64 solve (npweno_solve / npweno_solve_2d, host
    copy in and out, one at a time) is timed for probe_steps steps (max_steps) and for 2 x
    probe_steps; the difference gives the time per step, the rest the fixed cost.  Per family,
    time per step = a + b cells (least squares) and fixed cost = the sample mean."""
    import torch
    model = {}
    for fam in ("burgers", "euler1d", "euler2d"):
        idx = [i for i, r in enumerate(items) if r["family"] == fam]
        idx = sorted(idx, key=lambda i: items[i]["n"] * max(items[i]["ny"], 1))
        pick = [idx[int(j)] for j in np.linspace(0, len(idx) - 1, min(per_family, len(idx)))]
        cells, per_step, fixed = [], [], []
        for i in pick:
            r = items[i]
            ts = []
            for steps in (probe_steps, 2 * probe_steps):
                p = npw.Params(rbf=npw.NPW_RBF_GA, precision=npw.NPW_FP64, max_steps=steps, eta_max=SWEEP_ETA_MAX)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                u = torch.tensor(r["u0"], dtype=torch.float64, device="cuda")
                try:
                    if r["ny"]:
                        npw.npweno_solve_2d(u, r["dx"], r["dx"], 1e9, 0.5, r["kind"], r["bc"], p)
                    else:
                        npw.npweno_solve(u.view(r["m"], r["n"]), r["dx"], 1e9, 0.5, r["kind"], r["bc"], p)
                except npw.NpwError as e:
                    if e.status != npw.NPW_ETIMEOUT:
                        raise
                u.cpu()
                ts.append(time.perf_counter() - t0)
            c = r["n"] * max(r["ny"], 1) * r["m"]
            cells.append(c)
            per_step.append(max((ts[1] - ts[0]) / probe_steps, 0.0))
            fixed.append(max(ts[0] - probe_steps * per_step[-1], 0.0))
        A = np.vstack([np.ones(len(cells)), np.array(cells, dtype=float)]).T
        coef, *_ = np.linalg.lstsq(A, np.array(per_step), rcond=None)
        model[fam] = {"a_s": float(coef[0]), "b_s_per_cell": float(coef[1]), "fixed_s": float(np.mean(fixed)),
                      "sampled": len(pick)}
    return model


def serving_sweep(npw, rates, count: int = 2000, horizon_s: float = 60.0):
    """The C5-type serving sweep: per arrival rate, Poisson arrivals of the same payload sequence
    until `count` requests or `horizon_s` seconds of arrivals, served live by the two-lane
    server; the FP64 FIFO comparator (one request at a time) from its per-step model and the
    step counts the server reported."""
    q = lambda a, x: float(np.percentile(a, x) * 1e3) if len(a) else None
    gaps, items = sweep_payloads(count)
    model = fifo_per_step_model(npw, items)
    out = {"mode": "serving sweep (C5-type)", "requests_max": count, "horizon_s": horizon_s,
           "mix": "1/3 periodic Burgers (N 64..8192), 1/3 transmissive 1D Euler (N 256..65536), 1/3 periodic 2D "
                  "Euler squares (128^2..1024^2); T x U(0.1, 1); 1/10 FP64 class (tol 1e-10), 9/10 float class "
                  "(1e-4); |eta| <= 100 in both lanes and the comparator",
           "server": "npw_server: two lanes (NPW_FP32_MIXED, NPW_FP64), each with its own stream and rounds; per "
                     "lane the requests grouped by instance shape, each group on a stream with the queue kernel "
                     "specialised for it (fused RK3 steps for the float lane's 1D requests); 32-step rounds",
           "fifo_comparator": "FP64, one request at a time, per-stage kernels, no graphs; service time = fixed + "
                              "steps x (a + b cells) per family, measured on a size-spread sample",
           "fifo_model": model, "rates": []}
    for rate in rates:
        arr = np.cumsum(gaps) / rate
        n_req = int(min(count, np.searchsorted(arr, horizon_s)))
        reqs = [dict(arrival=float(arr[k]), **items[k]) for k in range(n_req)]
        t_start = time.perf_counter()
        done = run_serving_stream(npw, reqs, heap_cells=96 * 1024 * 1024, max_slots=1024)
        wall = time.perf_counter() - t_start
        lat = np.array([done[i]["done_s"] - reqs[i]["arrival"] for i in range(n_req)])
        prec = np.array([done[i]["precision"] for i in range(n_req)])
        steps = np.array([done[i]["steps"] for i in range(n_req)])
        cu = np.array([reqs[i]["n"] * max(reqs[i]["ny"], 1) * steps[i] for i in range(n_req)], dtype=float)
        span = max(done[i]["done_s"] for i in done) - reqs[0]["arrival"]
        # FIFO: the same requests in arrival order, FP64, one at a time
        svc = []
        for i in range(n_req):
            mdl = model[reqs[i]["family"]]
            c = reqs[i]["n"] * max(reqs[i]["ny"], 1) * reqs[i]["m"]
            svc.append(mdl["fixed_s"] + steps[i] * max(mdl["a_s"] + mdl["b_s_per_cell"] * c, 0.0))
        flat, fend = fifo_latencies(np.array(svc), [r["arrival"] for r in reqs])
        fam_lat = {f: q(lat[[r["family"] == f for r in reqs]], 99) for f in ("burgers", "euler1d", "euler2d")}
        out["rates"].append({
            "rate_per_s": rate, "requests": n_req, "wall_s": wall,
            "server": {"p50_ms": q(lat, 50), "p99_ms": q(lat, 99), "mean_ms": float(lat.mean() * 1e3),
                       "p99_ms_fp32_lane": q(lat[prec == 1], 99), "p99_ms_fp64_lane": q(lat[prec == 0], 99),
                       "p99_ms_by_family": fam_lat, "cell_updates_per_s": float(cu.sum() / span),
                       "all_ok": all(done[i]["status"] == 0 for i in done),
                       "status_counts": {str(k): int(v) for k, v in zip(*np.unique(
                           [done[i]["status"] for i in done], return_counts=True))}},
            "fp64_fifo": {"p50_ms": q(flat, 50), "p99_ms": q(flat, 99),
                          "cell_updates_per_s": float(cu.sum() / (fend - reqs[0]["arrival"]))},
        })
        print(json.dumps(out["rates"][-1]), file=sys.stderr, flush=True)
    return out


# ------------------------------------------------------------------------------- ranks
def rank_seed(base: int, rank: int) -> int:
    """Seed index of a rank's batch: every rank solves its own seeded batch of the same family
    and size (weak scaling; the instances are independent, so no data crosses ranks)."""
    return base + 1000 * rank


def job_totals(total_ms: float, units: float, world: int, device):
    """Whole-job figures: the slowest rank's time and the units all ranks processed (the only
    two collectives of the benchmark; none on the data path)."""
    if world <= 1:
        return total_ms, units
    import torch
    t = torch.tensor([float(total_ms)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    c = torch.tensor([float(units)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(c, op=torch.distributed.ReduceOp.SUM)
    return t.item(), c.item()


def reference_arm(args, cores):
    """The FP64 oracle on the host cores, a bounded sample of the headline workload per step."""
    inst = I.burgers_batch(count=args.instances, seed_index=1)
    for _ in range(args.warmup):
        cpu_sample(inst, cores)
    vals, walls = [], []
    desc = ""
    for _ in range(args.steps):
        v, wall, desc = cpu_sample(inst, cores)
        vals.append(v)
        walls.append(wall)
    value = float(np.mean(vals))
    print(json.dumps({
        "metric": "cell-updates/s", "value": value, "unit": "cell-updates/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * float(np.mean(walls)),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded)", "impl": "reference",
        "config": {"workload": WORKLOAD, "instances": args.instances, "sample": desc},
        "cpu_baseline": {"value": value, "unit": "cell-updates/s", "cores": cores, "kind": "oracle", "sample": desc},
        "e2e": {"value": value, "unit": "cell-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--instances", type=int, default=4096)
    ap.add_argument("--t-end", type=float, default=T_END, help="final time (shorter only for profiling runs)")
    ap.add_argument("--blocks", default="c1,c3,c3char,c4,serving",
                    help="the other workloads' blocks (comma list of c1, c3, c3char, c4, serving; empty: none)")
    ap.add_argument("--euler-t-frac", type=float, default=1.0, help="1D Euler block: fraction of each end time")
    ap.add_argument("--euler-char-t-frac", type=float, default=0.1,
                    help="1D Euler characteristic block: fraction of each end time")
    ap.add_argument("--sizes2d", default="256,512,1024,2048", help="2D Euler block: square sizes")
    ap.add_argument("--steps2d", type=int, default=100, help="2D Euler block: RK3 steps per solve")
    ap.add_argument("--euler-tile", type=int, default=0, help="1D Euler blocks: cells per tile (0: the library's)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--eta-eval", type=int, default=0, choices=[0, 1],
                    help="mixed path: 0 = eta from float pairs, double-float quotient (the library default); "
                         "1 = eta in FP64")
    ap.add_argument("--serve-requests", type=int, default=60, help="requests of the serving run")
    ap.add_argument("--serve-rates", default="10,100,1000", help="Poisson arrival rates of the serving runs (1/s)")
    ap.add_argument("--variant-steps", type=int, default=1,
                    help="timed solves of each variant reported beside the headline (0: skip)")
    ap.add_argument("--out-dir", default=os.path.join(tempfile.gettempdir(), "npweno_bench"),
                    help="where the clock samples are written")
    ap.add_argument("--serving-sweep", action="store_true",
                    help="run only the C5-type serving sweep (rates 10..1000 /s, 2000 requests or 60 s each)")
    ap.add_argument("--sweep-rates", default="10,30,100,300,1000")
    ap.add_argument("--sweep-requests", type=int, default=2000)
    ap.add_argument("--sweep-horizon", type=float, default=60.0)
    args = ap.parse_args()
    args.sizes2d = [int(x) for x in args.sizes2d.split(",") if x]
    blocks = {b.strip() for b in args.blocks.split(",") if b.strip()}
    os.makedirs(args.out_dir, exist_ok=True)
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    cores = os.cpu_count() or 1

    if args.impl == "reference":
        if rank == 0:
            reference_arm(args, cores)
        return

    import torch
    import paper_1602_00182_gb300.npweno as npw
    from paper_1602_00182_gb300 import build as b
    if local_rank == 0 or not os.path.exists(npw.LIB_PATH):
        b.build()
    if world > 1:
        torch.distributed.init_process_group("nccl")
        torch.distributed.barrier()
    torch.cuda.set_device(local_rank)
    if args.serving_sweep:
        if rank == 0:
            print(json.dumps(serving_sweep(npw, [float(x) for x in args.sweep_rates.split(",")],
                                           args.sweep_requests, args.sweep_horizon)))
        return
    out, sample = headline_burgers(args, rank, world, local_rank)
    single = rank == 0 and world == 1
    cfg, leg = {}, {}
    if single and "c1" in blocks:
        cfg["advection_fp64_n200"], leg["c1"] = block_advection(args)
    if single and "c3" in blocks:
        cfg["euler1d_component"], leg["c3"] = block_euler1d(args, 0)
    if single and "c3char" in blocks:
        cfg["euler1d_characteristic"], leg["c3char"] = block_euler1d(args, 1)
    if single and "c4" in blocks:
        cfg["euler2d"] = block_euler2d(args)
        leg["c4"] = accuracy_run_2d(npw)
    if cfg:
        out["configs"] = cfg
    if single and "serving" in blocks and args.serve_requests > 0:
        out["serving"] = serving_block(npw, args.serve_requests, [float(x) for x in args.serve_rates.split(",")])
    if rank == 0:
        if not args.no_cpu_baseline:
            # the CPU leg: the FP64 oracle on bounded samples, timed on the host cores; its results
            # also give each block's difference from the oracle
            v, wall, desc = cpu_sample(sample["inst"], cores)
            out["cpu_baseline"] = {"value": v, "unit": "cell-updates/s", "cores": cores, "kind": "oracle",
                                   "sample": desc}
            out["accuracy"] = cpu_leg_headline(sample, cores)
            if "c1" in leg:
                cfg["advection_fp64_n200"].update(cpu_leg_advection(leg["c1"], cores))
            if "c3" in leg:
                cfg["euler1d_component"].update(cpu_leg_euler1d(leg["c3"], cores))
            if "c3char" in leg:
                cfg["euler1d_characteristic"].update(cpu_leg_euler1d(leg["c3char"], cores))
            if "c4" in leg:
                cfg["euler2d"].update(cpu_leg_euler2d(leg["c4"], cores))
        print(json.dumps(out))
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
