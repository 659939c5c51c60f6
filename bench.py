#!/usr/bin/env python3
"""Benchmark: batched 1D Burgers with the non-polynomial RBF-WENO5 method on one GB300 per rank.

Workload (one "step" = one whole solve of the batch): 4096 periodic Burgers instances on
[0, 2 pi], N log-uniform in [64, 8192] (seeded), u0 = 1 + four Fourier modes + up to two
jumps, Gaussian perturbation with the monotone switch, Lax-Friedrichs flux, TVD-RK3 at
CFL 0.5, run past shock formation to T = 1.5.  Float state, candidates, weights and flux;
the shape parameter eta in double; switch and ENO decisions certified equal to their double
evaluation.  Each instance keeps its own dt; every instance fits in shared memory, so the
batch runs in the resident whole-solve kernel (four size classes on side streams).

`--workload euler1d` (512 transmissive Euler instances, per-stage kernels) and
`--workload euler2d` (2D Euler on 2048^2 squares) print their own lines.

Prints one JSON line (rank 0).  `--impl reference` times the FP64 CPU oracle instead, on
a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import ctypes
import json
import os
import statistics
import subprocess
import sys
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


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ------------------------------------------------------------------------------- CPU oracle leg
def _oracle_job(args):
    u0, dx, steps = args
    import oracle as O
    t0 = time.perf_counter()
    O.solve(u0, dx, T_END, CFL, O.BURGERS, O.PERIODIC, O.Params(rbf=O.GA), max_steps=steps)
    return time.perf_counter() - t0


def cpu_sample(inst, cores: int):
    """The FP64 oracle on a bounded sample: every SAMPLE_STRIDE-th instance (sorted by N), the
    first SAMPLE_STEPS RK3 steps each, spread over `cores` spawned processes."""
    import multiprocessing as mp
    import oracle as O
    O.build()
    order = sorted(range(len(inst)), key=lambda i: inst[i].n)
    pick = order[SAMPLE_STRIDE // 2::SAMPLE_STRIDE]
    jobs = [(inst[i].u0[0].astype(np.float64), inst[i].dx, SAMPLE_STEPS) for i in pick]
    cells = sum(inst[i].n for i in pick) * SAMPLE_STEPS
    ctx = mp.get_context("spawn")
    t0 = time.perf_counter()
    with ctx.Pool(cores) as pool:
        pool.map(_oracle_job, jobs, chunksize=1)
    wall = time.perf_counter() - t0
    return cells / wall, wall, (f"{len(pick)} instances (every {SAMPLE_STRIDE}th by N, N={inst[pick[0]].n}.."
                                f"{inst[pick[-1]].n}), first {SAMPLE_STEPS} RK3 steps each, FP64 oracle, "
                                f"{cores} spawned processes")


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


# ------------------------------------------------------------------------------- GPU leg
def run_gpu(args, rank, world, local_rank):
    import torch
    import paper_1602_00182_gb300.npweno as npw
    from paper_1602_00182_gb300 import build as b

    if local_rank == 0 or not os.path.exists(npw.LIB_PATH):
        b.build()
    if world > 1:
        torch.distributed.barrier()
    lib = npw.load()
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)

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
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # > L2
    stream = torch.cuda.current_stream()

    def one_solve():
        st, stats = npw.npweno_batch_solve(arena, table, 1, npw.NPW_FLUX_BURGERS, params, workspace=ws)
        if st != 0:
            raise RuntimeError(f"batch solve failed with status {st}")
        return stats

    # warm-up (also yields the per-instance step counts: the work of one step)
    for _ in range(args.warmup):
        arena.copy_(pristine)
        stats = one_solve()
    cell_updates = sum(n * s["steps"] for n, s in zip(ns, stats))

    pr = npw_profile()
    lib.npw_profile_reset()
    lib.npw_profile_enable(1)
    times = []
    clocks = Clocks(os.path.join(args.out_dir, f"clocks_rank{rank}.csv"))
    with clocks:
        for _ in range(args.steps):
            arena.copy_(pristine)
            flush.fill_(1.0)  # evict the working set from L2 between timed steps
            if world > 1:
                torch.distributed.barrier()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            one_solve()
            e1.record(stream)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
    lib.npw_profile_read(ctypes.byref(pr))
    lib.npw_profile_enable(0)
    tmax, cu_all = job_totals(sum(times), cell_updates * args.steps, world, dev)
    value = cu_all / (tmax / 1e3)

    # Roofline of the dominant kernel.  Every instance of this workload fits in shared memory,
    # so the batch runs in the resident whole-solve kernel; its largest size class (n > 4096,
    # ~3/4 of the work) is the dominant launch.  It is bound by the FP64 pipe (the shape
    # parameter), not by HBM: achieved = FP64-pipe instructions of the eta evaluations
    # (FP64_OPS_PER_ETA per face and stage, counted over all n+1 faces: an upper bound, since
    # faces where the switch fires skip it) / the class-A launch time.
    big = [k for k, n in enumerate(ns) if n > 4096]
    faces_a = sum((ns[k] + 1) * 3 * stats[k]["steps"] for k in big) * args.steps
    res_s = pr.resident_ms[0] / 1e3
    achieved = FP64_OPS_PER_ETA * faces_a / res_s / 1e9 if res_s > 0 else None
    peak = FP64_PIPE_PEAK / 1e9
    traffic = _ncu_traffic()

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
            flush.fill_(1.0)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            st, vstats = npw.npweno_batch_solve(arena, table, 1, npw.NPW_FLUX_BURGERS, pv, workspace=ws)
            e1.record(stream)
            torch.cuda.synchronize()
            vt.append(e0.elapsed_time(e1))
        vcu = sum(n * s["steps"] for n, s in zip(ns, vstats))
        variants[label] = {"value": vcu * len(vt) / (sum(vt) / 1e3), "unit": "cell-updates/s",
                           "ms_per_step": sum(vt) / len(vt)}

    if args.variant_steps > 0 and args.eta_eval == 0 and world == 1:
        time_variant(npw.Params(rbf=npw.NPW_RBF_GA, precision=npw.NPW_FP32_MIXED, eta_eval=1),
                     "eta_eval=1 (exact double-float eta, no FP64 instruction)")
        time_variant(npw.Params(k=2, rbf=npw.NPW_RBF_GA, precision=npw.NPW_FP32_MIXED, eta_max=1.0),
                     "k=2 RBF-WENO3 Gaussian + switch (Table k2; resident kernels, eta in FP64), |eta| <= 1 "
                     "(the printed k = 2 eta is singular where u crosses zero)")

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
            "precision": ("NPW_FP32_MIXED: f32 state, candidates, beta, weights, flux, update; eta in FP64 "
                          f"(eta_eval={args.eta_eval}); switch decisions equal to FP64 evaluation"),
            "l2": "flushed (256 MB write) before every timed step; working set 3 x 4 B x cells",
            "parallelism": f"independent instance batches, one per rank (x{world})",
        },
        "roofline": {
            "bound": "alu",
            "achieved": achieved,
            "peak": peak,
            "unit": "G FP64-pipe instr/s",
            "frac": (achieved / peak) if achieved else None,
            "traffic": traffic,
            "kernel": "solve1d_resident_kernel<BURGERS>, size class n > 4096 (512 threads, 2 CTAs/SM)",
            "resident_launches": [int(x) for x in pr.resident_launches],
            "resident_ms": [float(x) for x in pr.resident_ms],
            "peak_source": ("derived: 2 FP64-pipe instr/clk/SM x 152 SMs x 2.07 GHz (nominal 1.25 TFLOP/s FP64); "
                            "probe of DFMA chains: 1.19 TFLOP/s"),
            "hbm_bytes_per_cell_update": "8 per solve (state read once, written once)",
            "kernel_source_sha256": kernel_source_hash(),
        },
        "e2e": {"value": e2e_value, "unit": "cell-updates/s", "h2d_bytes_per_step": int(host0.nbytes),
                "d2h_bytes_per_step": int(host0.nbytes)},
        "gpu_launches": int(pr.kernel_launches),
        "variants": variants,
        "clocks": clocks.summary(local_rank),
    }
    return out, inst


class npw_profile(ctypes.Structure):
    _fields_ = [("kernel_launches", ctypes.c_int64), ("stage_launches", ctypes.c_int64), ("stage_ms", ctypes.c_double),
                ("timed_launches", ctypes.c_int64), ("resident_launches", ctypes.c_int64 * 4),
                ("resident_ms", ctypes.c_double * 4)]


# FP64-pipe instructions of one shape-parameter evaluation in the mixed path (eta_fp64 in
# csrc/npw_fast.cuh): 2 adds (the numerator pair and the denominator pair, which carries
# eps_M, to double), 1 multiply and 2 multiply-adds (the Newton-corrected quotient); the
# format changes between float and double (the pairs, the seed, the result) are integer work.
FP64_OPS_PER_ETA = 5
# FP64 pipe peak: 1.25 TFLOP/s nominal FP64 = 0.625e12 FMA/s over 152 SMs at 2.07 GHz, i.e.
# 2 FP64-pipe instructions per clock per SM (a probe of independent DFMA chains measured 1.19 TFLOP/s)
FP64_PIPE_PEAK = 2.0 * 152 * 2.07e9


def kernel_source_hash() -> str:
    """sha256 over the device sources of the mixed-precision kernels (ncu figures are valid only
    for the sources they were taken from)."""
    import hashlib
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1602_00182_gb300", "csrc")
    for f in ("npw_internal.h", "npw_device.cuh", "npw_fast.cuh", "npw_kernels.cuh", "npw_fp32.cu"):
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _ncu_traffic():
    """DRAM bytes per launch of the dominant launch from the committed ncu summary, when it was
    taken from the current kernel sources (null otherwise)."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(p) as fh:
            d = json.load(fh)
        if d.get("kernel_source_sha256") != kernel_source_hash():
            return None
        return d.get("solve1d_resident_burgers_classA_dram_bytes_per_launch")
    except Exception:
        return None


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


def run_serving(npw, reqs, max_steps: int = 32):
    """Continuous batching: requests are submitted at their arrival times and stepped together."""
    import torch
    p = npw.Params(rbf=npw.NPW_RBF_GA, precision=npw.NPW_FP32_MIXED, batch_mode=1)
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
    p = npw.Params(rbf=npw.NPW_RBF_GA, precision=npw.NPW_FP64)
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
           "server_mode": "continuous batching, NPW_FP32_MIXED, per-stage kernels, 32-step rounds",
           "fp64_fifo_mode": "one request at a time, npweno_solve / npweno_solve_2d NPW_FP64; latencies from "
                             "measured service times",
           "rates": []}
    for rate in rates:
        reqs = serving_requests(count, rate)
        lat, thr, ok = run_serving(npw, reqs)
        flat, fend = fifo_latencies(svc, [r["arrival"] for r in reqs])
        out["rates"].append({
            "rate_per_s": rate,
            "server": {"p50_ms": q(lat, 50), "p99_ms": q(lat, 99), "cell_updates_per_s": thr, "all_ok": ok},
            "fp64_fifo": {"p50_ms": q(flat, 50), "p99_ms": q(flat, 99),
                          "cell_updates_per_s": float(fcells.sum() / (fend - reqs[0]["arrival"]))},
        })
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


# ------------------------------------------------------------------------------- other workloads
def _timed(fn, steps, flush, world):
    import torch
    times = []
    for _ in range(steps):
        flush.fill_(1.0)
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    return times


def run_euler1d(args, rank, world, local_rank):
    """Batched 1D Euler (512 instances, N log-uniform in [256, 65536], transmissive, Riemann and
    Shu-Osher-type data) through the per-stage kernels (batch_mode 1), to t_frac of each end time."""
    import torch
    import paper_1602_00182_gb300.npweno as npw
    from paper_1602_00182_gb300 import build as b
    b.build()
    lib = npw.load()
    torch.cuda.set_device(local_rank)
    inst = I.euler_batch(count=512, seed_index=rank_seed(2, rank))
    ns = [it.n for it in inst]
    tends = [args.t_frac * it.t_end for it in inst]
    table, total = npw.make_instances(ns, [it.dx for it in inst], tends, [CFL] * len(ns), [1] * len(ns), m=3)
    host0 = np.concatenate([it.u0.ravel() for it in inst]).astype(np.float32)
    pristine = torch.tensor(host0, device="cuda")
    arena = pristine.clone()
    # characteristic runs bound |eta| by 1 (the printed eta of a characteristic field blows up at
    # the foot of the Mach-3 shock of the Shu-Osher-type data)
    p = npw.Params(precision=npw.NPW_FP32_MIXED, characteristic=args.characteristic, batch_mode=1,
                   eta_max=1.0 if args.characteristic else 0.0)
    tile = npw.npw_autotune_1d(npw.NPW_FLUX_EULER1D, 3, p)  # later runs with tile_1d = 0 use it
    ws = torch.empty(npw.npw_batch_workspace_size(table, 3, p), dtype=torch.uint8, device="cuda")
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    holder = {}

    def one():
        arena.copy_(pristine)
        st, stats = npw.npweno_batch_solve(arena, table, 3, npw.NPW_FLUX_EULER1D, p, workspace=ws)
        if st != 0:
            raise RuntimeError(f"batch solve failed: {st}")
        holder["stats"] = stats

    for _ in range(args.warmup):
        one()
    pr = npw_profile()
    lib.npw_profile_reset()
    lib.npw_profile_enable(1)
    clocks = Clocks(os.path.join(args.out_dir, f"clocks_rank{rank}.csv"))
    with clocks:
        times = _timed(one, args.steps, flush, world)
    lib.npw_profile_read(ctypes.byref(pr))
    lib.npw_profile_enable(0)
    stats = holder["stats"]
    cu = sum(n * s["steps"] for n, s in zip(ns, stats))
    faces = sum((n + 1) * 3 * 3 * s["steps"] for n, s in zip(ns, stats)) * args.steps
    st_s = pr.stage_ms / 1e3
    fp64 = FP64_OPS_PER_ETA * faces / st_s / 1e9 if (st_s > 0 and not args.characteristic) else None
    alg_bytes = cu * args.steps * 3 * 44  # per field: 12 + 12 + 20 B over the three compensated stages
    tmax, cu_all = job_totals(sum(times), cu * args.steps, world, torch.device("cuda", local_rank))
    return {
        "metric": "cell-updates/s", "value": cu_all / (tmax / 1e3), "unit": "cell-updates/s",
        "ms_per_step": tmax / len(times),
        "config": {"workload": ("batched 1D Euler (m=3, gamma=1.4), transmissive: 512 instances, N log-uniform "
                                f"[256,65536], Riemann + Shu-Osher-type data, {'characteristic' if args.characteristic else 'component'}-wise, "
                                f"RBF-WENO5 MQ + switch, LF, TVD-RK3 CFL 0.5 to {args.t_frac} x each end time"),
                   "instances": 512, "cells": int(sum(ns)), "cell_updates_per_step": int(cu),
                   "path": f"per-stage fused kernels (batch_mode 1), {tile}-cell tiles (autotuned), steps replayed "
                           "as CUDA graphs", "l2": "flushed before every timed step"},
        "roofline": {"bound": "alu", "achieved": fp64, "peak": FP64_PIPE_PEAK / 1e9, "unit": "G FP64-pipe instr/s",
                     "frac": (fp64 / (FP64_PIPE_PEAK / 1e9)) if fp64 else None, "traffic": None,
                     "kernel": ("stage1d_kernel<float, EULER1D> (characteristic, face-based)" if args.characteristic
                                else "stage1d_fast_kernel<EULER1D>"),
                     "hbm_view": {"achieved_gbs": alg_bytes / st_s / 1e9 if st_s > 0 else None,
                                  "peak_gbs": _peaks()[0], "bytes_per_cell_update": 132},
                     "stage_launches": int(pr.stage_launches), "stage_ms": pr.stage_ms},
        "gpu_launches": int(pr.kernel_launches),
        "clocks": clocks.summary(local_rank),
    }


def run_euler2d(args, rank, world, local_rank):
    """2D Euler, dimension by dimension, on periodic squares: 4 x 2048^2 (2^24 cells), isentropic
    vortices and four-quadrant data, ~100 RK3 steps at CFL 0.5 each."""
    import torch
    import paper_1602_00182_gb300.npweno as npw
    from paper_1602_00182_gb300 import build as b
    b.build()
    lib = npw.load()
    torch.cuda.set_device(local_rank)
    n = args.n2d
    count = max(1, (1 << 24) // (n * n))
    doms = I.euler2d_batch(n, count, seed_index=rank_seed(3, rank))
    p = npw.Params(precision=npw.NPW_FP32_MIXED, k=args.k, cross_2d=args.cross_2d)
    pristine = [torch.tensor(U.astype(np.float32), device="cuda") for U, d in doms]
    work = [x.clone() for x in pristine]
    ws = torch.empty(npw.npw_workspace_size_2d(n, n, 4, p), dtype=torch.uint8, device="cuda")
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    tends = []
    for U, d in doms:
        rho, mx, my, E = U
        u, v = mx / rho, my / rho
        c = np.sqrt(1.4 * 0.4 * (E - 0.5 * rho * (u * u + v * v)) / rho)
        rate = (np.abs(u) + c).max() / d + (np.abs(v) + c).max() / d
        tends.append(args.steps2d * CFL / rate)
    holder = {}

    def one():
        tot = 0
        for k, (U, d) in enumerate(doms):
            work[k].copy_(pristine[k])
            st = npw.npweno_solve_2d(work[k], d, d, tends[k], CFL, npw.NPW_FLUX_EULER2D, 0, p, workspace=ws)
            tot += n * n * st["steps"]
        holder["cu"] = tot

    for _ in range(args.warmup):
        one()
    pr = npw_profile()
    lib.npw_profile_reset()
    lib.npw_profile_enable(1)
    clocks = Clocks(os.path.join(args.out_dir, f"clocks_rank{rank}.csv"))
    with clocks:
        times = _timed(one, args.steps, flush, world)
    lib.npw_profile_read(ctypes.byref(pr))
    lib.npw_profile_enable(0)
    cu = holder["cu"]
    st_s = pr.stage_ms / 1e3
    # FP64-pipe view for k = 3 only (k = 2 evaluates two literal FP64 quotients per face)
    fp64 = FP64_OPS_PER_ETA * cu * args.steps * 3 * 4 * 2 / st_s / 1e9 if (st_s > 0 and args.k == 3) else None
    tmax, cu_all = job_totals(sum(times), cu * args.steps, world, torch.device("cuda", local_rank))
    return {
        "metric": "cell-updates/s", "value": cu_all / (tmax / 1e3), "unit": "cell-updates/s",
        "ms_per_step": tmax / len(times),
        "config": {"workload": (f"2D Euler dimension by dimension, periodic {n}^2 x {count} (isentropic vortex + "
                                "four-quadrant), "
                                + ("RBF-WENO5 MQ" if args.k == 3 else
                                   "RBF-WENO3 MQ" + (" with the Sec. 6 cross shape parameter" if args.cross_2d else ""))
                                + f" + switch, one midpoint point per face, ~{args.steps2d} RK3 steps at CFL 0.5"),
                   "domains": count, "cells": n * n * count, "cell_updates_per_step": int(cu),
                   "l2": "flushed before every timed step"},
        "roofline": {"bound": "alu", "achieved": fp64, "peak": FP64_PIPE_PEAK / 1e9, "unit": "G FP64-pipe instr/s",
                     "frac": (fp64 / (FP64_PIPE_PEAK / 1e9)) if fp64 else None, "traffic": None,
                     "kernel": f"stage2d_fast_kernel<EULER2D, k={args.k}>",
                     "hbm_view": {"achieved_gbs": cu * args.steps * 128 / st_s / 1e9 if st_s > 0 else None,
                                  "peak_gbs": _peaks()[0], "bytes_per_cell_update": 128},
                     "stage_launches": int(pr.stage_launches), "stage_ms": pr.stage_ms},
        "gpu_launches": int(pr.kernel_launches),
        "clocks": clocks.summary(local_rank),
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--instances", type=int, default=4096)
    ap.add_argument("--t-end", type=float, default=T_END, help="final time (shorter only for profiling runs)")
    ap.add_argument("--workload", default="burgers", choices=["burgers", "euler1d", "euler2d"],
                    help="burgers: the headline batch; euler1d / euler2d: the other families (separate lines)")
    ap.add_argument("--t-frac", type=float, default=0.1, help="euler1d: fraction of each instance's end time")
    ap.add_argument("--characteristic", type=int, default=0, help="euler1d: characteristic-wise reconstruction")
    ap.add_argument("--n2d", type=int, default=2048, help="euler2d: square size")
    ap.add_argument("--steps2d", type=int, default=100, help="euler2d: RK3 steps per solve")
    ap.add_argument("--k", type=int, default=3, choices=[2, 3], help="euler2d: ENO order parameter (Table k3 / k2)")
    ap.add_argument("--cross-2d", type=int, default=0, choices=[0, 1],
                    help="euler2d with --k 2: shape parameter on the 5-cell cross (Sec. 6)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--eta-eval", type=int, default=0, choices=[0, 1],
                    help="0: eta in FP64 (the configuration's FP64 shape-parameter step); 1: exact double-float")
    ap.add_argument("--serve-requests", type=int, default=60, help="requests of the serving run (0: skip)")
    ap.add_argument("--serve-rates", default="10,100,1000", help="Poisson arrival rates of the serving runs (1/s)")
    ap.add_argument("--variant-steps", type=int, default=1,
                    help="timed solves of the eta_eval=1 variant reported beside the headline (0: skip)")
    ap.add_argument("--out-dir", default=os.path.join(ROOT, "gpurun_out"))
    args = ap.parse_args()
    os.makedirs(args.out_dir, exist_ok=True)
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    cores = os.cpu_count() or 1

    if args.impl == "reference":
        if rank != 0:
            return
        inst = I.burgers_batch(count=args.instances, seed_index=1)
        vals = []
        for _ in range(args.warmup):
            cpu_sample(inst, cores)
        walls = []
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
            "cpu_baseline": {"value": value, "unit": "cell-updates/s", "cores": cores, "kind": "oracle",
                             "sample": desc},
            "e2e": {"value": value, "unit": "cell-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        }))
        return

    if world > 1:
        import torch
        torch.distributed.init_process_group("nccl")
    if args.workload != "burgers":
        fn = run_euler1d if args.workload == "euler1d" else run_euler2d
        out = fn(args, rank, world, local_rank)
        out.update({"n_gpus": world, "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
                    "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded)", "impl": "ours"})
        if rank == 0:
            print(json.dumps(out))
        if world > 1:
            import torch
            torch.distributed.destroy_process_group()
        return
    out, inst = run_gpu(args, rank, world, local_rank)
    if rank == 0 and world == 1 and args.serve_requests > 0:
        import paper_1602_00182_gb300.npweno as npw
        out["serving"] = serving_block(npw, args.serve_requests, [float(x) for x in args.serve_rates.split(",")])
    if rank == 0:
        if not args.no_cpu_baseline:
            v, wall, desc = cpu_sample(inst, cores)
            out["cpu_baseline"] = {"value": v, "unit": "cell-updates/s", "cores": cores, "kind": "oracle",
                                   "sample": desc}
        print(json.dumps(out))
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
