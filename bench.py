#!/usr/bin/env python
"""Benchmark: time to solution of one implicit Stokes step at 1e-8 relative
residual on the 2D 1024^2 Gaussian-bump workload (liquid = 8 seeded bumps,
moving solid disk, log-uniform viscosity 1e-2..1e2, density 1 / 1000 by
region, FP32 stencil inside FP64 iterative refinement).

One step = every stage of the hot path on device-resident inputs: weights,
coefficients and masks from the level sets, right-hand side, mixed-precision
CG with FP64 refinement to a true relative residual of 1e-8, velocity
recovery.  L2 (129 MB) is flushed before every timed step by writing a
512 MB buffer (outside the timed interval).

Prints one JSON line.  ``--impl reference`` times the FP64 CPU oracle on the
same workload instead (host cores; bounded sample, see ``cpu_sample``).
Under torchrun every rank solves its own instance (seed + rank): replicas,
weak scaling, no collective on the data path.
"""
import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM_GBS = 6800.0

# Source files of each reported kernel (the ncu traffic below is valid only
# for the hash of these files it was taken with; see profiles/).
KERNEL_SOURCES = {
    "k_schwarz_gemv": ("schwarz.cuh", "schwarz_plan.cuh", "internal.cuh", "ctx.cuh"),
    "k_apply2d": ("apply.cu", "apply2d_tile.cuh", "internal.cuh", "ctx.cuh"),
    "k_apply3d": ("apply.cu", "internal.cuh", "ctx.cuh"),
}
# (workload, mode, kernel) -> (source hash, dram__bytes_read.sum +
# dram__bytes_write.sum per launch from one ncu capture of the same command)
NCU_TRAFFIC = {
    ("bumps1024", "fp32", "k_schwarz_gemv"): ("79664602fe4c8660", 241.689344e6),   # ncu capture of this command
}


def kernel_source_hash(kernel):
    h = hashlib.sha256()
    for f in KERNEL_SOURCES[kernel]:
        h.update(open(os.path.join(ROOT, "paper_1010_2832_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def ncu_traffic(workload, mode, kernel):
    tr = NCU_TRAFFIC.get((workload, mode, kernel))
    return tr[1] if tr and tr[0] == kernel_source_hash(kernel) else None


def hbm_peak():
    try:
        d = json.load(open(PEAKS_FILE))
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


class ClockSampler:
    """nvidia-smi clock/throttle sampling during the timed region."""

    def __init__(self, gpu_index=0):
        self.gpu = gpu_index
        self.proc = None
        self.rows = []

    def __enter__(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([s.strip() for s in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if len(r) > 3 + i and "Active" in r[3 + i]
                          and "Not" not in r[3 + i]})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


WORKLOADS = {
    "bumps1024": dict(desc="2D 1024x1024, 8 Gaussian-bump liquid, moving disk r=0.1 at (0.5,0), "
                           "mu log-uniform 1e-2..1e2, rho 1|1000, dt=0.01, tol 1e-8", dim=2),
    "column256": dict(desc="3D 256^3 liquid column r=0.05 on a solid floor, rho=1000, mu=10, dt=1e-3, tol 1e-8",
                      dim=3),
    "column128": dict(desc="the 3D column workload at 128^3 (a small case for profiler captures)", dim=3),
    "batch64": dict(desc="64 independent 2D instances, n ~ U{64..512}, Gaussian-bump liquid, random moving disk, "
                         "mu log-uniform 1e-2..1e2, rho=1, each to 1e-8, one persistent launch under a CUDA graph",
                    dim=2),
    "jet150": dict(desc="the planar viscous jet at 150^2 (circle container r=0.4, inflow D=0.06 at U=-0.5, "
                        "mu=0.075, rho=1, g=-9.81, dt=0.002): one Navier-Stokes step = transport + weight build "
                        "+ Schwarz setup + Stokes step to 1e-8", dim=2),
}


def run_batched(args, rank, world):
    """Config-4 step: weights of all instances, then one batched step
    (right-hand sides, the Schwarz setup of every instance, persistent FP64
    PCG of every instance with the additive Schwarz preconditioner (or
    Jacobi), recovery) replayed from a CUDA graph.  Baseline: the same
    instances one by one with plain FP64 Jacobi-PCG."""
    import torch
    from paper_1010_2832_gb300 import stokes, workloads as W
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    wls = W.batch_instances(count=64, seed0=replica_seed(4000, 1000 * rank))
    made = [stokes.context_for(wl) for wl in wls]
    ctxs = [m[0] for m in made]
    devs = [m[1] for m in made]
    precond = 2 if args.precond == "schwarz" else 0
    opt = stokes.default_options(mode=0, tol=args.tol, precond=precond)
    t0 = time.perf_counter()
    batch = stokes.Batch(ctxs, opt)
    tune_s = time.perf_counter() - t0

    def outs(wl):
        nx, ny = wl.n
        return ([torch.zeros(a.shape, dtype=torch.float64, device=dev) for a in wl.u_star],
                [torch.zeros(nx * ny, dtype=torch.float64, device=dev),
                 torch.zeros((nx + 1) * (ny + 1), dtype=torch.float64, device=dev)],
                torch.zeros(nx * ny, dtype=torch.float64, device=dev))
    o = [outs(wl) for wl in wls]
    args_io = ([d["u_star"] for d in devs], [x[0] for x in o], [x[1] for x in o], [x[2] for x in o])
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for _ in range(args.warmup):
        stats, ms = batch.solve(*args_io)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    times = []
    with ClockSampler(dev.index) as clk:
        for k in range(args.steps):
            torch.cuda.synchronize()
            ev0.record()
            for c, d in zip(ctxs, devs):
                c.build_weights(d["phi_liquid"], d["phi_solid"], d["rho"], d["mu"], d["u_bc"])
            torch.cuda.synchronize()
            stats, ms = batch.solve(*args_io)
            ev1.record()
            torch.cuda.synchronize()
            times.append(ev0.elapsed_time(ev1))
    if world > 1:
        torch.distributed.barrier()
    ms_step = max_over_ranks(float(np.mean(times)), world, dev)
    # baseline: the same instances one at a time (plain FP64 Jacobi-PCG, graph loop)
    seq_ms, seq_iters = 0.0, []
    opt_plain = stokes.default_options(mode=0, tol=args.tol, precond=0)
    for (c, d), wl, oo in zip(zip(ctxs, devs), wls, o):
        st = c.solve_step(d["u_star"], oo[0], oo[1], oo[2], opt_plain)
        seq_ms += st.ms_rhs + st.ms_solve + st.ms_recover
        seq_iters.append(st.iterations)
    tun = batch.tuning()
    return {
        "metric": "time-to-solution per implicit step at 1e-8 rel. residual", "value": ms_step, "unit": "ms",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded)",
        "config": {"workload": "batch64", "desc": WORKLOADS["batch64"]["desc"],
                   "preconditioner": ["jacobi", "learned", "schwarz"][precond],
                   "sizes": [wl.n[0] for wl in wls], "l2": "inputs 64 instances (> L2 in total)"},
        "batched": {"ms_batched_solve": float(ms), "tuning": tun, "tuning_s": tune_s,
                    "iterations_max": max(s["iterations"] for s in stats),
                    "failed": sum(1 for s in stats if s["status"] != 0),
                    "worst_rel_residual": max(s["rel_residual"] for s in stats)},
        "one_by_one": {"ms_sum": seq_ms, "iterations_max": max(seq_iters),
                       "note": "same instances solved one after another, FP64 Jacobi-PCG each in its own graph"},
        "clocks": clk.summary(),
    }


def replica_seed(base, rank):
    """Seed of rank ``rank``'s instance: every replica solves its own problem."""
    return base + rank


def max_over_ranks(value, world, device=None):
    """Largest value over the ranks (the slowest replica sets the step time)."""
    if world <= 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def make_workload(name, rank):
    from paper_1010_2832_gb300 import workloads as W
    if name == "bumps1024":
        return W.bumps_2d(1024, seed=replica_seed(2, rank))
    if name == "column256":
        return W.column_3d(256)
    if name == "column128":
        return W.column_3d(128)
    raise SystemExit(f"unknown workload {name}")


def mode_id(m):
    return {"fp64": 0, "fp32": 1, "bf16": 2}[m]


def bytes_per_slot_apply(dim, prec):
    # CG-mode apply: read z, p_old, coefficients; write p_new, q
    nf, nc = (3, 6) if dim == 2 else (6, 11)
    vb = 8 if prec == 0 else 4
    cb = 8 if prec == 0 else (4 if prec == 1 else 2)
    return 4 * nf * vb + nc * cb


def run_jet(args, rank, world):
    """Navier-Stokes step of the planar jet: transport (stokes_advect), the
    weights of the new geometry with the Schwarz setup, one mixed-precision
    Stokes step.  The state evolves from step to step, so the simulation is
    first advanced untimed to t = 1.0 s (after the jet hits the bottom), then
    W warm-up steps, then K timed steps (device events around each step;
    e2e: wall time of the public call JetSim.step, which keeps the state on
    the device and reads back only its statistics and diagnostics)."""
    import torch
    from paper_1010_2832_gb300 import jet
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    sim = jet.JetSim(150, dt=0.002)
    while sim.t < 1.0 - 1e-9:
        sim.step()
    for _ in range(args.warmup):
        sim.step()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    dev_ms, wall_ms = [], []
    with ClockSampler(dev.index) as clk:
        for _ in range(args.steps):
            t0 = time.perf_counter()
            rec = sim.step()
            wall_ms.append((time.perf_counter() - t0) * 1e3)
            dev_ms.append(rec["ms"])
            if rec["status"] != 0:
                raise SystemExit(f"jet step failed: {rec}")
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    ms = max_over_ranks(float(np.mean(dev_ms)), world, dev)
    e2e = max_over_ranks(float(np.mean(wall_ms)), world, dev)
    its = [r["iterations"] for r in sim.history[-args.steps:]]
    sim.close()
    # read back per step: the solver statistics (stokes_stats) and five diagnostics
    d2h = 56 + 5 * 8
    return {
        "metric": "time per Navier-Stokes step (transport, weights, Schwarz setup, Stokes step to 1e-8)",
        "value": ms, "unit": "ms", "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64 transport, f32 CG inside f64 refinement", "data": "synthetic (the paper's jet set-up)",
        "config": {"workload": "jet150", "desc": WORKLOADS["jet150"]["desc"], "t_start": 1.0,
                   "l2": "working set < L2 (150^2); no flush between steps (the state carries over)",
                   "parallelism": f"replicas x{world}"},
        "solver": {"iterations_mean": float(np.mean(its)), "iterations_max": int(max(its))},
        "e2e": {"value": e2e, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": d2h},
        "clocks": clk.summary(),
    }


def run_ours(args, rank, world):
    import torch
    from paper_1010_2832_gb300 import stokes

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    wl = make_workload(args.workload, rank)
    ctx, d = stokes.context_for(wl)
    nf = ctx.layout.nfields
    n = wl.n
    if wl.dim == 2:
        sizes = [n[0] * n[1], (n[0] + 1) * (n[1] + 1), n[0] * n[1]]
    else:
        nx, ny, nz = n
        sizes = [nx * ny * nz, nx * ny * nz, nz * (ny + 1) * (nx + 1), (nz + 1) * ny * (nx + 1),
                 (nz + 1) * (ny + 1) * nx, nx * ny * nz]
    u_out = [torch.zeros_like(t) for t in d["u_star"]]
    taus = [torch.zeros(s, dtype=torch.float64, device=dev) for s in sizes[:-1]]
    p = torch.zeros(sizes[-1], dtype=torch.float64, device=dev)
    precond = {"jacobi": 0, "schwarz": 2}[args.precond]
    if wl.dim != 2:
        precond = 0                    # the Schwarz preconditioner is 2D only
    opt = stokes.default_options(mode=mode_id(args.mode), tol=args.tol, inner_tol=args.inner_tol,
                                 use_graph=0 if args.no_graph else 1, precond=precond)
    flush = torch.empty(args.flush_mb * (1 << 20) // 4, dtype=torch.float32, device=dev)

    wev0, wev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    weights_ms = []

    def step():
        wev0.record()
        ctx.build_weights(d["phi_liquid"], d["phi_solid"], d["rho"], d["mu"], d["u_bc"])   # synchronises
        wev1.record()
        st = ctx.solve_step(d["u_star"], u_out, taus, p, opt)
        weights_ms.append(wev0.elapsed_time(wev1))
        return st

    for _ in range(args.warmup):
        st = step()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    times, stats = [], []
    weights_ms.clear()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(dev.index) as clk:
        for k in range(args.steps):
            flush.fill_(float(k))
            ev0.record()
            st = step()
            ev1.record()
            torch.cuda.synchronize()
            times.append(ev0.elapsed_time(ev1))
            stats.append(st.as_dict())
    if world > 1:
        torch.distributed.barrier()
    if args.quick:   # profiling runs: the timed steps only
        return {"quick": True, "ms": times, "stats": stats}, wl
    ms = max_over_ranks(float(np.mean(times)), world, dev)
    bad = [s for s in stats if s["status"] != 0 or s["rel_residual"] > args.tol]
    iters = int(np.mean([s["iterations"] for s in stats]))
    outer = int(np.mean([s["outer"] for s in stats]))
    # launches per step: weights (5), rhs (1), outer init (1), per refinement
    # step [graph: init + 2 per CG iteration (+2 when the body stops midway),
    # refinement update, residual apply], recovery (1), stress/p unpack (1)
    launches = 5 + 1 + 1 + outer * 5 + 2 * iters + 2

    # ---- end to end through the public API with host buffers -------------
    pin = lambda t: t.cpu().pin_memory()
    h_in = dict(phi_liquid=pin(d["phi_liquid"]), phi_solid=pin(d["phi_solid"]), rho=[pin(t) for t in d["rho"]],
                mu=[pin(t) for t in d["mu"]], u_bc=[pin(t) for t in d["u_bc"]], u_star=[pin(t) for t in d["u_star"]])
    h_out = [pin(t) for t in u_out] + [pin(t) for t in taus] + [pin(p)]
    bi = sum(t.numel() * 8 for v in h_in.values() for t in (v if isinstance(v, list) else [v]))
    bo = sum(t.numel() * 8 for t in h_out)
    e2e_times = []
    for k in range(max(2, args.steps // 2) + 1):
        flush.fill_(float(k))
        torch.cuda.synchronize()
        ev0.record()
        for key in ("phi_liquid", "phi_solid"):
            d[key].copy_(h_in[key], non_blocking=True)
        for key in ("rho", "mu", "u_bc", "u_star"):
            for a, b in zip(d[key], h_in[key]):
                a.copy_(b, non_blocking=True)
        step()
        for a, b in zip(h_out, u_out + taus + [p]):
            a.copy_(b, non_blocking=True)
        ev1.record()
        torch.cuda.synchronize()
        if k > 0:
            e2e_times.append(ev0.elapsed_time(ev1))
    e2e_ms = float(np.mean(e2e_times))

    # ---- roofline of the dominant kernel ----------------------------------
    prec = mode_id(args.mode)
    peak, peak_kind = hbm_peak()
    ms_apply, ms_update = ctx.bench_cg_kernels(prec, 50)
    tiles = ctx.active_tiles()
    slots = tiles * (256 if wl.dim == 2 else 512)
    apply_kernel = "k_apply2d" if wl.dim == 2 else "k_apply3d"
    apply_bytes = slots * bytes_per_slot_apply(wl.dim, prec)
    apply_gbs = apply_bytes / (ms_apply * 1e-3) / 1e9
    if precond == 2:
        ms_local, ms_gather, local_bytes = ctx.bench_schwarz_kernels(50)
        achieved = local_bytes / (ms_local * 1e-3) / 1e9
        roofline = {"kernel": "k_schwarz_gemv (local patch solves of the Schwarz preconditioner)", "bound": "hbm",
                    "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                    "peak_source": peak_kind, "traffic": ncu_traffic(args.workload, args.mode, "k_schwarz_gemv"),
                    "ms_per_launch": ms_local, "bytes_per_launch": local_bytes,
                    "units_per_launch": "every active patch (4x4-slot core + ring)",
                    "gather_ms_per_launch": ms_gather, "source_hash": kernel_source_hash("k_schwarz_gemv")}
    else:
        roofline = {"kernel": f"{apply_kernel} (CG mode: p = z + beta p, q = A p, p.q)", "bound": "hbm",
                    "achieved": apply_gbs, "peak": peak, "unit": "GB/s", "frac": apply_gbs / peak,
                    "peak_source": peak_kind, "traffic": ncu_traffic(args.workload, args.mode, apply_kernel),
                    "ms_per_launch": ms_apply, "bytes_per_launch": apply_bytes, "units_per_launch": slots,
                    "bytes_per_unit": bytes_per_slot_apply(wl.dim, prec), "update_ms_per_launch": ms_update,
                    "source_hash": kernel_source_hash(apply_kernel)}
    stencil = {"kernel": f"{apply_kernel} (CG mode)", "workload": args.workload, "achieved": apply_gbs,
               "unit": "GB/s", "frac": apply_gbs / peak, "ms_per_launch": ms_apply, "bytes_per_launch": apply_bytes,
               "update_ms_per_launch": ms_update}
    if not args.no_dense_apply:
        stencil["dense"] = [dense_apply(dim, n, pr, peak) for dim, n in ((2, 4096), (2, 1024), (3, 256))
                            for pr in (1, 0, 2)]
    out = {
        "metric": "time-to-solution per implicit step at 1e-8 rel. residual",
        "value": ms, "unit": "ms", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 stencil/CG inside f64 refinement" if prec else "f64", "data": "synthetic (seeded)",
        "config": {"workload": args.workload, "desc": WORKLOADS[args.workload]["desc"], "mode": args.mode,
                   "preconditioner": ["jacobi", "learned", "schwarz"][precond],
                   "tol": args.tol, "inner_tol": args.inner_tol, "l2": "flushed (512 MB write) before each step",
                   "parallelism": f"replicas x{world}"},
        "solver": {"iterations": iters, "outer": outer, "rel_residual": max(s["rel_residual"] for s in stats),
                   "failed_steps": len(bad), "ms_rhs": float(np.mean([s["ms_rhs"] for s in stats])),
                   "ms_solve": float(np.mean([s["ms_solve"] for s in stats])),
                   "ms_recover": float(np.mean([s["ms_recover"] for s in stats])),
                   "ms_weights": float(np.mean(weights_ms[:args.steps])) if weights_ms else None,
                   "ms_schwarz_setup": ctx.schwarz_setup_ms() if precond == 2 else None,
                   "steps_per_s_all_ranks": world * 1000.0 / ms},
        "e2e": {"value": e2e_ms, "unit": "ms", "h2d_bytes_per_step": bi, "d2h_bytes_per_step": bo},
        "gpu_launches": launches * args.steps,
        "roofline": roofline,
        "stencil_apply": stencil,
        "clocks": clk.summary(),
    }
    return out, wl


def dense_apply(dim, n, prec, peak):
    """The CG-mode apply on an n^dim box full of liquid, where every tile is
    active: the stencil's streaming bandwidth at scale (precision 0 FP64,
    1 FP32, 2 BF16 coefficients with FP32 vectors)."""
    import torch
    from paper_1010_2832_gb300 import stokes, workloads as W
    wl = W.full_box(n, dim)
    ctx, d = stokes.context_for(wl)
    if dim == 2:
        sizes = [n * n, (n + 1) ** 2, n * n]
    else:
        sizes = [n ** 3, n ** 3, n * (n + 1) ** 2, n * (n + 1) ** 2, n * (n + 1) ** 2, n ** 3]
    u = [torch.zeros_like(t) for t in d["u_star"]]
    taus = [torch.zeros(s, dtype=torch.float64, device=u[0].device) for s in sizes[:-1]]
    p = torch.zeros(sizes[-1], dtype=torch.float64, device=u[0].device)
    ctx.solve_step(d["u_star"], u, taus, p, stokes.default_options(mode=prec, precond=0, max_iter=4))
    ms_a, ms_u = ctx.bench_cg_kernels(prec, 30)
    slots = ctx.active_tiles() * (256 if dim == 2 else 512)
    by = slots * bytes_per_slot_apply(dim, prec)
    gbs = by / (ms_a * 1e-3) / 1e9
    ctx.close()
    del u, taus, p, d
    torch.cuda.empty_cache()
    return {"workload": f"{dim}D {n}^{dim} box full of liquid", "precision": ["fp64", "fp32", "bf16"][prec],
            "achieved": gbs, "frac": gbs / peak, "ms_per_launch": ms_a, "bytes_per_launch": by,
            "units_per_launch": slots, "bytes_per_unit": bytes_per_slot_apply(dim, prec),
            "update_ms_per_launch": ms_u}


def cpu_sample(wl, n_iter_fp64, budget_s=12.0,
               count_source="the FP64 Jacobi-PCG count on the GPU for the same system"):
    """Time the oracle as it stands on host cores: system build (fractions,
    validity, explicit CSR assembly, right-hand side) once, a bounded number
    of its Jacobi-PCG iterations, one recovery; extrapolate to the number of
    FP64 PCG iterations the step needs."""
    from oracle import solve as So
    from oracle import system as S_
    t0 = time.perf_counter()
    S = S_.build_system(S_.StokesInput(**wl.as_oracle_kwargs()))
    t_build = time.perf_counter() - t0
    k = 5
    t_it = So.time_pcg_iterations(S.A, S.b, k) / k
    k2 = int(max(5, min(200, budget_s / max(t_it, 1e-6))))
    t_it = So.time_pcg_iterations(S.A, S.b, k2) / k2
    t0 = time.perf_counter()
    S_.recover_velocity(S, np.zeros(S.A.shape[0]))
    t_rec = time.perf_counter() - t0
    est = t_build + n_iter_fp64 * t_it + t_rec
    return {"value": est * 1000.0, "unit": "ms", "cores": 1, "kind": "oracle",
            "sample": f"oracle build ({t_build:.1f} s) + {k2} Jacobi-PCG iterations ({t_it * 1e3:.1f} ms each) "
                      f"+ recovery on the full system, extrapolated to {n_iter_fp64} iterations ({count_source})"}


def fp64_iterations(wl, with_time=False):
    """Plain FP64 Jacobi-PCG on the same system: iterations (and device ms)."""
    import torch
    from paper_1010_2832_gb300 import stokes
    ctx, d = stokes.context_for(wl)
    b = ctx.new_vector()
    x = ctx.new_vector()
    ctx.rhs(d["u_star"], b)
    st = ctx.solve_system(b, x, stokes.default_options(mode=0, tol=1e-8))
    torch.cuda.synchronize()
    if with_time:
        return st.iterations, st.ms_solve, st.status
    return st.iterations


def run_reference(args):
    """The oracle timed on host cores (the reference arm of this build)."""
    from paper_1010_2832_gb300 import workloads as W  # noqa: F401
    wl = make_workload(args.workload, 0)
    n_it = None
    source = "the FP64 Jacobi-PCG count on the GPU for the same system"
    try:
        n_it = fp64_iterations(wl)
    except Exception:
        n_it = None
    if n_it is None:
        n_it = 20000
        source = "a fixed count: no GPU to measure the FP64 Jacobi-PCG count, which is about 1.6e5 on this system"
    vals = []
    for k in range(args.warmup + args.steps):
        s = cpu_sample(wl, n_it, budget_s=3.0, count_source=source)
        if k >= args.warmup:
            vals.append(s["value"])
    v = float(np.mean(vals))
    return {"impl": "reference", "metric": "time-to-solution per implicit step at 1e-8 rel. residual", "value": v,
            "unit": "ms", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": v,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded)", "config": {"workload": args.workload,
                                                     "desc": WORKLOADS[args.workload]["desc"]},
            "cpu_baseline": dict(s, value=v),
            "e2e": {"value": v, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="bumps1024", choices=list(WORKLOADS))
    ap.add_argument("--mode", default="fp32", choices=["fp64", "fp32", "bf16"])
    ap.add_argument("--precond", default="schwarz", choices=["jacobi", "schwarz"])
    ap.add_argument("--tol", type=float, default=1e-8)
    ap.add_argument("--inner-tol", type=float, default=1e-4)
    ap.add_argument("--flush-mb", type=int, default=512)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-dense-apply", action="store_true", help="skip the dense-box apply measurement")
    ap.add_argument("--quick", action="store_true", help="timed steps only (for profiler runs)")
    ap.add_argument("--no-graph", action="store_true",
                    help="host-driven CG loop (profilers cannot enter conditional graphs)")
    args = ap.parse_args()
    if args.quick:
        args.no_cpu_baseline = True
        args.no_dense_apply = True
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(run_reference(args)))
        return
    import torch
    if world > 1:
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        torch.distributed.init_process_group("nccl")
    if args.workload in ("batch64", "jet150"):
        out = (run_batched if args.workload == "batch64" else run_jet)(args, rank, world)
        if rank == 0:
            print(json.dumps(out))
        if world > 1:
            torch.distributed.destroy_process_group()
        return
    out, wl = run_ours(args, rank, world)
    if rank == 0 and not args.no_cpu_baseline:
        try:
            n_it, ms64, st64 = fp64_iterations(wl, with_time=True)
            out["plain_fp64_pcg"] = {"iterations": n_it, "ms_solve": ms64, "status": st64,
                                     "note": "plain FP64 Jacobi-PCG on the same system (solve only)"}
            out["cpu_baseline"] = cpu_sample(wl, n_it)
            out["solver"]["fp64_pcg_iterations"] = n_it
        except Exception as e:  # the baseline must not hide the GPU result
            out["cpu_baseline"] = {"value": None, "error": repr(e)}
    if rank == 0:
        print(json.dumps(out))
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
