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
import re
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM_GBS = 6800.0

# Sources of each reported kernel: whole files, or (file, struct names) for
# the definitions of the types a kernel takes from a shared header (the ncu
# traffic below is valid only for the hash of these sources it was taken
# with; see profiles/).
KERNEL_SOURCES = {
    "k_schwarz_gemv": ("schwarz.cuh", "schwarz_plan.cuh", ("internal.cuh", ("Layout", "CgScalars"))),
    "k_apply2d": ("apply.cu", "apply2d_tile.cuh", "internal.cuh", "ctx.cuh"),
    "k_apply3d": ("apply.cu", "internal.cuh", "ctx.cuh"),
}
# (workload, mode, kernel) -> (source hash, dram__bytes_read.sum +
# dram__bytes_write.sum per launch from one ncu capture of the same command)
NCU_TRAFFIC = {
    ("bumps1024", "fp32", "k_schwarz_gemv"): ("fff896e2cd21474e", 244.706048e6),   # ncu capture of this command
}


def struct_source(text, name):
    """The definition of ``struct name`` in a header: from its opening line to
    the first ``};`` at the start of a line."""
    m = re.search(r"^struct " + re.escape(name) + r" \{.*?^\};", text, re.S | re.M)
    if m is None:
        raise KeyError(f"struct {name} not found")
    return m.group(0)


def kernel_source_hash(kernel, csrc=None):
    csrc = csrc or os.path.join(ROOT, "paper_1010_2832_gb300", "csrc")
    h = hashlib.sha256()
    for f in KERNEL_SOURCES[kernel]:
        if isinstance(f, tuple):
            text = open(os.path.join(csrc, f[0])).read()
            for name in f[1]:
                h.update(struct_source(text, name).encode())
        else:
            h.update(open(os.path.join(csrc, f), "rb").read())
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
    "learned128": dict(desc="3D Gaussian-bump instances (8 bumps, moving sphere, log-uniform mu 1e-2..1e2, rho 1|1000; "
                            "face-mass floor 0.01): BF16 3-level U-Net (tensor cores) trained on 2,000 solver-generated "
                            "residual/error pairs (64^3 windows of 20 128^3 instances), then held-out 128^3 and 256^3 "
                            "instances solved to 1e-8 by the learned flexible CG, by Jacobi-CG in the same mixed "
                            "precision and by plain FP64 Jacobi-PCG", dim=3),
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


def run_learned(args, rank, world):
    """The learned preconditioner at the stated scale (one run, not a timed
    loop: the training itself is the work; value = device time of the
    learned solve on the first held-out 128^3 instance)."""
    import torch
    from paper_1010_2832_gb300 import learned
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    with ClockSampler(dev.index) as clk:
        res = learned.config5(log=lambda m: print(m, file=sys.stderr, flush=True))
    first = res["eval"][0]
    return {
        "metric": "time-to-solution per implicit step at 1e-8 rel. residual", "value": first["learned"]["ms_device"],
        "unit": "ms", "n_gpus": world, "steps": 1, "warmup": 0, "ms_per_step": first["learned"]["ms_device"],
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": "bf16 network (f32 accumulation), f32 flexible CG inside f64 refinement", "data": "synthetic (seeded)",
        "config": {"workload": "learned128", "desc": WORKLOADS["learned128"]["desc"], "parallelism": f"replicas x{world}"},
        "learned": res, "clocks": clk.summary(),
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
    u_out, taus, p = _outputs(wl, d)
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
    active_slots = count_active_slots(ctx, wl)
    active_bytes = active_slots * bytes_per_slot_apply(wl.dim, prec)
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
               "units_per_launch": f"{slots} slots of active tiles",
               "active_slots": active_slots, "achieved_over_active_slots": active_bytes / (ms_apply * 1e-3) / 1e9,
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
        "velocity_error_vs_oracle": velocity_error(u_out, oracle_velocity_samples(args.workload)),
        "gpu_launches": launches * args.steps,
        "roofline": roofline,
        "stencil_apply": stencil,
        "clocks": clk.summary(),
        "_ctx": (ctx, d),
    }
    return out, wl


def count_active_slots(ctx, wl):
    """Slots (i, j[, k]) holding at least one active unknown."""
    act = ctx.export(3).cpu().numpy().astype(bool)
    n = wl.n
    if wl.dim == 2:
        nx, ny = n
        shapes = [(ny, nx), (ny + 1, nx + 1), (ny, nx)]
        lat = np.zeros((ny + 1, nx + 1), dtype=bool)
    else:
        nx, ny, nz = n
        shapes = [(nz, ny, nx), (nz, ny, nx), (nz, ny + 1, nx + 1), (nz + 1, ny, nx + 1), (nz + 1, ny + 1, nx),
                  (nz, ny, nx)]
        lat = np.zeros((nz + 1, ny + 1, nx + 1), dtype=bool)
    o = 0
    for shp in shapes:
        m = int(np.prod(shp))
        a = act[o:o + m].reshape(shp)
        lat[tuple(slice(0, t) for t in shp)] |= a
        o += m
    return int(lat.sum())


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


GOLDEN = os.path.join(ROOT, "tests", "golden")


def oracle_pcg_count(n):
    """The oracle's own FP64 Jacobi-PCG iteration count to 1e-8 on the 2D
    Gaussian-bump workload at n^2 (written by
    tests/golden/make_oracle_pcg_counts.py, which runs only the oracle), and
    the whole table for the report."""
    path = os.path.join(GOLDEN, "oracle_pcg_counts.txt")
    rows, head = {}, []
    if os.path.exists(path):
        for line in open(path):
            if line.startswith("#"):
                head.append(line[1:].strip())
            elif line.strip():
                f = line.split()
                rows[int(f[0])] = dict(iterations=int(f[1]), rel_residual=float(f[2]), build_s=float(f[3]),
                                       solve_s=float(f[4]), ms_per_iteration=float(f[5]), active=int(f[6]),
                                       blas_threads=int(f[7]) if len(f) > 7 else None)
    return rows.get(n, {}).get("iterations"), {"rows": rows, "header": head}


def oracle_velocity_samples(name):
    """(face indices, oracle velocities, scale) from
    tests/golden/oracle_velocity_<name>.txt, or None."""
    path = os.path.join(GOLDEN, f"oracle_velocity_{name}.txt")
    if not os.path.exists(path):
        return None
    scale = None
    idx, val = [], []
    for line in open(path):
        if line.startswith("# scale"):
            scale = float(line.split(":")[1])
        elif line.strip() and not line.startswith("#"):
            a, b = line.split()
            idx.append(int(a))
            val.append(float(b))
    return np.array(idx), np.array(val), scale


def window_face_to_full(idx, n, win):
    """Face indices of a window's face fields (u, v, w concatenated) to the
    full n^3 grid's."""
    i0, j0, k0, ni, nj, nk = win
    wsh = [(nk, nj, ni + 1), (nk, nj + 1, ni), (nk + 1, nj, ni)]
    fsh = [(n, n, n + 1), (n, n + 1, n), (n + 1, n, n)]
    woff = np.cumsum([0] + [int(np.prod(t)) for t in wsh])
    foff = np.cumsum([0] + [int(np.prod(t)) for t in fsh])
    out = np.empty_like(idx)
    for d in range(3):
        m = (idx >= woff[d]) & (idx < woff[d + 1])
        k, j, i = np.unravel_index(idx[m] - woff[d], wsh[d])
        out[m] = foff[d] + np.ravel_multi_index((k + k0, j + j0, i + i0), fsh[d])
    return out


def velocity_error(u_fields, samples, index_map=None):
    """Largest |u - u_oracle| over the stored samples, relative to the
    oracle's largest live-face |u|."""
    if samples is None:
        return None
    idx, val, scale = samples
    u = np.concatenate([t.detach().cpu().numpy().ravel() for t in u_fields])
    if index_map is not None:
        idx = index_map(idx)
    return float(np.abs(u[idx] - val).max() / scale)


def host_cpu():
    model = None
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except OSError:
        pass
    if model is None:
        import platform
        model = platform.processor() or platform.machine()
    return model, os.cpu_count()


BLAS_ENV = ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS")


def _capped_child(conn, fn, args):
    try:
        conn.send(("ok", fn(*args)))
    except BaseException as e:  # reported to the parent
        conn.send(("error", repr(e)))
    conn.close()


def run_blas_capped(fn, *args, threads=None):
    """fn(*args) with numpy's BLAS pool capped at ``threads`` (None: the
    default pool).  With threadpoolctl the cap is set in this process;
    where it is not installed, fn runs in a spawned process started with
    the BLAS thread variables set (spawned, not forked: this process may
    hold a CUDA context).  Returns (result, how the cap was set)."""
    if threads is None:
        return fn(*args), "default pool"
    try:
        from threadpoolctl import threadpool_limits
    except ImportError:
        threadpool_limits = None
    if threadpool_limits is not None:
        with threadpool_limits(limits=threads):
            return fn(*args), "threadpoolctl"
    import multiprocessing as mp
    old = {k: os.environ.get(k) for k in BLAS_ENV}
    try:
        for k in BLAS_ENV:
            os.environ[k] = str(threads)
        ctx = mp.get_context("spawn")
        parent, child = ctx.Pipe(duplex=False)
        proc = ctx.Process(target=_capped_child, args=(child, fn, args))
        proc.start()
        child.close()
        try:
            kind, res = parent.recv()      # EOFError if the child died before sending
        finally:
            proc.join()
        if kind != "ok":
            raise RuntimeError(f"capped oracle run failed: {res}")
    finally:
        for k, v in old.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    return res, "spawned process, BLAS thread variables set"


def _pcg_iteration_sample(A, b, budget_s):
    """Seconds per oracle Jacobi-PCG iteration: 5 iterations to size the
    sample, then as many as fit in budget_s (5..400)."""
    from oracle import solve as So
    k = 5
    t_it = So.time_pcg_iterations(A, b, k) / k
    k2 = int(max(5, min(400, budget_s / max(t_it, 1e-6))))
    return So.time_pcg_iterations(A, b, k2) / k2, k2


def _timed_pcg(A, b, tol):
    from oracle import solve as So
    t0 = time.perf_counter()
    _, it, rel = So.pcg(A, b, tol=tol, max_iter=10 ** 7)
    return (time.perf_counter() - t0) * 1e3, it, rel


def cpu_sample(wl, n_iter, budget_s=8.0, count_source="", threads=None, S=None):
    """Time the oracle as it stands on host cores: the system build
    (fractions, validity, explicit CSR assembly, right-hand side) once, a
    bounded number of its Jacobi-PCG iterations, one recovery; extrapolate to
    ``n_iter`` iterations.  ``threads`` caps numpy's BLAS pool (None: the
    default pool; scipy's sparse product runs on one thread either way)."""
    from oracle import system as S_
    t_build = None
    if S is None:
        t0 = time.perf_counter()
        S = S_.build_system(S_.StokesInput(**wl.as_oracle_kwargs()))
        t_build = time.perf_counter() - t0
    (t_it, k2), _ = run_blas_capped(_pcg_iteration_sample, S.A, S.b, budget_s, threads=threads)
    t0 = time.perf_counter()
    S_.recover_velocity(S, np.zeros(S.A.shape[0]))
    t_rec = time.perf_counter() - t0
    return S, t_build, t_it, t_rec, k2


def cpu_baseline(wl, n, budget_s=8.0):
    """The oracle on this host: build once, then bounded samples of its
    Jacobi-PCG iterations on all host cores (default BLAS pool) and on one
    thread, extrapolated to the oracle's own iteration count for this
    workload."""
    n_it, table = oracle_pcg_count(n)
    model, ncpu = host_cpu()
    if n_it is None:
        return {"value": None, "unit": "ms", "kind": "oracle", "cores": ncpu,
                "error": "no oracle iteration count for this workload in tests/golden/oracle_pcg_counts.txt"}
    S, t_build, t_all, t_rec, k_all = cpu_sample(wl, n_it, budget_s)
    _, _, t_one, _, k_one = cpu_sample(wl, n_it, budget_s, threads=1, S=S)
    est = lambda t: (t_build + n_it * t + t_rec) * 1000.0
    return {"value": est(t_all), "unit": "ms", "cores": ncpu, "kind": "oracle",
            "sample": f"oracle build ({t_build:.1f} s), {k_all} of its FP64 Jacobi-PCG iterations "
                      f"({t_all * 1e3:.2f} ms each) and one recovery on the full system, extrapolated to the "
                      f"oracle's own {n_it} iterations to 1e-8 (tests/golden/oracle_pcg_counts.txt); "
                      f"numpy's default BLAS pool on {ncpu} cores (the sparse product itself is one thread)",
            "single_thread": {"value": est(t_one), "ms_per_iteration": t_one * 1e3, "iterations_sampled": k_one},
            "ms_per_iteration": t_all * 1e3, "build_s": t_build, "iterations": n_it,
            "cpu": model, "complete_solves_elsewhere": table}


def gpu_plain_fp64(ctx, d):
    """Plain FP64 Jacobi-PCG on the GPU on the same system (solve only)."""
    import torch
    from paper_1010_2832_gb300 import stokes
    b = ctx.new_vector()
    x = ctx.new_vector()
    ctx.rhs(d["u_star"], b)
    st = ctx.solve_system(b, x, stokes.default_options(mode=0, tol=1e-8))
    torch.cuda.synchronize()
    return {"iterations": st.iterations, "ms_solve": st.ms_solve, "status": st.status,
            "rel_residual": st.rel_residual, "note": "plain FP64 Jacobi-PCG on the same system (solve only)"}


def _outputs(wl, d):
    import torch
    n = wl.n
    dev = d["u_star"][0].device
    if wl.dim == 2:
        sizes = [n[0] * n[1], (n[0] + 1) * (n[1] + 1), n[0] * n[1]]
    else:
        nx, ny, nz = n
        sizes = [nx * ny * nz, nx * ny * nz, nz * (ny + 1) * (nx + 1), (nz + 1) * ny * (nx + 1),
                 (nz + 1) * (ny + 1) * nx, nx * ny * nz]
    u_out = [torch.zeros_like(t) for t in d["u_star"]]
    taus = [torch.zeros(s, dtype=torch.float64, device=dev) for s in sizes[:-1]]
    p = torch.zeros(sizes[-1], dtype=torch.float64, device=dev)
    return u_out, taus, p


def config_column256(args, flush):
    """The 3D 256^3 falling column: the mixed-precision step (weights, right-
    hand side, FP32 Jacobi-CG in FP64 refinement, recovery) timed like the
    headline step, the same step in plain FP64 PCG, and both velocities
    against the oracle on the column's liquid window."""
    import torch
    from paper_1010_2832_gb300 import stokes, workloads as W
    wl = W.column_3d(256)
    ctx, d = stokes.context_for(wl)
    u_out, taus, p = _outputs(wl, d)
    samples = oracle_velocity_samples("column256")
    win = (111, 0, 111, 34, 160, 34)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    out = {"workload": "column256", "desc": WORKLOADS["column256"]["desc"]}
    for name, opt in (("mixed_fp32_jacobi", stokes.default_options(mode=1, tol=1e-8)),
                      ("plain_fp64_pcg", stokes.default_options(mode=0, tol=1e-8))):
        times, stats = [], []
        for k in range(2 + 3):
            flush.fill_(float(k))
            ev0.record()
            ctx.build_weights(d["phi_liquid"], d["phi_solid"], d["rho"], d["mu"], d["u_bc"])
            st = ctx.solve_step(d["u_star"], u_out, taus, p, opt)
            ev1.record()
            torch.cuda.synchronize()
            if k >= 2:
                times.append(ev0.elapsed_time(ev1))
                stats.append(st.as_dict())
        out[name] = {"ms_per_step": float(np.mean(times)), "iterations": stats[-1]["iterations"],
                     "outer": stats[-1]["outer"], "rel_residual": stats[-1]["rel_residual"],
                     "status": stats[-1]["status"], "ms_solve": float(np.mean([s["ms_solve"] for s in stats])),
                     "velocity_error_vs_oracle": velocity_error(
                         u_out, samples, lambda i: window_face_to_full(i, 256, win))}
    ctx.close()
    del u_out, taus, p, d
    torch.cuda.empty_cache()
    out["note"] = ("3 timed steps after 2 warm-up steps each, weights included, L2 flushed; velocity error = max "
                   "over 4,096 oracle samples on the liquid window of |u - u_oracle| / max|u_oracle|")
    return out


def config_batch64(args):
    """64 uneven 2D instances: the batched step (persistent FP64 Schwarz-PCG
    under a CUDA graph) against the same instances one after another with
    plain FP64 Jacobi-PCG and with the single-instance mixed Schwarz-CG."""
    import torch
    from paper_1010_2832_gb300 import stokes, workloads as W
    wls = W.batch_instances(count=64, seed0=4000)
    made = [stokes.context_for(wl) for wl in wls]
    ctxs = [m[0] for m in made]
    devs = [m[1] for m in made]
    batch = stokes.Batch(ctxs, stokes.default_options(mode=0, tol=1e-8, precond=2))
    o = [_outputs(wl, d) for wl, d in zip(wls, devs)]
    args_io = ([d["u_star"] for d in devs], [x[0] for x in o], [x[1] for x in o], [x[2] for x in o])
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    batch.solve(*args_io)
    times = []
    for _ in range(2):
        torch.cuda.synchronize()
        ev0.record()
        for c, d in zip(ctxs, devs):
            c.build_weights(d["phi_liquid"], d["phi_solid"], d["rho"], d["mu"], d["u_bc"])
        stats, ms = batch.solve(*args_io)
        ev1.record()
        torch.cuda.synchronize()
        times.append(ev0.elapsed_time(ev1))
    res = {"workload": "batch64", "desc": WORKLOADS["batch64"]["desc"],
           "batched_fp64_schwarz": {"ms_per_step": float(np.mean(times)),
                                    "iterations_max": max(s["iterations"] for s in stats),
                                    "failed": sum(1 for s in stats if s["status"] != 0),
                                    "worst_rel_residual": max(s["rel_residual"] for s in stats),
                                    "tuning": batch.tuning()}}
    batch.close()
    for name, opt in (("one_by_one_plain_fp64_pcg", stokes.default_options(mode=0, tol=1e-8, precond=0)),
                      ("one_by_one_mixed_fp32_schwarz", stokes.default_options(mode=1, tol=1e-8, precond=2))):
        total, its, bad = 0.0, [], 0
        for c, d, oo in zip(ctxs, devs, o):
            ev0.record()
            c.build_weights(d["phi_liquid"], d["phi_solid"], d["rho"], d["mu"], d["u_bc"])
            st = c.solve_step(d["u_star"], oo[0], oo[1], oo[2], opt)
            ev1.record()
            torch.cuda.synchronize()
            total += ev0.elapsed_time(ev1)
            its.append(st.iterations)
            bad += st.status != 0
        res[name] = {"ms_sum": total, "iterations_max": max(its), "failed": bad}
    for c in ctxs:
        c.close()
    torch.cuda.empty_cache()
    res["note"] = "weights included in every form; batched: mean of 2 steps after one warm-up"
    return res


def run_reference(args):
    """The oracle timed on host cores (the reference arm of this build): no
    GPU and no library of this package; the input generators only."""
    from paper_1010_2832_gb300 import workloads as W  # seeded inputs, no method arithmetic
    from oracle import solve as So
    from oracle import system as S_
    if args.workload != "bumps1024":
        return {"impl": "reference", "unavailable": "the oracle's iteration count is recorded for the 2D "
                                                    "Gaussian-bump workload only"}
    n = args.ref_size
    wl = W.bumps_2d(n, seed=2)
    n_it, table = oracle_pcg_count(n)
    model, ncpu = host_cpu()
    if n_it is None:
        return {"impl": "reference", "unavailable": f"tests/golden/oracle_pcg_counts.txt holds no {n}^2 count"}
    t0 = time.perf_counter()
    S = S_.build_system(S_.StokesInput(**wl.as_oracle_kwargs()))
    t_build = time.perf_counter() - t0
    vals, per_it = [], []
    for k in range(args.warmup + args.steps):
        _, _, t_it, t_rec, k2 = cpu_sample(wl, n_it, budget_s=2.0, S=S)
        if k >= args.warmup:
            per_it.append(t_it)
            vals.append((t_build + n_it * t_it + t_rec) * 1000.0)
    v = float(np.mean(vals))
    # complete oracle solves on this host: config 1 (32^2 disk, FP64 PCG to
    # 1e-10) and the bump workload at a small size (to 1e-8), on all cores
    # and on one
    complete = {}
    nb = args.ref_complete_size
    for label, wlc, tol in (("disk32_config1", W.disk_in_box(32, seed=1), 1e-10),
                            (f"bumps{nb}", W.bumps_2d(nb, seed=2), 1e-8)):
        Sc = S_.build_system(S_.StokesInput(**wlc.as_oracle_kwargs()))
        for th_name, th in (("all_cores", None), ("one_thread", 1)):
            (ms, it, rel), how = run_blas_capped(_timed_pcg, Sc.A, Sc.b, tol, threads=th)
            complete[f"{label}_{th_name}"] = {"ms": ms, "iterations": it, "rel_residual": rel, "threads": how}
    sample = (f"oracle build ({t_build:.1f} s, once) + per step a bounded sample of its FP64 Jacobi-PCG iterations "
              f"on the full {n}^2 system ({np.mean(per_it) * 1e3:.2f} ms each), extrapolated to the oracle's own "
              f"{n_it} iterations to 1e-8 (tests/golden/oracle_pcg_counts.txt); numpy's default BLAS pool on "
              f"{ncpu} cores (the sparse product is one thread)")
    return {"impl": "reference", "metric": "time-to-solution per implicit step at 1e-8 rel. residual", "value": v,
            "unit": "ms", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": v,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded)", "config": {"workload": args.workload,
                                                     "desc": WORKLOADS[args.workload]["desc"]},
            "cpu_baseline": {"value": v, "unit": "ms", "cores": ncpu, "kind": "oracle", "sample": sample,
                             "cpu": model, "complete_solves": complete,
                             "complete_solves_elsewhere": table},
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
    ap.add_argument("--no-configs", action="store_true", help="skip the 3D column and 64-instance batch lines")
    ap.add_argument("--ref-size", type=int, default=1024, help=argparse.SUPPRESS)
    ap.add_argument("--ref-complete-size", type=int, default=128, help=argparse.SUPPRESS)
    ap.add_argument("--no-dense-apply", action="store_true", help="skip the dense-box apply measurement")
    ap.add_argument("--quick", action="store_true", help="timed steps only (for profiler runs)")
    ap.add_argument("--no-graph", action="store_true",
                    help="host-driven CG loop (profilers cannot enter conditional graphs)")
    ap.add_argument("--dense-apply-only", metavar="DIM:N:PREC",
                    help="only the CG-mode apply on an N^DIM box full of liquid (PREC 0 FP64, 1 FP32, 2 BF16 "
                         "coefficients): one JSON line (for profiler runs)")
    args = ap.parse_args()
    if args.dense_apply_only:
        dim, n, prec = (int(v) for v in args.dense_apply_only.split(":"))
        print(json.dumps(dense_apply(dim, n, prec, hbm_peak()[0])))
        return
    if args.quick:
        args.no_cpu_baseline = True
        args.no_dense_apply = True
        args.no_configs = True
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
    if args.workload in ("batch64", "jet150", "learned128"):
        out = {"batch64": run_batched, "jet150": run_jet, "learned128": run_learned}[args.workload](args, rank, world)
        if rank == 0:
            print(json.dumps(out))
        if world > 1:
            torch.distributed.destroy_process_group()
        return
    out, wl = run_ours(args, rank, world)
    if rank == 0 and not args.quick:
        try:
            out["plain_fp64_pcg"] = gpu_plain_fp64(*out.pop("_ctx"))
            out["solver"]["fp64_pcg_iterations"] = out["plain_fp64_pcg"]["iterations"]
        except Exception as e:  # a baseline must not hide the GPU result
            out["plain_fp64_pcg"] = {"error": repr(e)}
    out.pop("_ctx", None)
    if rank == 0 and not args.quick and not args.no_configs and args.workload == "bumps1024":
        flush = torch.empty(args.flush_mb * (1 << 20) // 4, dtype=torch.float32, device="cuda")
        out["configs"] = {}
        for key, fn in (("column256", lambda: config_column256(args, flush)), ("batch64", lambda: config_batch64(args))):
            try:
                out["configs"][key] = fn()
            except Exception as e:
                out["configs"][key] = {"error": repr(e)}
    if rank == 0 and not args.no_cpu_baseline and wl.dim == 2 and args.workload == "bumps1024":
        try:
            out["cpu_baseline"] = cpu_baseline(wl, wl.n[0])
        except Exception as e:  # the baseline must not hide the GPU result
            out["cpu_baseline"] = {"value": None, "error": repr(e)}
    if rank == 0:
        print(json.dumps(out))
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
