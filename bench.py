"""Benchmark of one outer iteration of the memory-reduced iterative DVM scheme
(arXiv 1810.00348) on the GB300, printed as one JSON line.

Workload: the 3D lid-driven cavity with 64^3 uniform cells and 32^3 uniform
velocities on [-4, 4]^3 (trapezoid weights), Shakhov Pr = 2/3, omega = 0.81,
Kn = 1, lid speed 0.16 (synthetic problem definition, no dataset).  A step is
one outer iteration: coefficients, all sweep stages with the fused
equilibrium and moments, and the FP64 closure (moments -> macros, wall
densities, mass rescale, residual).  The headline value is the mixed form
(FP32 sweep and equilibrium, FP64 moment partials and closure); the plain
FP64 form is measured beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the FP64 CPU oracle (the reference arm of this build)
on a bounded sample of the same workload.  Under torchrun each rank runs an
independent replica of the workload (the solver is single-GPU; weak scaling).
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "phase-point updates/s"
WORKLOAD = "3D lid-driven cavity 64^3 cells x 32^3 velocities, Kn=1, lid 0.16"
N_CELL, N_VEL, KN, LID = 64, 32, 1.0, 0.16

# Algorithmic FP32/FP64 operations per phase-point update in the sweep kernel
# (FMA = 2): equilibrium of Eq. (2) 20 + exp 1; implicit update of Eq. (7)
# 13 (with the division); 13 moment sums about U^n 34.
FLOPS_PER_PP = 68
# The second-order sweep adds three extrapolated upwind values
# h_d = f_1 + (f_1 - f_2)/3 (a subtraction and an FMA each) and the scaled
# coefficients 3 a_d / 2.
FLOPS_PER_PP_ORDER2 = FLOPS_PER_PP + 9 + 3
# dram__bytes_read.sum + dram__bytes_write.sum of one sweep launch (ncu, 32^3
# cells x 32^3 velocities, 256 velocities per CTA, blocks 8x8x32): 2.897e9 B
# over 1.074e9 phase points
TRAFFIC_BYTES_PER_PP = 2.897e9 / 1.074e9
TRAFFIC_SHAPE = (256, 32)
SM_COUNT = 152
FP32_LANES_PER_SM = 128
FP64_PEAK_TFLOPS = 1.25  # nominal dense FP64 of the GB300


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return json.load(f)
    except OSError:
        return {}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = str(gpu_index)
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", self.gpu, "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def max_over_ranks(x, dist=None, device="cpu"):
    """Largest value of x over the ranks of the default process group (x
    itself when there is none): the whole-job time of a step is the slowest
    rank's."""
    if dist is None:
        return float(x)
    import torch

    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def rel_errors(got, ref):
    """Largest relative field errors: rho and T pointwise, U and q normalised
    by the largest magnitude of the reference field (they pass through zero)."""
    g = np.asarray(got).reshape(8, -1)
    r = np.asarray(ref).reshape(8, -1)
    err = {"rho": float(np.max(np.abs(g[0] - r[0]) / np.abs(r[0]))),
           "T": float(np.max(np.abs(g[4] - r[4]) / np.abs(r[4])))}
    for name, sl in (("U", slice(1, 4)), ("q", slice(5, 8))):
        err[name] = float(np.max(np.abs(g[sl] - r[sl])) / max(np.max(np.abs(r[sl])), 1e-300))
    # the scales of the two normalised fields (q is small early in a run)
    err["ref_max_abs"] = {"U": float(np.max(np.abs(r[1:4]))), "q": float(np.max(np.abs(r[5:8])))}
    return err


def time_oracle_sample(kgs=None, threads=1):
    """Oracle (plain FP64 C) on a bounded sample of the workload: the
    64^3-cell cavity with an 8^3 velocity grid (one outer iteration, about 15 s
    on one core).  threads > 1 runs the oracle's concurrent velocity ranges
    on that many host threads (the same arithmetic, summed in range order).
    Given the library, the GPU FP64 and mixed paths run the same iteration and
    their errors against the oracle's result are reported."""
    from oracle import Oracle, parallel_build
    from paper_1810_00348_gb300 import inputs

    if threads > 1 and not parallel_build():
        threads = 1
    prob = inputs.cavity(N_CELL, 8, Kn=KN, lid=LID)
    o = Oracle(prob, threads=threads)
    t0 = time.perf_counter()
    o.iterate()
    dt = time.perf_counter() - t0
    pp = prob.phase_points()
    out = {"value": pp / dt, "unit": "phase-point updates/s", "cores": threads, "kind": "oracle",
           "sample": "one outer iteration of the 64^3-cell cavity with an 8^3 velocity grid "
                     "(%d phase points, %.1f s on %d host thread%s)" % (pp, dt, threads, "s" if threads > 1 else "")}
    if kgs is not None:
        ref = o.macros()
        out["gpu_error_vs_oracle"] = {}
        for name, prec in (("fp64", kgs.KGS_FP64), ("mixed", kgs.KGS_MIXED)):
            c = kgs.kgs_setup(prob, precision=prec)
            kgs.kgs_iterate(c, 1)
            out["gpu_error_vs_oracle"][name] = rel_errors(kgs.kgs_moments(c), ref)
            del c
    return out


def run_reference(args, world, rank):
    if rank != 0:
        return
    # the oracle is plain CPU code with no warm-up effects: every step is a
    # timed sample, run on all host cores so that the whole run stays within
    # a few minutes
    cores = os.cpu_count() or 1
    cb = time_oracle_sample(threads=cores)
    vals = [cb["value"]]
    for _ in range(max(args.steps - 1, 0)):
        vals.append(time_oracle_sample(threads=cores)["value"])
    v = statistics.median(vals)
    cb["value"] = v
    sample_pp = float(N_CELL ** 3 * 8 ** 3)  # phase points of one sampled step
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "phase-point updates/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sample_pp / v, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD + " (oracle sample: 8^3 velocities)"},
            "cpu_baseline": cb,
            "e2e": {"value": v, "unit": "phase-point updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args, world, rank, local):
    import torch

    from paper_1810_00348_gb300 import inputs, kgs

    torch.cuda.set_device(local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        pg = dist
    kgs.load()
    prob = inputs.cavity(args.cells, args.vels, Kn=KN, lid=LID)
    pp = prob.phase_points()
    peaks = _peaks()
    workload = WORKLOAD if (args.cells, args.vels) == (N_CELL, N_VEL) else \
        "3D lid-driven cavity %d^3 cells x %d^3 velocities, Kn=1, lid 0.16" % (args.cells, args.vels)
    if args.dev_source:
        workload += ", deviation-form FP32 source"

    def barrier():
        if pg is not None:
            pg.barrier()
        torch.cuda.synchronize()

    def timed(ctx, steps):
        kgs.kgs_profile(ctx)  # reset counters
        barrier()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record()
        for _ in range(steps):
            rc, done, res = kgs.kgs_iterate(ctx, 1)
            if rc != kgs.KGS_OK:
                raise RuntimeError("kgs_iterate returned %d" % rc)
        ev1.record()
        barrier()
        ms = ev0.elapsed_time(ev1)
        sweep_ms, sweep_launches, launches = kgs.kgs_profile(ctx)
        ms = max_over_ranks(ms, pg, "cuda")
        return ms, sweep_ms, sweep_launches, launches

    # ---- mixed precision (headline) ----
    ctx = kgs.kgs_setup(prob, precision=kgs.KGS_MIXED, v_per_cta=args.v_per_cta, block_z=args.block_z,
                        dev_source=args.dev_source)
    kgs.kgs_set_profiling(ctx, True)
    info = kgs.kgs_info(ctx)
    kgs.kgs_iterate(ctx, args.warmup)
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    ms, sweep_ms, sweep_launches, launches = timed(ctx, args.steps)
    clocks = sampler.stop()
    value = pp * args.steps * world / (ms / 1e3)
    ms_step = ms / args.steps
    sweep_ms_iter = sweep_ms / args.steps
    sm_mhz = peaks.get("sm_max_mhz", 2070.0)
    fp32_peak = SM_COUNT * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12
    achieved = FLOPS_PER_PP * pp / (sweep_ms_iter / 1e3) / 1e12
    # DRAM bytes per launch from an ncu capture of this kernel at 32^3 cells x
    # 32^3 velocities with the same sweep shape, scaled by phase points
    traffic = None
    if TRAFFIC_BYTES_PER_PP and (info["v_per_cta"], info["block_z"]) == TRAFFIC_SHAPE:
        traffic = TRAFFIC_BYTES_PER_PP * pp
    roofline = {"bound": "alu", "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
                "frac": achieved / fp32_peak, "traffic": traffic,
                "kernel": "sweep_persistent_kernel<float>", "flops_per_phase_point": FLOPS_PER_PP,
                "peak_basis": "FP32 FMA lanes: %d SMs x %d lanes x 2 x %.0f MHz (derived)" % (
                    SM_COUNT, FP32_LANES_PER_SM, sm_mhz),
                "sweep_ms_per_step": sweep_ms_iter, "sweep_share_of_step": sweep_ms_iter / ms_step}

    # ---- end to end through the C ABI with pinned host buffers ----
    state_bytes = kgs.kgs_save_size(ctx)
    h_state = torch.empty(state_bytes, dtype=torch.uint8, pin_memory=True)
    h_out = torch.empty(8 * prob.ncell, dtype=torch.float64, pin_memory=True)
    kgs.kgs_save_ptr(ctx, h_state.data_ptr(), state_bytes)
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        kgs.kgs_load_ptr(ctx, h_state.data_ptr(), state_bytes)
        kgs.kgs_iterate(ctx, 1)
        kgs.kgs_moments_ptr(ctx, h_out.data_ptr())
    barrier()
    e2e_s = time.perf_counter() - t0
    e2e = {"value": pp * args.steps * world / e2e_s, "unit": "phase-point updates/s",
           "h2d_bytes_per_step": state_bytes, "d2h_bytes_per_step": 8 * 8 * prob.ncell + 16,
           "api": "kgs_load (state from pinned host) + kgs_iterate(1) + kgs_moments (to pinned host)"}
    del ctx

    # ---- plain FP64 beside it ----
    fp64 = None
    if not args.no_fp64:
        c64 = kgs.kgs_setup(prob, precision=kgs.KGS_FP64, block_z=args.block_z)
        kgs.kgs_set_profiling(c64, True)
        kgs.kgs_iterate(c64, 1)
        k64 = max(1, min(args.steps, 3))
        ms64, sw64, _, _ = timed(c64, k64)
        a64 = FLOPS_PER_PP * pp / (sw64 / k64 / 1e3) / 1e12
        fp64 = {"value": pp * k64 * world / (ms64 / 1e3), "unit": "phase-point updates/s", "steps": k64,
                "ms_per_step": ms64 / k64,
                "roofline": {"bound": "alu", "achieved": a64, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                             "frac": a64 / FP64_PEAK_TFLOPS, "peak_basis": "nominal dense FP64 1.25 TFLOP/s"}}
        del c64
        if rank == 0 and args.cells == N_CELL and args.vels == N_VEL:
            # mixed against FP64 at the full size after two iterations from the
            # uniform start, for both Knudsen numbers of the workload family
            fp64["mixed_vs_fp64_after_2_iterations"] = {}
            for kn in (KN, 0.1):
                pk = inputs.cavity(N_CELL, N_VEL, Kn=kn, lid=LID)
                m = {}
                for prec in (kgs.KGS_FP64, kgs.KGS_MIXED):
                    c = kgs.kgs_setup(pk, precision=prec, block_z=args.block_z)
                    kgs.kgs_iterate(c, 2)
                    m[prec] = kgs.kgs_moments(c)
                    del c
                fp64["mixed_vs_fp64_after_2_iterations"]["Kn=%g" % kn] = rel_errors(m[kgs.KGS_MIXED], m[kgs.KGS_FP64])

    extras = {}
    if not args.no_extras:
        extras = run_extras(args, kgs, inputs, torch, peaks)
        if not args.no_surrogate:
            extras["surrogate"] = run_surrogate(args, kgs, inputs, torch, peaks)
            if args.c5_kn:
                try:
                    extras["time_to_1e-6_128"] = run_config5(args, kgs, inputs, torch)
                except Exception as e:  # noqa: BLE001 - reported in the JSON line
                    extras["time_to_1e-6_128"] = {"error": repr(e)}

    if rank != 0:
        return
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        cpu = time_oracle_sample(kgs)
        cores = os.cpu_count() or 1
        if cores > 1:
            # the same sample on every host core (concurrent velocity ranges)
            try:
                allc = time_oracle_sample(threads=cores)
                if allc["cores"] > 1:
                    cpu["all_cores"] = {"value": allc["value"], "cores": allc["cores"], "sample": allc["sample"]}
            except Exception as e:  # noqa: BLE001 - reported in the JSON line
                cpu["all_cores"] = {"error": repr(e)}
    line = {
        "metric": METRIC, "value": value, "unit": "phase-point updates/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32 sweep / f64 moments", "data": "synthetic",
        "config": {"workload": workload, "cells": prob.ncell, "velocities": prob.nvel,
                   "phase_points_per_step": pp, "precision": "mixed", "v_per_cta": info["v_per_cta"],
                   "block_z": info["block_z"], "sweep_stages": info["n_stages"],
                   "device_bytes": info["device_bytes"],
                   "l2": "working set larger than L2 (face planes and moment partials, %.1f GB)" % (
                       info["device_bytes"] / 1e9),
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
        "clocks": clocks, "fp64": fp64,
    }
    line.update(extras)
    print(json.dumps(line), flush=True)


def run_extras(args, kgs, inputs, torch, peaks):
    """The other workloads of the hot path, measured beside the headline:
    the batched cavities (one persistent sweep launch per outer iteration for
    all instances) and the supersonic flow past a cube (solid mask, free
    stream, stretched velocity grid).  Each is guarded so that a failure is
    reported in the line instead of aborting the benchmark."""
    out = {}
    try:
        probs = inputs.batch_cavities(n=64, seed=0)
        pp = sum(p.phase_points() for p in probs)
        t0 = time.perf_counter()
        b = kgs.kgs_batch_setup(probs, precision=kgs.KGS_MIXED)
        setup_s = time.perf_counter() - t0
        kgs.kgs_batch_iterate(b, 3)
        kgs.kgs_batch_profile(b)
        n_it = args.batch_iters
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rc, done, res = kgs.kgs_batch_iterate(b, n_it)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        sweep_ms, sweeps, launches = kgs.kgs_batch_profile(b)
        info = kgs.kgs_batch_info(b, 0)
        out["batch"] = {
            "workload": "64 cavities (splitmix64 seed 0): Kn log-uniform [0.05,10], lid U[0.05,0.3], "
                        "16-48 cells and 16-32 velocities per side",
            "value": pp * n_it / dt, "unit": "phase-point updates/s", "iterations": n_it,
            "phase_points_per_iteration": pp, "ms_per_iteration": 1e3 * dt / n_it,
            "sweep_ms_per_iteration": sweep_ms / max(sweeps, 1), "rc": rc,
            "shape": {"v_per_cta": info["v_per_cta"], "block_z": info["block_z"], "autotuned": True},
            "setup_s": setup_s, "gpu_launches": launches,
            "roofline_frac": FLOPS_PER_PP * pp / (sweep_ms / max(sweeps, 1) / 1e3) / 1e12 /
                             (SM_COUNT * FP32_LANES_PER_SM * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12),
        }
        del b
    except Exception as e:  # noqa: BLE001 - reported in the JSON line
        out["batch"] = {"error": repr(e)}
    try:
        # the same instances solved to residual 1e-6: mixed iterations per
        # instance while the residual keeps falling, then FP64 from that state
        # (kgs_batch_solve), instances retiring from each batch as they finish
        probs = inputs.batch_cavities(n=64, seed=0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rc, b, nm, nd, res = kgs.kgs_batch_solve(probs, tol=1e-6, max_iters=args.batch_max_iters)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        slow = sorted(range(len(probs)), key=lambda i: -(nm[i] + nd[i]))[:3]
        out["batch_convergence"] = {
            "workload": "the 64 batch cavities solved to residual 1e-6 (kgs_batch_solve: mixed while it makes "
                        "progress, then FP64, per instance)",
            "rc": rc, "seconds": dt, "instances": len(probs), "converged": sum(1 for r in res if r < 1e-6),
            "iterations_mixed": {"median": sorted(nm)[len(nm) // 2], "max": max(nm)},
            "iterations_fp64": {"median": sorted(nd)[len(nd) // 2], "max": max(nd)},
            "slowest": [{"Kn": probs[i].Kn, "cells": probs[i].nx, "vels": len(probs[i].xi_x),
                         "iterations": [nm[i], nd[i]], "residual": res[i]} for i in slow]}
        del b
    except Exception as e:  # noqa: BLE001
        out["batch_convergence"] = {"error": repr(e)}
    try:
        p = inputs.cube()
        pp = p.phase_points()
        c = kgs.kgs_setup(p, precision=kgs.KGS_MIXED)
        kgs.kgs_set_profiling(c, True)
        kgs.kgs_iterate(c, 3)
        kgs.kgs_profile(c)
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        n_it = 3
        ev0.record()
        kgs.kgs_iterate(c, n_it)
        ev1.record()
        torch.cuda.synchronize()
        ms = ev0.elapsed_time(ev1)
        sweep_ms, _, _ = kgs.kgs_profile(c)
        out["cube"] = {
            "workload": "Mach 2 flow past a cube: 96x64x64 cells (cube 16^3 solid), Kn 0.1, "
                        "48^3 stretched velocities on [-8,8]^3",
            "value": pp * n_it / (ms / 1e3), "unit": "phase-point updates/s", "iterations": n_it,
            "phase_points_per_iteration": pp, "ms_per_iteration": ms / n_it,
            "sweep_ms_per_iteration": sweep_ms / n_it,
        }
        del c
    except Exception as e:  # noqa: BLE001
        out["cube"] = {"error": repr(e)}
    try:
        # the first-order sweep with the deviation-form FP32 source (the form
        # the mixed phase of kgs_solve uses on wall-bounded uniform grids)
        p = inputs.cavity(N_CELL, N_VEL, Kn=KN, lid=LID)
        pp = p.phase_points()
        c = kgs.kgs_setup(p, precision=kgs.KGS_MIXED, dev_source=1)
        kgs.kgs_set_profiling(c, True)
        kgs.kgs_iterate(c, 3)
        kgs.kgs_profile(c)
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        n_it = 5
        ev0.record()
        rc, _, _ = kgs.kgs_iterate(c, n_it)
        ev1.record()
        torch.cuda.synchronize()
        ms = ev0.elapsed_time(ev1)
        sweep_ms, _, _ = kgs.kgs_profile(c)
        out["dev_source"] = {
            "workload": WORKLOAD + ", deviation-form FP32 source, mixed",
            "value": pp * n_it / (ms / 1e3), "unit": "phase-point updates/s", "iterations": n_it, "rc": rc,
            "ms_per_iteration": ms / n_it, "sweep_ms_per_iteration": sweep_ms / n_it}
        del c
    except Exception as e:  # noqa: BLE001
        out["dev_source"] = {"error": repr(e)}
    try:
        # the second-order upwind sweep (Section 6's next step) on the
        # headline cavity: two resident slices, 128 velocities per CTA
        p = inputs.cavity(N_CELL, N_VEL, Kn=KN, lid=LID)
        p.order = 2
        pp = p.phase_points()
        c = kgs.kgs_setup(p, precision=kgs.KGS_MIXED)
        kgs.kgs_set_profiling(c, True)
        kgs.kgs_iterate(c, 3)
        kgs.kgs_profile(c)
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        n_it = 5
        ev0.record()
        rc, _, _ = kgs.kgs_iterate(c, n_it)
        ev1.record()
        torch.cuda.synchronize()
        ms = ev0.elapsed_time(ev1)
        sweep_ms, _, _ = kgs.kgs_profile(c)
        tflops = FLOPS_PER_PP_ORDER2 * pp / (sweep_ms / n_it / 1e3) / 1e12
        peak = SM_COUNT * FP32_LANES_PER_SM * 2 * 2070e6 / 1e12
        out["order2"] = {
            "workload": WORKLOAD + ", second-order upwind sweep, mixed",
            "value": pp * n_it / (ms / 1e3), "unit": "phase-point updates/s", "iterations": n_it, "rc": rc,
            "ms_per_iteration": ms / n_it, "sweep_ms_per_iteration": sweep_ms / n_it,
            "roofline": {"bound": "alu", "achieved": tflops, "peak": peak, "unit": "TFLOP/s",
                         "frac": tflops / peak, "flops_per_phase_point": FLOPS_PER_PP_ORDER2},
            "device_bytes": kgs.kgs_info(c)["device_bytes"]}
        del c
    except Exception as e:  # noqa: BLE001
        out["order2"] = {"error": repr(e)}
    if args.paper_cube:
        try:
            # the cube on the paper's stretched mesh (Section 4.2): per-cell
            # upwind coefficients, 6.9e11 phase points per iteration
            p = inputs.cube_paper_mesh()
            pp = p.phase_points()
            t0 = time.perf_counter()
            c = kgs.kgs_setup(p, precision=kgs.KGS_MIXED)
            setup_s = time.perf_counter() - t0
            kgs.kgs_set_profiling(c, True)
            kgs.kgs_iterate(c, 1)
            kgs.kgs_profile(c)
            torch.cuda.synchronize()
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            n_it = 2
            ev0.record()
            rc, _, res = kgs.kgs_iterate(c, n_it)
            ev1.record()
            torch.cuda.synchronize()
            ms = ev0.elapsed_time(ev1)
            sweep_ms, _, _ = kgs.kgs_profile(c)
            out["cube_paper_mesh"] = {
                "workload": "Mach 2 flow past a unit cube, %dx%dx%d stretched cells (ratios 1.02 / 1.03), Kn 1, "
                            "48^3 uniform velocities on [-4,4]^3, mixed" % (p.nx, p.ny, p.nz),
                "value": pp * n_it / (ms / 1e3), "unit": "phase-point updates/s", "iterations": n_it,
                "phase_points_per_iteration": pp, "ms_per_iteration": ms / n_it,
                "sweep_ms_per_iteration": sweep_ms / n_it, "setup_s": setup_s, "rc": rc,
                "device_bytes": kgs.kgs_info(c)["device_bytes"]}
            del c
        except Exception as e:  # noqa: BLE001
            out["cube_paper_mesh"] = {"error": repr(e)}
    return out


def run_surrogate(args, kgs, inputs, torch, peaks):
    """The learned initial guess: tensor-core throughput of the network's
    forward pass at 128^3 voxels and of a training step, then the time to a
    residual of 1e-6 on held-out cavities from the uniform state (FP64, and
    mixed then FP64) and from the network's guess (coarse solve, inference and
    fine solve all counted)."""
    import numpy as np

    from paper_1810_00348_gb300 import surrogate
    out = {}
    bf16_peak = float(peaks.get("bf16_tflops", 1900.0))
    ch = surrogate.DEFAULT_CHANNELS
    flops_per_voxel = 2.0 * 27 * sum(a * b for a, b in zip(ch[:-1], ch[1:]))
    s = surrogate.Surrogate(seed=0)

    def ev_time(fn, reps):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    try:
        shape = (1, 128, 128, 128)
        x = torch.randn(shape + (surrogate.N_FEATURES,), device="cuda")
        y = torch.empty(shape + (surrogate.N_FIELDS,), device="cuda")
        ms = ev_time(lambda: kgs.kgs_net_forward(s.net, x.data_ptr(), shape, y.data_ptr()), 5)
        tf = flops_per_voxel * np.prod(shape) / (ms / 1e3) / 1e12
        out["inference"] = {"workload": "forward pass, 1 x 128^3 voxels, channels %s" % "-".join(map(str, ch)),
                            "ms": ms, "tflops": tf,
                            "roofline": {"bound": "tensor", "achieved": tf, "peak": bf16_peak, "unit": "TFLOP/s",
                                         "frac": tf / bf16_peak, "peak_basis": "measured bf16 GEMM burst"}}
        shape = (8, 32, 32, 32)
        x = torch.randn(shape + (surrogate.N_FEATURES,), device="cuda")
        t = torch.randn(shape + (surrogate.N_FIELDS,), device="cuda")
        ms = ev_time(lambda: kgs.kgs_net_train_step(s.net, x.data_ptr(), t.data_ptr(), None, shape, 1e-5), 3)
        tf = 3 * flops_per_voxel * np.prod(shape) / (ms / 1e3) / 1e12
        out["training_step"] = {"workload": "forward + backward + Adam, 8 x 32^3 voxels", "ms": ms, "tflops": tf,
                                "roofline_frac": tf / bf16_peak}
        del x, t, y
    except Exception as e:  # noqa: BLE001
        out["throughput_error"] = repr(e)
    try:
        cells, vels, tol = args.surrogate_cells, 16, 1e-6
        t0 = time.perf_counter()
        train = surrogate.draw_cavities(args.surrogate_train, seed=1, cells=cells, vels=vels)
        samples = surrogate.make_samples(train, precision=kgs.KGS_FP64, tol=tol, max_iters=5000)
        t_data = time.perf_counter() - t0
        t0 = time.perf_counter()
        losses = s.train(samples, steps=400, batch=8, lr=1e-3, seed=0)
        torch.cuda.synchronize()
        t_train = time.perf_counter() - t0
        cases = []
        for p in surrogate.draw_cavities(4, seed=2, cells=cells, vels=vels):
            n_fp64, t_fp64, r_fp64, _ = surrogate.iterations_to(p, None, kgs.KGS_FP64, tol, 5000)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            rc_m, _, nm, nd, r_m = kgs.kgs_solve(p, None, tol, 5000)
            t_mixed = time.perf_counter() - t0
            t0 = time.perf_counter()
            coarse = surrogate.coarse_solution(p)
            guess, n_bad = s.guess(p, coarse)
            rc_s, _, sm, sd, r_s = kgs.kgs_solve(p, guess, tol, 5000)
            torch.cuda.synchronize()
            t_sur = time.perf_counter() - t0
            cases.append({"Kn": p.Kn, "lid": surrogate.lid_speed(p),
                          "fp64_uniform": {"iterations": n_fp64, "s": t_fp64, "residual": r_fp64},
                          "mixed_fp64_uniform": {"iterations": [nm, nd], "s": t_mixed, "residual": r_m},
                          "mixed_fp64_surrogate": {"iterations": [sm, sd], "s": t_sur, "residual": r_s,
                                                   "guess_rejected": guess is None,
                                                   "includes": "mixed coarse solve to 1e-4, inference, fine solve"}})
        out["time_to_1e-6"] = {
            "workload": "held-out lid-driven cavities (splitmix64 seed 2): %d^3 cells x %d^3 velocities, "
                        "Kn log-uniform [0.05,0.5], lid U[0.05,0.3]; coarse grid %d^3" % (cells, vels, cells // 2),
            "training": {"samples": len(samples), "steps": 400, "batch": 8, "data_s": t_data, "train_s": t_train,
                         "loss_first": float(np.mean(losses[:10])), "loss_last": float(np.mean(losses[-10:]))},
            "cases": cases,
            "speedup_vs_fp64": float(np.mean([c["fp64_uniform"]["s"] / c["mixed_fp64_surrogate"]["s"]
                                              for c in cases])),
        }
    except Exception as e:  # noqa: BLE001
        out["time_to_1e-6"] = {"error": repr(e)}
    return out


def run_config5(args, kgs, inputs, torch):
    """Time to residual 1e-6 on the surrogate-started cavity: 128^3 cells x
    32^3 velocities, lid 0.16, for each Knudsen number of --c5-kn, from four
    starts -- the uniform state in plain FP64; the uniform state, mixed then
    FP64 (kgs_solve); the upsampled coarse solution without the network; the
    network's guess -- where the last two count the coarse solve (mixed, to
    1e-4, on the grid twice as coarse) and, for the guess, the inference.
    The network (channels 11-48-112-112-112-48-8) is first trained on
    --c5-train solver-generated cavities of 16^3 cells x 16^3 velocities (Kn
    log-uniform [0.05, 0.5], lid U[0.05, 0.3], FP64 solves to 1e-6)."""
    from paper_1810_00348_gb300 import surrogate
    tol = 1e-6
    out = {"workload": "lid-driven cavity %d^3 cells x %d^3 velocities, lid 0.16, time to residual 1e-6"
                       % (args.c5_cells, args.c5_vels)}
    t0 = time.perf_counter()
    train = surrogate.draw_cavities(args.c5_train, seed=1, cells=16, vels=16)
    samples = surrogate.make_samples(train, precision=kgs.KGS_FP64, tol=tol, max_iters=5000)
    t_data = time.perf_counter() - t0
    s = surrogate.Surrogate(seed=0)
    t0 = time.perf_counter()
    losses = s.train(samples, steps=args.c5_steps, batch=16, lr=1e-3, seed=0)
    torch.cuda.synchronize()
    out["training"] = {"samples": len(samples), "cells": 16, "vels": 16, "steps": args.c5_steps,
                       "data_s": t_data, "train_s": time.perf_counter() - t0,
                       "loss_first": float(np.mean(losses[:20])), "loss_last": float(np.mean(losses[-20:]))}
    if args.only_c5:
        print(json.dumps({"training": out["training"]}), flush=True)
    cases = []
    for kn in [float(v) for v in args.c5_kn.split(",") if v]:
        p = inputs.cavity(args.c5_cells, args.c5_vels, Kn=kn, lid=LID)
        case = {"Kn": kn}
        if args.c5_fp64:
            n, dt, r, rc = surrogate.iterations_to(p, None, kgs.KGS_FP64, tol, args.c5_max_iters)
            case["fp64_uniform"] = {"iterations": n, "s": dt, "residual": r, "rc": rc}
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        rc, _, nm, nd, r = kgs.kgs_solve(p, None, tol, args.c5_max_iters)
        case["mixed_fp64_uniform"] = {"iterations": [nm, nd], "s": time.perf_counter() - t1, "residual": r, "rc": rc}
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        coarse = surrogate.coarse_solution(p)
        t_coarse = time.perf_counter() - t1
        _, up = surrogate.upsample(p, coarse)
        up = up.cpu().numpy()
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        rc, _, nm, nd, r = kgs.kgs_solve(p, up, tol, args.c5_max_iters)
        case["mixed_fp64_upsampled_coarse"] = {"iterations": [nm, nd], "s": t_coarse + time.perf_counter() - t1,
                                               "coarse_s": t_coarse, "residual": r, "rc": rc}
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        guess, n_bad = s.guess(p, coarse)
        rc, _, nm, nd, r = kgs.kgs_solve(p, guess, tol, args.c5_max_iters)
        case["mixed_fp64_network"] = {"iterations": [nm, nd], "s": t_coarse + time.perf_counter() - t1,
                                      "coarse_s": t_coarse, "residual": r, "rc": rc, "guess_rejected": guess is None}
        case["network_gain_over_upsampled_s"] = case["mixed_fp64_upsampled_coarse"]["s"] - \
            case["mixed_fp64_network"]["s"]
        cases.append(case)
        if args.only_c5:
            print(json.dumps({"case": case}), flush=True)  # each case as it completes
    out["cases"] = cases
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--v-per-cta", type=int, default=0)
    ap.add_argument("--block-z", type=int, default=0)
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the batched and cube workloads")
    ap.add_argument("--batch-iters", type=int, default=20)
    ap.add_argument("--batch-max-iters", type=int, default=3000, help="iteration budget per instance of the 1e-6 solve")
    ap.add_argument("--paper-cube", type=int, default=1, help="time the cube on the paper's 181x181x191 mesh")
    ap.add_argument("--no-surrogate", action="store_true", help="skip the learned-initial-guess measurements")
    ap.add_argument("--surrogate-cells", type=int, default=16, help="cells per side of the gain cavities")
    ap.add_argument("--surrogate-train", type=int, default=48, help="training cavities")
    ap.add_argument("--c5-kn", default="0.5", help="Knudsen numbers of the 128^3 time-to-1e-6 study (empty: skip)")
    ap.add_argument("--only-c5", action="store_true", help="run only the time-to-1e-6 study and print its JSON")
    ap.add_argument("--c5-cells", type=int, default=128)
    ap.add_argument("--c5-vels", type=int, default=32)
    ap.add_argument("--c5-train", type=int, default=512, help="training cavities of the study's network")
    ap.add_argument("--c5-steps", type=int, default=3000, help="training steps of the study's network")
    ap.add_argument("--c5-max-iters", type=int, default=1000)
    ap.add_argument("--c5-fp64", type=int, default=1, help="also time the plain FP64 solve from the uniform state")
    ap.add_argument("--cells", type=int, default=N_CELL, help="cells per side (profiling runs only)")
    ap.add_argument("--vels", type=int, default=N_VEL, help="velocities per side (profiling runs only)")
    ap.add_argument("--dev-source", type=int, default=0,
                    help="1: the headline leg with the deviation-form FP32 source (profiling runs only)")
    args = ap.parse_args()
    world, rank, local = dist_env()
    if args.only_c5:
        import torch

        from paper_1810_00348_gb300 import inputs, kgs
        kgs.load()
        print(json.dumps(run_config5(args, kgs, inputs, torch)), flush=True)
        return
    if args.impl == "reference":
        run_reference(args, world, rank)
    else:
        run_ours(args, world, rank, local)


if __name__ == "__main__":
    main()
