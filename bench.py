"""Benchmark of the stochastic-Galerkin slab operator apply (sg_apply).

One step = one application y = A^(n) x of the SG slab operator
(eq. local_rhs_tensor) to one slab vector, on the 2D 64x64 Q2, dG(1),
M=4 / P=3 (35 chaos modes) workload: 16,641 nodes x 2 time nodes x 35 modes =
1,164,870 unknowns.  Metric: GDoF*modes/s = unknowns x applies / s / 1e9.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 runs under torchrun, one process per GPU; every rank applies the
operator to its own replica of the workload (the apply has no exchange step
on one node), value = all ranks' unknowns / max-over-ranks time ("weak").
The reference arm times the CPU oracle (oracle/, FP64 numpy/scipy) on the
host cores, rank 0 only.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "SG operator applies"
UNIT = "GDoF*modes/s"
# FP64 FMA peak: SMs x 2 FP64 FMA lanes per SM per clock x 2 flop x maximum SM
# clock; on GB300 152 SMs at 2070 MHz give 1.259 TFLOP/s.  fp64_peak_tflops()
# reads the SM count and the maximum clock of the device that runs the bench.
FP64_FMA_PER_SM_CLOCK = 2
FP64_PEAK_TFLOPS = 152 * FP64_FMA_PER_SM_CLOCK * 2 * 2.070e9 / 1e12


# FP32 FMA lanes per SM per clock (the FP32 pipe) and FP32 instructions one
# double-word multiply-add takes (product with its exact error, TwoSum, two adds)
FP32_FMA_PER_SM_CLOCK = 128
DW_FP32_INSTR_PER_FMA = 12


def fp32_peak_tflops(sm_max_mhz=None):
    """FP32 FMA peak of cuda:0: SMs x 128 lanes x 2 flop x maximum SM clock."""
    try:
        import torch
        n_sm = torch.cuda.get_device_properties(0).multi_processor_count
    except Exception:
        n_sm = 152
    mhz = sm_max_mhz or peaks().get("sm_max_mhz") or 2070.0
    return n_sm * FP32_FMA_PER_SM_CLOCK * 2 * float(mhz) * 1e6 / 1e12


def fp64_peak_tflops(sm_max_mhz=None):
    """The FP64 FMA peak of cuda:0 (SM count from the device, the maximum SM
    clock sampled by nvidia-smi when given, else MEASURED_PEAKS.json's)."""
    global FP64_PEAK_TFLOPS
    try:
        import torch
        n_sm = torch.cuda.get_device_properties(0).multi_processor_count
    except Exception:
        return FP64_PEAK_TFLOPS
    mhz = sm_max_mhz or peaks().get("sm_max_mhz") or 2070.0
    FP64_PEAK_TFLOPS = n_sm * FP64_FMA_PER_SM_CLOCK * 2 * float(mhz) * 1e6 / 1e12
    return FP64_PEAK_TFLOPS
# algorithmic work of the sum-factorised apply per unknown (FP64 flop) and
# the algorithmic HBM bytes per unknown (read x, write y once)
FLOP_PER_UNKNOWN = 166.0
BYTES_PER_UNKNOWN = 16.0
L2_BYTES = 135_528_448
# V-cycle smoothing used by the solve measurements: one pre- and one
# post-smoothing Vanka step with damping 0.9 reaches 1e-8 fastest on GB300
# (2D: 9 iterations, 8.3 ms vs 8 iterations, 10.2 ms with nu = 2, omega = 0.7)
MG_NU, MG_OMEGA = 1, 0.9
# dram__bytes_read.sum + dram__bytes_write.sum of one FP64 chunk-kernel launch on
# this workload (ncu capture summarised in profiles/); None once the kernel changes
NCU_TRAFFIC_BYTES = 19_920_640 + 0


def workload():
    from paper_2605_21046_gb300 import inputs
    return inputs.config_2d_q2_64()


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {"hbm_gbs": 6800.0, "fallback": True}


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        if self.gpu < 0:
            return self
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
            time.sleep(0.3)
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

    def summary(self):
        rows = []
        try:
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        except Exception:
            pass
        finally:
            try:
                os.unlink(self.path)
            except Exception:
                pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows)}


def dist_init():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(v, world):
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    dev = "cuda" if torch.cuda.is_available() and dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def oracle_apply_rate(spec, budget_s=15.0, min_reps=1):
    """Times the oracle's Kronecker-sum apply (set-up excluded) for about
    budget_s seconds; returns (unknowns/s, reps, wall, cores used)."""
    import numpy as np
    from oracle import operator
    from paper_2605_21046_gb300 import inputs
    p = operator.SGProblem(spec)
    x = inputs.random_vector(spec)
    p.apply(x)  # warm
    reps, t0, c0 = 0, time.perf_counter(), time.process_time()
    while True:
        p.apply(x)
        reps += 1
        el = time.perf_counter() - t0
        if reps >= min_reps and el > budget_s:
            break
        if el > budget_s and reps >= 1:
            break
    wall = time.perf_counter() - t0
    cpu = time.process_time() - c0
    n = inputs.n_unknowns(spec)
    return n * reps / wall, reps, wall, max(1, round(cpu / wall))


def _oracle_rate_worker(args):
    """One process of the all-cores oracle timing (spawned; CPU only)."""
    spec, budget = args
    return oracle_apply_rate(spec, budget_s=budget)


def oracle_apply_rate_all_cores(spec, budget_s=10.0, procs=None):
    """The oracle's apply, as it stands, run as independent applies in one
    process per host core at the same time: (unknowns/s summed, processes)."""
    import multiprocessing as mp
    from concurrent.futures import ProcessPoolExecutor
    procs = procs or os.cpu_count() or 1
    # spawn: the parent already holds a CUDA context; a dead worker raises
    # (BrokenProcessPool) instead of leaving the pool waiting
    with ProcessPoolExecutor(max_workers=procs, mp_context=mp.get_context("spawn")) as ex:
        futs = [ex.submit(_oracle_rate_worker, (spec, budget_s)) for _ in range(procs)]
        res = [f.result(timeout=budget_s + 300) for f in futs]
    return sum(r[0] for r in res), procs


def oracle_solve_ms(spec, rtol=1e-8):
    """The oracle's slab solve (FGMRES, exact block-Jacobi LU) of one seeded
    right-hand side: (wall ms including the factorisation, iterations)."""
    from oracle import operator, solver
    from paper_2605_21046_gb300 import inputs
    t0 = time.perf_counter()
    p = operator.SGProblem(spec)
    pre = solver.BlockJacobiLU(p)
    b = inputs.random_rhs(spec)
    _, its, _ = solver.fgmres(p, b, pre.apply, rtol=rtol)
    return 1e3 * (time.perf_counter() - t0), its


def run_reference(args, world, rank):
    """The reference arm: the oracle's apply (numpy/scipy FP64) on the host
    cores, rank 0 only.  Each step is a bounded sample of the workload: the
    apply restricted to a contiguous block of spatial node rows (every chaos
    mode and time node), sized from one untimed full apply so that the W + K
    steps take about --ref-seconds; the whole apply when it fits."""
    spec = workload()
    from paper_2605_21046_gb300 import inputs
    if rank != 0:
        return
    import numpy as np
    from oracle import operator
    p = operator.SGProblem(spec)
    x = inputs.random_vector(spec)
    t0 = time.perf_counter()
    p.apply(x)
    t_full = time.perf_counter() - t0
    total = args.warmup + args.steps
    n_rows = int(min(p.n_x, max(1, p.n_x * args.ref_seconds / (total * t_full))))
    lo = (p.n_x - n_rows) // 2
    rows = np.arange(lo, lo + n_rows)
    step = (lambda: p.apply(x)) if n_rows == p.n_x else (lambda: p.apply_node_rows(x, rows))
    per_step = []
    c0, w0 = time.process_time(), time.perf_counter()
    for s in range(total):
        t0 = time.perf_counter()
        step()
        if s >= args.warmup:
            per_step.append(time.perf_counter() - t0)
    cores = max(1, round((time.process_time() - c0) / (time.perf_counter() - w0)))
    n = inputs.n_unknowns(spec)
    n_step = p.n_xi * p.n_t * n_rows
    t = sum(per_step)
    value = n_step * len(per_step) / t / 1e9
    sample = (f"{len(per_step)} full oracle applies of the {n}-unknown workload" if n_rows == p.n_x else
              f"{len(per_step)} steps, each the oracle apply restricted to {n_rows} of the {p.n_x} spatial "
              f"node rows ({n_step} of {n} unknowns; a full apply took {t_full:.2f} s)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / len(per_step),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": spec["name"], "unknowns": n, "mesh": "64x64 Q2 unit square",
                                            "time": "dG(1)", "M": 4, "P": 3, "chaos_modes": 35},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def time_applies(sg, torch, ctx, X, Y, steps, warmup, stream, world, sample_clocks, local, profile_range=False):
    """Device time of `steps` applies over rotating buffers; returns
    (elapsed_ms max over ranks, mean per-launch seconds, clocks).  With
    profile_range the timed launches are bracketed by cudaProfilerStart/Stop
    (for ncu --profile-from-start off)."""
    R = len(X)
    for s in range(warmup):
        sg.sg_apply(ctx, 0, X[s % R], Y[s % R], False, stream)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    with ClockSampler(local if sample_clocks else -1) as clk:
        barrier(world)
        torch.cuda.synchronize()
        t_start = torch.cuda.Event(enable_timing=True)
        t_end = torch.cuda.Event(enable_timing=True)
        if profile_range:
            torch.cuda.profiler.start()
        t_start.record(stream)
        for s in range(steps):
            ev[s][0].record(stream)
            sg.sg_apply(ctx, 0, X[s % R], Y[s % R], False, stream)
            ev[s][1].record(stream)
        t_end.record(stream)
        torch.cuda.synchronize()
        if profile_range:
            torch.cuda.profiler.stop()
        barrier(world)
    clocks = clk.summary() if sample_clocks else None
    elapsed_ms = max_over_ranks(t_start.elapsed_time(t_end), world)
    t_launch = statistics.mean(a.elapsed_time(b) for a, b in ev) / 1e3
    return elapsed_ms, t_launch, clocks


def measure_solve(sg, torch, spec, dev, reps=3, autotune=True, profile=None):
    """Time to a 1e-8 relative residual for one slab system, FGMRES(30) from a
    zero initial guess, for the precision splits.  profile names a split one
    more solve of which is bracketed by cudaProfilerStart/Stop."""
    from paper_2605_21046_gb300 import inputs
    b = torch.from_numpy(inputs.random_rhs(spec)).to(dev)
    out, ref = {}, None
    for name, apply_prec, mg_prec in (("fp64", sg.SG_PREC_FP64, sg.SG_PREC_FP64),
                                      ("fp32_mg", sg.SG_PREC_FP64, sg.SG_PREC_FP32),
                                      ("bf16_factors_mg", sg.SG_PREC_FP64, sg.SG_PREC_BF16),
                                      ("fp32_mg_dw_apply", sg.SG_PREC_DW, sg.SG_PREC_FP32)):
        ctx = sg.sg_setup_spec(spec, apply_prec)
        if autotune:
            sg.sg_autotune(ctx, reps=5)
        sg.sg_mg_setup(ctx, mg_prec, MG_NU, MG_OMEGA)
        x = torch.zeros_like(b)
        st = sg.sg_solve_slab(ctx, 0, b, x, rtol=1e-8)          # warm-up, records the V-cycle graph
        times = []
        for _ in range(reps):
            x.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            st = sg.sg_solve_slab(ctx, 0, b, x, rtol=1e-8)
            torch.cuda.synchronize()
            times.append(1e3 * (time.perf_counter() - t0))
        if profile == name:
            x.zero_()
            torch.cuda.synchronize()
            torch.cuda.profiler.start()
            sg.sg_solve_slab(ctx, 0, b, x, rtol=1e-8)
            torch.cuda.synchronize()
            torch.cuda.profiler.stop()
        if ref is None:
            ref = x.clone()
        err = float((x - ref).abs().max() / ref.abs().max())
        out[name] = {"ms_per_slab": statistics.median(times), "iterations": st["iterations"],
                     "rel_residual": st["rel_residual"], "max_rel_diff_vs_fp64_solution": err,
                     "mg_setup_ms": st["mg_setup_ms"]}
        ctx.destroy()
    return {"metric": "time to 1e-8 relative residual per slab", "unit": "ms",
            "solver": f"FGMRES(30), block-Jacobi GMG V-cycle (Vanka, nu={MG_NU}, omega={MG_OMEGA})", "splits": out}


def next_summary(rows):
    """The NEXT rows' headline figures, compact (the line's last key, so that a
    reader keeping only the end of the output still has them)."""
    if not rows:
        return None
    out = {}
    mp = rows.get("mixed_precision")
    if mp:
        sp = mp["splits"]
        out["mixed_3d_q2_32^3_M3P3_20slabs"] = {
            k: {"ms_per_slab": round(v["ms_per_slab"], 2), "setup_ms": round(v["mg_setup_ms"], 1),
                "ratio_vs_fp64_with_setup": round(v["time_ratio_vs_fp64_with_setup"], 3),
                "rel_diff_vs_fp64": float("%.2g" % v["max_rel_diff_vs_fp64"]),
                "its": v["iterations_mean"]} for k, v in sp.items()}
    mc = rows.get("mc_vs_sg")
    if mc:
        out["mc_vs_sg_4096_samples_50slabs"] = {
            "mc_s": round(mc["mc"]["ms"] / 1e3, 2), "sg_s": round(mc["sg_ms_both_meshes"] / 1e3, 3),
            "mc_err_mean_var": {k: [float("%.3g" % v["mc_error_mean_L2"]), float("%.3g" % v["mc_error_var_L2"])]
                                for k, v in mc["meshes"].items()},
            "sg_err_mean_var": {k: [float("%.3g" % v["sg_error_mean_L2"]), float("%.3g" % v["sg_error_var_L2"])]
                                for k, v in mc["meshes"].items()}}
    ad = rows.get("adjoint")
    if ad:
        out["adjoint_128^2_q2_M4P4_50slabs"] = {
            "grad_s": round(ad["grad_ms"] / 1e3, 2), "grad_over_forward": round(ad["grad_over_forward"], 2),
            "fd_rel_diff": {k: float("%.2g" % v["rel_diff"]) for k, v in ad["fd_checks"].items()}}
    return out


def run_ours(args, world, rank, local):
    import torch
    import paper_2605_21046_gb300 as sg
    from paper_2605_21046_gb300 import build, inputs
    build.build()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    spec = workload()
    ctx = sg.sg_setup_spec(spec, sg.SG_PREC_FP64)
    if not args.no_autotune:
        sg.sg_autotune(ctx, reps=10)
    n = ctx.info["n_unknowns"]
    # rotating x/y pairs whose total exceeds L2, so no step reads another's cache
    vec_bytes = 8 * n
    R = max(2, math.ceil(2.2 * L2_BYTES / (2 * vec_bytes)))
    gen = torch.Generator(device=dev)
    gen.manual_seed(inputs.SEED_X + rank)
    X = [torch.rand(n, dtype=torch.float64, device=dev, generator=gen) * 2 - 1 for _ in range(R)]
    Y = [torch.empty(n, dtype=torch.float64, device=dev) for _ in range(R)]
    stream = torch.cuda.current_stream(dev)
    elapsed_ms, t_launch, clocks = time_applies(sg, torch, ctx, X, Y, args.steps, args.warmup, stream,
                                                world, True, local,
                                                profile_range=args.profile_range and args.profile_variant == "fp64")
    fp64_peak_tflops((clocks or {}).get("sm_max_mhz"))
    value = world * n * args.steps / (elapsed_ms / 1e3) / 1e9
    assert torch.isfinite(Y[0]).all()
    y64 = Y[0].clone()

    # double-word variant (same tolerance), reported beside the FP64 headline
    dw = None
    if not args.no_dw:
        ctx_dw = sg.sg_setup_spec(spec, sg.SG_PREC_DW)
        if not args.no_autotune:
            sg.sg_autotune(ctx_dw, reps=10)
        e_dw, t_dw, _ = time_applies(sg, torch, ctx_dw, X, Y, args.steps, args.warmup, stream, world, False, local,
                                     profile_range=args.profile_range and args.profile_variant == "dw")
        sg.sg_apply(ctx_dw, 0, X[0], Y[0], False, stream)
        torch.cuda.synchronize()
        err = float((Y[0] - y64).abs().max() / y64.abs().max())
        v_dw = world * n * args.steps / (e_dw / 1e3) / 1e9
        dw = {"value": v_dw, "unit": UNIT, "ms_per_step": e_dw / args.steps, "dtype": "f32x2 double-word",
              "speedup_vs_fp64": v_dw / value, "max_rel_diff_vs_fp64": err,
              "fp64_equivalent_tflops": FLOP_PER_UNKNOWN * n / t_dw / 1e12,
              "gpu_launches": 2 * args.steps,
              "launch": {"chunk_cells": ctx_dw.info["chunk"], "grid": ctx_dw.info["grid"],
                         "threads": ctx_dw.info["threads"], "stagger": ctx_dw.info["stagger"]}}
        ctx_dw.destroy()

    # the same applies on one x/y pair (x, y and the tables stay in L2)
    e_hot, t_hot, _ = time_applies(sg, torch, ctx, X[:1], Y[:1], args.steps, args.warmup, stream, world, False, local)
    hot = {"value": world * n * args.steps / (e_hot / 1e3) / 1e9, "unit": UNIT,
           "ms_per_step": e_hot / args.steps, "l2": "one x/y pair, L2-resident",
           "fp64_tflops": FLOP_PER_UNKNOWN * n / t_hot / 1e12}

    solve = None if args.no_solve else measure_solve(sg, torch, spec, dev, autotune=not args.no_autotune,
                                                     profile=args.profile_solve)

    # end to end through the host-buffer entry points, every step copying its
    # x in from pinned host memory and its y back: the pipelined call (two
    # host buffer pairs in turn, one synchronize at the end) and the
    # synchronous one
    xh = [X[i].cpu().pin_memory() for i in range(2)]
    yh = [torch.empty_like(xh[0]).pin_memory() for _ in range(2)]
    k_e2e = max(3, min(args.steps, 200))
    side = torch.cuda.Stream(dev)
    for k in range(4):
        sg.sg_apply_host_async(ctx, 0, xh[k % 2], yh[k % 2], stream=side)
    side.synchronize()
    barrier(world)
    t0 = time.perf_counter()
    for k in range(k_e2e):
        sg.sg_apply_host_async(ctx, 0, xh[k % 2], yh[k % 2], stream=side)
    side.synchronize()
    e2e_s = max_over_ranks(time.perf_counter() - t0, world)
    e2e = world * n * k_e2e / e2e_s / 1e9
    assert torch.isfinite(yh[0]).all() and torch.isfinite(yh[1]).all()
    for _ in range(3):
        sg.sg_apply_host(ctx, 0, xh[0], yh[0])
    barrier(world)
    t0 = time.perf_counter()
    for _ in range(k_e2e):
        sg.sg_apply_host(ctx, 0, xh[0], yh[0])
    e2e_sync = world * n * k_e2e / max_over_ranks(time.perf_counter() - t0, world) / 1e9

    # the NEXT rows on their own workloads (single-GPU runs only)
    next_rows = None
    if world == 1 and not args.no_next:
        next_rows = {}
        for key, fn in (("mixed_precision", next_mixed_precision), ("mc_vs_sg", next_mc_vs_sg),
                        ("adjoint", next_adjoint)):
            t0 = time.perf_counter()
            next_rows[key] = fn(sg, torch, inputs)
            next_rows[key]["wall_s"] = time.perf_counter() - t0
            torch.cuda.empty_cache()

    pk = peaks()
    achieved_tf = FLOP_PER_UNKNOWN * n / t_launch / 1e12
    hbm_gbs = BYTES_PER_UNKNOWN * n / t_launch / 1e9
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        rate, reps, wall, cores = oracle_apply_rate(spec, budget_s=args.cpu_seconds)
        cpu = {"value": rate / 1e9, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"{reps} full oracle applies of the {n}-unknown workload in {wall:.1f} s"}
        if not args.no_cpu_all_cores:
            rate_all, procs = oracle_apply_rate_all_cores(spec, budget_s=min(args.cpu_seconds, 10.0))
            cpu["all_cores"] = {"value": rate_all / 1e9, "unit": UNIT, "processes": procs,
                                "sample": "one process per host core, each timing full oracle applies for 10 s"}
        if solve is not None:
            for name, sp in (("2d-q1-8x8-M2P2", inputs.config_small_2d_q1()), (spec["name"], spec)):
                ms, its = oracle_solve_ms(sp)
                solve.setdefault("cpu_oracle", {})[name] = {
                    "ms_per_slab": ms, "iterations": its, "cores": 1,
                    "solver": "oracle FGMRES(30) + exact block-Jacobi sparse LU, factorisation included"}
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": elapsed_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": spec["name"], "unknowns": n, "mesh": "64x64 Q2 unit square",
                       "time": "dG(1)", "M": 4, "P": 3, "chaos_modes": 35,
                       "l2": f"{R} rotating x/y pairs, {2 * R * vec_bytes / 1e6:.0f} MB > {L2_BYTES / 1e6:.0f} MB L2",
                       "parallelism": f"replicas x{world}",
                       "chunk_cells": ctx.info["chunk"], "grid": ctx.info["grid"],
                       "threads": ctx.info["threads"], "stagger": ctx.info["stagger"]},
            "gpu_launches": 2 * args.steps,
            "clocks": clocks,
            "e2e": {"value": e2e, "unit": UNIT, "h2d_bytes_per_step": vec_bytes, "d2h_bytes_per_step": vec_bytes,
                    "api": "sg_apply_host_async (pipelined, pinned host buffers, synchronized at the end)",
                    "synchronous": {"value": e2e_sync, "api": "sg_apply_host (returns when y is on the host)"}},
            "roofline": {"bound": "alu", "achieved": achieved_tf, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                         "frac": achieved_tf / FP64_PEAK_TFLOPS, "traffic": NCU_TRAFFIC_BYTES,
                         "kernel": "sg_apply (init + chunk kernel, per-launch CUDA events)",
                         "hbm": {"achieved": hbm_gbs, "peak": pk.get("hbm_gbs"), "unit": "GB/s",
                                 "frac": hbm_gbs / pk.get("hbm_gbs", 6800.0)}},
            "cpu_baseline": cpu,
            "variants": {"dw": dw, "l2_hot": hot},
            "solve": solve,
            "next_detail": next_rows,
            "next": next_summary(next_rows),
        }
        if dw is not None:
            # the double-word apply runs on the FP32 pipe: 12 FP32 instructions per
            # FP64-equivalent multiply-add, so its ceiling is the FP32 FMA peak / 12
            fp32_peak = fp32_peak_tflops((clocks or {}).get("sm_max_mhz"))
            dw_tf = dw["fp64_equivalent_tflops"]
            line["roofline"]["dw"] = {"bound": "alu", "achieved": dw_tf, "peak": fp32_peak / DW_FP32_INSTR_PER_FMA,
                                      "unit": "TFLOP/s (FP64-equivalent)",
                                      "frac": dw_tf / (fp32_peak / DW_FP32_INSTR_PER_FMA),
                                      "fp32_fma_peak_tflops": fp32_peak,
                                      "fp32_instr_per_fp64_fma": DW_FP32_INSTR_PER_FMA}
        print(json.dumps(line), flush=True)
    ctx.destroy()


# ---------------------------------------------------------------- NEXT rows
# ``--suite next`` measures the solver-side rows on their own workloads and
# prints one JSON line per row: the mixed-precision 3D solve, batched
# Monte-Carlo against SG on the same GPU, and the adjoint gradient.

def exact_for(sg, M, q, dim, eta=0.35, T=(0.0, 1.0, 1.0)):
    """Manufactured finite-chaos solution: c_alpha = eta^|alpha|,
    Phi_alpha = prod_d sin(pi f x_d) with f = 1 + (alpha_{d mod M} mod 2),
    T(t) polynomial; Lambda_q in the library's order."""
    tiny = sg.sg_setup(dict(dim=2, cells=(2, 2), lo=(0.0, 0.0), hi=(1.0, 1.0)), 1, 0, 1, 1.0, M, q,
                       [dict(mu=(0,) * M, amp=1.0, factors=[("one", 0), ("one", 0)])])
    idx = sg.sg_get_multi_indices(tiny)
    tiny.destroy()
    c = [eta ** int(sum(a)) for a in idx]
    freq = [[1 + int(a[d % M]) % 2 for d in range(dim)] for a in idx]
    return {"q": q, "c": c, "freq": freq, "T": list(T)}


def march(sg, torch, ctx, rtol, slabs=None):
    """Slab marching with the manufactured right-hand sides; returns the last
    slab, total device-synchronised wall ms and per-slab iteration counts."""
    n = ctx.info["n_unknowns"]
    slabs = ctx.info["n_slabs"] if slabs is None else slabs
    dev = torch.device("cuda", torch.cuda.current_device())
    rhs = torch.empty(n, dtype=torch.float64, device=dev)
    u = torch.zeros(n, dtype=torch.float64, device=dev)
    u_prev = torch.zeros_like(u)
    its = []
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for s in range(slabs):
        sg.sg_rhs(ctx, s, u_prev if s else None, rhs)
        st = sg.sg_solve_slab(ctx, s, rhs, u, rtol=rtol)
        its.append(st["iterations"])
        u_prev.copy_(u)
    torch.cuda.synchronize()
    return u, 1e3 * (time.perf_counter() - t0), its


def next_mixed_precision(sg, torch, inputs):
    """Mixed-precision solve on the 3D 32^3 Q2, M=3 / P=3 workload: FP64
    V-cycle vs FP32 V-cycle vs FP32 V-cycle with bf16-stored Vanka factors
    (FP64 FGMRES, Arnoldi and residual), marching all 20 slabs to a 1e-8
    relative residual per slab."""
    spec = inputs.config_3d_q2_32()
    exact = exact_for(sg, spec["M"], 2, 3)
    out, ref = {}, None
    for name, ap, mp in (("fp64", sg.SG_PREC_FP64, sg.SG_PREC_FP64),
                         ("fp32_mg", sg.SG_PREC_FP64, sg.SG_PREC_FP32),
                         ("bf16_factors_mg", sg.SG_PREC_FP64, sg.SG_PREC_BF16),
                         ("bf16_factors_mg_dw_apply", sg.SG_PREC_DW, sg.SG_PREC_BF16)):
        ctx = sg.sg_setup_spec(spec, ap)
        sg.sg_autotune(ctx, reps=3)
        sg.sg_set_exact(ctx, exact)
        t0 = time.perf_counter()
        sg.sg_mg_setup(ctx, mp, MG_NU, MG_OMEGA)
        setup_ms = 1e3 * (time.perf_counter() - t0)
        setup_split = sg.sg_mg_setup_times(ctx)
        march(sg, torch, ctx, 1e-8, slabs=1)                     # warm-up: graphs, workspaces
        u, ms, its = march(sg, torch, ctx, 1e-8)
        err = sg.sg_qoi_errors(ctx, u, spec["n_slabs"] - 1)
        if ref is None:
            ref = u.clone()
        diff = float((u - ref).abs().max() / ref.abs().max())
        out[name] = {"march_ms": ms, "ms_per_slab": ms / spec["n_slabs"], "mg_setup_ms": setup_ms,
                     "mg_setup_split_ms": setup_split, "march_plus_setup_ms": ms + setup_ms,
                     "iterations_mean": sum(its) / len(its), "iterations_max": max(its),
                     "max_rel_diff_vs_fp64": diff,
                     "qoi_errors_T": err}
        ctx.destroy()
        del u
        torch.cuda.empty_cache()
    for k in out:
        out[k]["time_ratio_vs_fp64"] = out[k]["march_ms"] / out["fp64"]["march_ms"]
        out[k]["time_ratio_vs_fp64_with_setup"] = out[k]["march_plus_setup_ms"] / out["fp64"]["march_plus_setup_ms"]
    return {"row": "mixed precision", "workload": spec["name"], "unknowns_per_slab": inputs.n_unknowns(spec),
            "slabs": spec["n_slabs"], "rtol": 1e-8, "exact": "finite chaos q=2, eta=0.35, T(t)=t+t^2",
            "splits": out}


def next_mc_vs_sg(sg, torch, inputs, n_samples=4096, tile=64):
    """Batched Monte-Carlo against SG on the same GPU: the coefficient of the
    64x64 Q2 workload, dG(1), 50 slabs to t = 1; half the samples on 64x64,
    half on 128x128, all of them in ONE system per slab (mc_solve_meshes: one
    apply launch over both meshes); errors of the mean and variance at t = 1
    against the manufactured solution's exact statistics."""
    import numpy as np
    base = dict(inputs.config_2d_q2_64(), n_slabs=50)
    exact = exact_for(sg, 4, 2, 2)
    xi = np.random.default_rng(4096).standard_normal((n_samples, 4))
    half = n_samples // 2
    dev = torch.device("cuda", torch.cuda.current_device())
    meshes = (("64x64", (64, 64), xi[:half]), ("128x128", (128, 128), xi[half:]))
    ctxs = []
    for _, cells, _ in meshes:
        c = sg.sg_setup_spec(dict(base, cells=cells, P=0))
        sg.sg_set_exact(c, exact)
        ctxs.append(c)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    means, vars_, _, st = sg.mc_solve_meshes(ctxs, [m[2] for m in meshes], tile=tile,
                                             mg_precision=sg.SG_PREC_FP32, rtol=1e-8)
    torch.cuda.synchronize()
    mc_ms = 1e3 * (time.perf_counter() - t0)
    e_mc = [sg.sg_stat_errors(c, m, v, 1.0) for c, m, v in zip(ctxs, means, vars_)]
    for c in ctxs:
        c.destroy()
    rows, sg_total = {}, 0.0
    for (name, cells, xs), em in zip(meshes, e_mc):
        spec = dict(base, cells=cells)
        ctx = sg.sg_setup_spec(spec)
        sg.sg_autotune(ctx, reps=3)
        sg.sg_set_exact(ctx, exact)
        sg.sg_mg_setup(ctx, sg.SG_PREC_FP32, MG_NU, MG_OMEGA)
        march(sg, torch, ctx, 1e-8, slabs=1)
        u, sg_ms, its = march(sg, torch, ctx, 1e-8)
        m = torch.empty(ctx.info["n_x"], dtype=torch.float64, device=dev)
        v = torch.empty_like(m)
        sg.sg_moments(ctx, u, ctx.info["n_t"] - 1, m, v)
        e_sg = sg.sg_stat_errors(ctx, m, v, 1.0)
        ctx.destroy()
        sg_total += sg_ms
        rows[name] = {"mc_samples": int(xs.shape[0]), "mc_error_mean_L2": em["mean"], "mc_error_var_L2": em["var"],
                      "sg_chaos_modes": 35, "sg_ms": sg_ms, "sg_iterations_mean": sum(its) / len(its),
                      "sg_error_mean_L2": e_sg["mean"], "sg_error_var_L2": e_sg["var"],
                      "sg_more_accurate": e_sg["mean"] < em["mean"] and e_sg["var"] < em["var"]}
        torch.cuda.empty_cache()
    return {"row": "batched Monte-Carlo vs SG", "slabs": 50, "samples": n_samples,
            "xi": "default_rng(4096).standard_normal((4096, 4))", "rtol": 1e-8,
            "mc": {"ms": mc_ms, "one_system": "both meshes, all samples, one apply launch per FGMRES step",
                   "tile_cap": tile, "tile_autotuned": st["tile"], "chunk_autotuned": st["chunk"],
                   "groups": st["batches"], "fgmres_iterations_total": st["total_iterations"],
                   "max_slab_iterations": st["max_slab_iterations"], "max_rel_residual": st["max_rel_residual"]},
            "sg_ms_both_meshes": sg_total, "sg_faster": sg_total < mc_ms, "meshes": rows}


def next_adjoint(sg, torch, inputs, fd_rel_step=1e-6):
    """Adjoint gradient on the 128x128 Q2, M=4 / P=4 workload (70 modes,
    50 slabs): J = E ||u(T)||^2, dJ/d(sigma_m) and dJ/d(a0 per cell),
    checkpoints every 10 slabs; central differences for sigma_1 and one cell."""
    import numpy as np
    spec = inputs.config_2d_q2_128()
    exact = exact_for(sg, 4, 2, 2)
    ctx = sg.sg_setup_spec(spec)
    sg.sg_autotune(ctx, reps=3)
    sg.sg_set_exact(ctx, exact)
    sg.sg_mg_setup(ctx, sg.SG_PREC_FP32, MG_NU, MG_OMEGA)
    rtol = 1e-11
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    J, g_amp, g_cell, st = sg.sg_adjoint_gradient(ctx, rtol=rtol, checkpoint_every=10, cell_piece=0)
    grad_ms = 1e3 * (time.perf_counter() - t0)
    t0 = time.perf_counter()
    J_fwd = sg.sg_adjoint_gradient(ctx, rtol=rtol, checkpoint_every=10, gradient=False)[0]
    fwd_ms = 1e3 * (time.perf_counter() - t0)
    coef = [dict(p) for p in spec["coef"]]
    fd = {}
    # sigma_1 (piece 1) and the a0 value of the centre cell (piece 0)
    c_mid = (spec["cells"][1] // 2) * spec["cells"][0] + spec["cells"][0] // 2
    for name, kind in (("sigma_1", 1), (f"a0_cell_{c_mid}", 0)):
        vals = []
        for sgn in (1.0, -1.0):
            pc = [dict(p) for p in coef]
            if kind == 1:
                h = fd_rel_step * pc[1]["amp"]
                pc[1]["amp"] = pc[1]["amp"] + sgn * h
            else:
                cs = np.array(pc[0]["cell_scale"], dtype=np.float64)
                h = fd_rel_step * cs[c_mid]
                cs[c_mid] += sgn * h
                pc[0]["cell_scale"] = cs
            sg.sg_set_coefficient(ctx, pc)
            vals.append(sg.sg_adjoint_gradient(ctx, rtol=rtol, checkpoint_every=10, gradient=False)[0])
        fdv = (vals[0] - vals[1]) / (2 * h)
        adj = float(g_amp[1]) if kind == 1 else float(g_cell[c_mid])
        fd[name] = {"adjoint": adj, "central_difference": fdv, "rel_diff": abs(adj - fdv) / abs(fdv)}
    sg.sg_set_coefficient(ctx, coef)
    ctx.destroy()
    return {"row": "adjoint gradient", "workload": spec["name"], "unknowns_per_slab": inputs.n_unknowns(spec),
            "slabs": spec["n_slabs"], "checkpoint_every": 10, "rtol": rtol, "mg": "fp32 V-cycle, fp64 FGMRES",
            "J": J, "J_forward_only": J_fwd, "grad_ms": grad_ms, "forward_only_ms": fwd_ms,
            "grad_over_forward": grad_ms / fwd_ms, "forward_solves": st["forward_solves"],
            "adjoint_solves": st["adjoint_solves"], "max_iterations": st["max_iterations"],
            "grad_sigma": [float(v) for v in g_amp[1:]], "grad_a0_norm": float(np.linalg.norm(g_cell)),
            "fd_relative_step": fd_rel_step, "fd_checks": fd}


# algorithmic FP64 flop per unknown of the sum-factorised apply (operation count of
# the forward/backward sum factorisation plus the point kernel) per workload
FLOP_PER_UNKNOWN_BY_WORKLOAD = {"2d-q2-64x64-M4P3": 166.0, "3d-q2-32x32x32-M3P3": 345.0,
                                "2d-q2-128x128-M4P4": 172.0}


def next_applies(sg, torch, inputs, steps=100, warmup=10):
    """The apply on the two large workloads (32^3 Q2 M=3 P=3, 10.99 M unknowns;
    128x128 Q2 M=4 P=4, 9.25 M unknowns): FP64 forward, FP64 transpose (the
    adjoint apply) and double-word forward, autotuned launch shape, over
    rotating x/y pairs larger than L2, per-launch CUDA events."""
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream(dev)
    out = {}
    for maker in (inputs.config_3d_q2_32, inputs.config_2d_q2_128):
        spec = maker()
        row = {}
        X = Y = None
        for vname, prec, transpose in (("fp64", sg.SG_PREC_FP64, False), ("fp64_transpose", sg.SG_PREC_FP64, True),
                                       ("dw", sg.SG_PREC_DW, False)):
            ctx = sg.sg_setup_spec(spec, prec)
            sg.sg_autotune(ctx, reps=5)
            n = ctx.info["n_unknowns"]
            if X is None:
                R = max(2, math.ceil(2.2 * L2_BYTES / (16 * n)))
                gen = torch.Generator(device=dev)
                gen.manual_seed(inputs.SEED_X)
                X = [torch.rand(n, dtype=torch.float64, device=dev, generator=gen) * 2 - 1 for _ in range(R)]
                Y = [torch.empty(n, dtype=torch.float64, device=dev) for _ in range(R)]
            for s_ in range(warmup):
                sg.sg_apply(ctx, 0, X[s_ % R], Y[s_ % R], transpose, stream)
            torch.cuda.synchronize()
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
            with ClockSampler(torch.cuda.current_device()) as clk:
                torch.cuda.synchronize()
                for s_ in range(steps):
                    ev[s_][0].record(stream)
                    sg.sg_apply(ctx, 0, X[s_ % R], Y[s_ % R], transpose, stream)
                    ev[s_][1].record(stream)
                torch.cuda.synchronize()
            t = statistics.mean(a.elapsed_time(b) for a, b in ev) / 1e3
            tf = FLOP_PER_UNKNOWN_BY_WORKLOAD[spec["name"]] * n / t / 1e12
            row[vname] = {"value": n / t / 1e9, "unit": UNIT, "ms_per_apply": 1e3 * t,
                          "fp64_equivalent_tflops": tf, "frac_of_fp64_peak": tf / FP64_PEAK_TFLOPS,
                          "hbm_gbs": BYTES_PER_UNKNOWN * n / t / 1e9,
                          "launch": {"chunk_cells": ctx.info["chunk"], "grid": ctx.info["grid"],
                                     "threads": ctx.info["threads"], "stagger": ctx.info["stagger"]},
                          "clocks": clk.summary()}
            ctx.destroy()
        row["unknowns"] = n
        row["l2"] = f"{R} rotating x/y pairs, {16 * R * n / 1e6:.0f} MB > {L2_BYTES / 1e6:.0f} MB L2"
        out[spec["name"]] = row
        del X, Y
        torch.cuda.empty_cache()
    return {"row": "applies", "metric": METRIC, "unit": UNIT,
            "flop_per_unknown": FLOP_PER_UNKNOWN_BY_WORKLOAD, "fp64_peak_tflops": FP64_PEAK_TFLOPS,
            "workloads": out}


# the paper's own apply throughput on its discretisation, by chaos degree, on its
# CPU cluster - context beside the GPU figure, not a target.  The paper prints no
# rate: each figure is N_SG x vmult calls / accumulated apply seconds, taken from
# the columns of its solver-performance table (Sec. 6), in G unknowns/s.
PAPER_TABLE2_GUPS = {0: 1.265, 1: 0.434, 2: 0.286, 3: 0.237}


def next_paper(sg, torch, inputs, steps=30, warmup=5):
    """The FP64 apply on the paper's own benchmark discretisation (128x128 Q3 on
    (-1, 1)^2, dG(3), M = 4, the squared coefficient with 11 modes) for chaos
    degree 0..3 (148,225 nodes x 4 time nodes x 1..35 modes), autotuned shape,
    rotating x/y pairs larger than L2, mean per-launch CUDA-event time."""
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream(dev)
    out = {}
    for P in sorted(PAPER_TABLE2_GUPS):
        spec = inputs.config_paper_q3(P=P)
        ctx = sg.sg_setup_spec(spec, sg.SG_PREC_FP64)
        try:
            sg.sg_autotune(ctx, reps=5)
            n = ctx.info["n_unknowns"]
            R = max(2, math.ceil(2.2 * L2_BYTES / (16 * n)))
            gen = torch.Generator(device=dev)
            gen.manual_seed(inputs.SEED_X)
            X = [torch.rand(n, dtype=torch.float64, device=dev, generator=gen) * 2 - 1 for _ in range(R)]
            Y = [torch.empty(n, dtype=torch.float64, device=dev) for _ in range(R)]
            for k in range(warmup):
                sg.sg_apply(ctx, 0, X[k % R], Y[k % R], False, stream)
            torch.cuda.synchronize()
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
            with ClockSampler(torch.cuda.current_device()) as clk:
                for k in range(steps):
                    ev[k][0].record(stream)
                    sg.sg_apply(ctx, 0, X[k % R], Y[k % R], False, stream)
                    ev[k][1].record(stream)
                torch.cuda.synchronize()
            assert torch.isfinite(Y[0]).all()
            t = statistics.mean(a.elapsed_time(b) for a, b in ev) / 1e3
            out[f"P{P}"] = {"chaos_modes": ctx.info["n_xi"], "unknowns": n, "ms_per_apply": 1e3 * t,
                            "value": n / t / 1e9, "unit": UNIT, "paper_table2_cpu_cluster": PAPER_TABLE2_GUPS[P],
                            "launch": {"chunk_cells": ctx.info["chunk"], "grid": ctx.info["grid"],
                                       "threads": ctx.info["threads"], "stagger": ctx.info["stagger"]},
                            "clocks": clk.summary()}
            del X, Y
        finally:
            ctx.destroy()
            torch.cuda.empty_cache()
    return {"row": "paper discretisation", "metric": METRIC, "unit": UNIT,
            "workload": "128x128 Q3 on (-1,1)^2, dG(3), M=4, squared coefficient (11 modes)",
            "paper_context": "Table 2 of the paper, its CPU cluster; context only", "degrees": out}


def next_vcycle(sg, torch, inputs, profile_range=False, profile_mg="fp32", profile_workload="3d"):
    """One V-cycle of the block-Jacobi multigrid (all modes at once) on the
    64x64 Q2 P=3 and 32^3 Q2 P=3 workloads, per precision: device ms per
    V-cycle (10 graph launches after 3 warm-up ones).  With profile_range one
    more V-cycle (profile_mg precision) with the solver's sweeps and damping on
    the profile_workload ("3d" or "2d") is bracketed by cudaProfilerStart/Stop."""
    out = {}
    for wname, maker in (("2d-q2-64x64-M4P3", inputs.config_2d_q2_64), ("3d-q2-32x32x32-M3P3", inputs.config_3d_q2_32)):
        spec = maker()
        ctx = sg.sg_setup_spec(spec)
        n = ctx.info["n_unknowns"]
        r = torch.rand(n, dtype=torch.float64, device="cuda")
        z = torch.empty_like(r)
        row = {}
        for pname, prec in (("fp64", sg.SG_PREC_FP64), ("fp32", sg.SG_PREC_FP32), ("bf16_factors", sg.SG_PREC_BF16)):
            for nu, om in ((2, 0.7), (MG_NU, MG_OMEGA)):
                sg.sg_mg_setup(ctx, prec, nu, om)
                for _ in range(3):
                    sg.sg_vcycle(ctx, r, z)
                torch.cuda.synchronize()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record()
                for _ in range(10):
                    sg.sg_vcycle(ctx, r, z)
                b.record()
                torch.cuda.synchronize()
                row[f"{pname}_nu{nu}"] = a.elapsed_time(b) / 10
                if prec == sg.SG_PREC_BF16 and nu == MG_NU:
                    # the same V-cycle with each Vanka sweep forced on every level
                    # (the tensor-core sweep with one and with two staging buffers)
                    for kname, kind, chunk in (("ffma", 0, 0), ("tensor_1buf", 1, 1), ("tensor_2buf", 1, 2)):
                        try:
                            sg.sg_mg_set_level_variant(ctx, -1, -1, chunk, -1, kind)
                        except sg.SGError:
                            continue
                        for _ in range(3):
                            sg.sg_vcycle(ctx, r, z)
                        torch.cuda.synchronize()
                        a.record()
                        for _ in range(10):
                            sg.sg_vcycle(ctx, r, z)
                        b.record()
                        torch.cuda.synchronize()
                        row[f"{pname}_nu{nu}_vanka_{kname}"] = a.elapsed_time(b) / 10
        if profile_range and wname.startswith(profile_workload):
            sg.sg_mg_setup(ctx, sg.SG_PREC_BF16 if profile_mg.startswith("bf16") else sg.SG_PREC_FP32,
                           MG_NU, MG_OMEGA)
            if profile_mg in ("bf16-tensor", "bf16-tensor-1buf"):
                sg.sg_mg_set_level_variant(ctx, -1, -1, 1 if profile_mg.endswith("1buf") else 2, -1, 1)
            row["profiled_levels"] = [sg.sg_mg_level_info(ctx, lev) for lev in range(sg.sg_mg_level_info(ctx, 0)["levels"])]
            sg.sg_vcycle(ctx, r, z)
            torch.cuda.synchronize()
            torch.cuda.profiler.start()
            sg.sg_vcycle(ctx, r, z)
            torch.cuda.synchronize()
            torch.cuda.profiler.stop()
        ctx.destroy()
        out[wname] = row
    return {"row": "V-cycle", "unit": "ms per V-cycle", "workloads": out}


def next_krylov(sg, torch, inputs):
    """Cost of one FGMRES iteration outside the preconditioner and the operator:
    slab solves cut off after 1, 3, 5, 7 and 9 iterations (restart 30, a
    tolerance they cannot reach), device time per solve (median of CUDA-event
    times, host set-up of the call included), a straight-line fit over the
    iteration count; the slope minus one V-cycle and one FP64 apply, each timed
    alone, is the Arnoldi step's own part (Gram-Schmidt passes, next basis
    vector, Hessenberg update).  64x64 Q2 P=3 with the FP32 V-cycle and 32^3 Q2
    P=3 with bf16 factors, as in the solve and mixed-precision rows."""
    import numpy as np
    out = {}
    for wname, maker, prec, reps in (("2d-q2-64x64-M4P3", inputs.config_2d_q2_64, sg.SG_PREC_FP32, 10),
                                     ("3d-q2-32x32x32-M3P3", inputs.config_3d_q2_32, sg.SG_PREC_BF16, 3)):
        ctx = sg.sg_setup_spec(maker())
        sg.sg_mg_setup(ctx, prec, MG_NU, MG_OMEGA)
        n = ctx.info["n_unknowns"]
        gen = torch.Generator(device="cpu").manual_seed(3)
        b = torch.rand(n, dtype=torch.float64, generator=gen).cuda()
        x = torch.zeros_like(b)
        for _ in range(2):
            x.zero_()
            sg.sg_solve_slab(ctx, 0, b, x, rtol=1e-14, max_it=9, restart=30, check=False)
        torch.cuda.synchronize()
        pts = []
        for mi in (1, 3, 5, 7, 9):
            ts = []
            for _ in range(reps):
                x.zero_()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                st = sg.sg_solve_slab(ctx, 0, b, x, rtol=1e-14, max_it=mi, restart=30, check=False)
                e1.record()
                torch.cuda.synchronize()
                ts.append(e0.elapsed_time(e1))
            pts.append((st["iterations"], statistics.median(ts)))
        its = np.array([q[0] for q in pts], dtype=np.float64)
        slope, icpt = np.polyfit(its, np.array([q[1] for q in pts]), 1)
        z = torch.empty_like(b)
        y = torch.empty_like(b)
        for _ in range(3):
            sg.sg_vcycle(ctx, b, z)
            ctx.apply(b, y)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(10):
            sg.sg_vcycle(ctx, b, z)
        e1.record()
        torch.cuda.synchronize()
        vc = e0.elapsed_time(e1) / 10
        e0.record()
        for _ in range(10):
            ctx.apply(b, y)
        e1.record()
        torch.cuda.synchronize()
        ap = e0.elapsed_time(e1) / 10
        out[wname] = {"unknowns": n, "mg": "fp32" if prec == sg.SG_PREC_FP32 else "bf16 factors",
                      "iterations_ms": [[int(i), round(t, 4)] for i, t in pts],
                      "slope_ms_per_iteration": float(slope), "intercept_ms": float(icpt),
                      "vcycle_ms": vc, "apply_ms": ap, "arnoldi_step_ms": float(slope) - vc - ap}
        ctx.destroy()
    return {"row": "FGMRES iteration", "unit": "ms", "workloads": out}


def run_next(args, world, rank, local):
    import torch
    import paper_2605_21046_gb300 as sg
    from paper_2605_21046_gb300 import build, inputs
    build.build()
    torch.cuda.set_device(torch.device("cuda", local))
    if rank != 0:
        return
    rows = [s.strip() for s in args.rows.split(",")]
    for row in rows:
        t0 = time.perf_counter()
        try:
            if row == "mixed":
                out = next_mixed_precision(sg, torch, inputs)
            elif row == "mc":
                out = next_mc_vs_sg(sg, torch, inputs, n_samples=args.mc_samples)
            elif row == "adjoint":
                out = next_adjoint(sg, torch, inputs)
            elif row == "vcycle":
                out = next_vcycle(sg, torch, inputs, profile_range=args.profile_range, profile_mg=args.profile_mg,
                                  profile_workload=args.profile_workload)
            elif row == "applies":
                out = next_applies(sg, torch, inputs)
            elif row == "paper":
                out = next_paper(sg, torch, inputs)
            elif row == "krylov":
                out = next_krylov(sg, torch, inputs)
            else:
                raise ValueError(row)
        except sg.SGError as ex:
            out = {"row": row, "error": str(ex)}
            torch.cuda.empty_cache()
        out.update({"suite": "next", "impl": "ours", "wall_s": time.perf_counter() - t0,
                    "gpu": torch.cuda.get_device_name()})
        print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--ref-seconds", type=float, default=90.0,
                    help="--impl reference: target duration of the W + K oracle steps")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-cpu-all-cores", action="store_true", help="skip the all-cores oracle timing")
    ap.add_argument("--no-dw", action="store_true", help="skip the double-word variant")
    ap.add_argument("--no-solve", action="store_true", help="skip the slab-solve timing")
    ap.add_argument("--profile-variant", choices=["fp64", "dw"], default="fp64",
                    help="which timed apply loop --profile-range brackets")
    ap.add_argument("--profile-solve", choices=["fp64", "fp32_mg", "bf16_factors_mg", "fp32_mg_dw_apply"],
                    default=None, help="bracket one more slab solve of this split with cudaProfilerStart/Stop")
    ap.add_argument("--profile-workload", choices=["3d", "2d"], default="3d",
                    help="workload of the V-cycle --profile-range brackets (--rows vcycle): 32^3 Q2 or 64x64 Q2")
    ap.add_argument("--profile-mg", choices=["fp32", "bf16", "bf16-tensor", "bf16-tensor-1buf"], default="fp32",
                    help="multigrid precision of the V-cycle --profile-range brackets (--rows vcycle)")
    ap.add_argument("--no-next", action="store_true",
                    help="skip the NEXT rows (mixed precision, Monte-Carlo vs SG, adjoint) of the default line")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default launch shapes")
    ap.add_argument("--profile-range", action="store_true",
                    help="bracket the timed FP64 applies with cudaProfilerStart/Stop")
    ap.add_argument("--suite", choices=["apply", "next"], default="apply",
                    help="apply: the headline line; next: one line per solver-side row")
    ap.add_argument("--rows", default="mixed,mc,adjoint", help="rows of --suite next "
                    "(mixed, mc, adjoint, vcycle, applies, paper, krylov)")
    ap.add_argument("--mc-samples", type=int, default=4096)
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    world, rank, local = dist_init()
    if args.impl == "reference":
        run_reference(args, world, rank)
    elif args.suite == "next":
        run_next(args, world, rank, local)
    else:
        run_ours(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
