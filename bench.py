#!/usr/bin/env python3
"""Benchmark: red-black SOR on the paper-sized plate (4098 x 4098 array, 4096^2
interior), 1000 iterations with the max|change| reduction every 50, FP64.

One step = one complete solve through the C ABI (pack, 1000 red-black
iterations, residual of the result, unpack), inputs already in HBM.
Prints ONE JSON line (rank 0).  ``--impl reference`` times the CPU oracle on
a bounded sample of the same workload instead.

Multi-GPU (torchrun): the path does not shard; every rank solves its own
plate (replicas), ``value`` counts the updates of all ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N = 4096
ITERS = 1000
CHECK = 50
METRIC = "red-black SOR GLUP/s + % HBM roofline; solves/s & p99 latency at 1e-10 residual"
WORKLOAD = "paper-sized plain sweep: 4098x4098 array (4096^2 interior), random uniform[0,100] edges (seed 0), " \
           "interior 0, f=0, w_opt, 1000 iterations, max|change| every 50"
FP64_FLOPS_PER_LUP = 6.0    # (1-w)u + (w/4)(N+S+W+E): 3 adds, 2 multiplies, 1 add
HBM_BYTES_PER_LUP = {"f64": 16.0, "f32": 8.0}  # read + write of each cell once per iteration
NOMINAL_FP64_TFLOPS = 1.25  # GB300 FP64 (non-tensor) nominal rate: 152 SMs x 2 lanes/clk x 2.07 GHz x 2 flops
# dram__bytes_read.sum + dram__bytes_write.sum of one k_fast_chain launch (50 iterations) on this workload,
# from the ncu capture of the current kernel (None: no capture of the current kernel yet)
FAST64_DRAM_BYTES_PER_LAUNCH = 11405769728 + 6608791552
# the same counters for one k_sweep_tb<6,0> launch (6 fused iterations) on the FP32 plate, per update
# (captured again after the kernel lost its unused 16 KB right-hand-side ring)
TB32_DRAM_BYTES_PER_UPDATE = (68468992 + 21732096) / (6.0 * 4096 * 4096)


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class Clocks:
    """Samples SM clocks and throttle reasons with nvidia-smi while running."""

    FIELDS = "clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown," \
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown," \
             "clocks_event_reasons.sw_power_cap"

    def __init__(self, index: int):
        self.index = index
        self.samples = []
        self._stop = threading.Event()
        self._th = None

    def _run(self):
        while not self._stop.is_set():
            try:
                out = subprocess.run(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                      "--format=csv,noheader,nounits"], capture_output=True, text=True,
                                     timeout=5).stdout.strip()
                if out:
                    self.samples.append([x.strip() for x in out.split(",")])
            except Exception:
                pass
            self._stop.wait(0.2)

    def __enter__(self):
        self._th = threading.Thread(target=self._run, daemon=True)
        self._th.start()
        return self

    def __exit__(self, *exc):
        self._stop.set()
        if self._th:
            self._th.join(timeout=10)

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for s in self.samples for k in range(4) if len(s) > 3 + k and
                          s[3 + k].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.samples)}


def max_over_ranks(value: float, ws: int) -> float:
    """Largest value over the ranks of the default process group (the timing
    rule: the slowest rank's time counts); the value itself when ws == 1."""
    if ws <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_glups(lups_per_rank: float, ms_max: float, ws: int) -> float:
    """Whole-job throughput: every rank solved its own plate (replicas), so
    the work is ws * lups_per_rank over the slowest rank's time."""
    return ws * lups_per_rank / (ms_max * 1e-3) / 1e9


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def oracle_sample(n_iters: int):
    """Time the CPU oracle on the same plate for n_iters iterations."""
    import numpy as np  # noqa: F401

    import oracle
    from paper_1401_0763_gb300 import workloads as wl
    u0 = wl.random_edges(N, 0)
    w = oracle.omega_opt(N)
    oracle.build()
    t0 = time.perf_counter()
    oracle.sor_f64(u0, w, max_iters=n_iters, check_every=CHECK, tol=-1.0)
    dt = time.perf_counter() - t0
    return (N * N * n_iters) / dt / 1e9, dt


def allcore_sample(n_iters: int):
    """Time the threaded CPU twin of the oracle (bitwise equal to it) on every
    host core, same plate."""
    import cpu_baseline
    import oracle
    from paper_1401_0763_gb300 import workloads as wl
    u0 = wl.random_edges(N, 0)
    cpu_baseline.build()
    w = oracle.omega_opt(N)
    cores = cpu_baseline.host_cores()
    t0 = time.perf_counter()
    r = cpu_baseline.sor_f64_mt(u0, w, max_iters=n_iters, check_every=CHECK, tol=-1.0, threads=cores)
    dt = time.perf_counter() - t0
    return (N * N * n_iters) / dt / 1e9, dt, r["threads"]


def run_reference(args, ws, rank):
    if rank != 0:
        return 0
    iters = args.ref_iters
    for _ in range(args.warmup):
        oracle_sample(max(1, iters // 10))
    vals = []
    t_all = 0.0
    for _ in range(args.steps):
        v, dt = oracle_sample(iters)
        vals.append(v)
        t_all += dt
    total_lups = N * N * iters * args.steps
    value = total_lups / t_all / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "GLUP/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * t_all / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample": f"{iters} of the {ITERS} iterations per step", "l2": "n/a (CPU)"},
        "cpu_baseline": {"value": value, "unit": "GLUP/s", "cores": 1, "kind": "oracle",
                         "sample": f"4096^2 plate, {iters} iterations per step, {args.steps} steps"},
        "e2e": {"value": value, "unit": "GLUP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args, ws, rank, local):
    import numpy as np
    import torch

    from paper_1401_0763_gb300 import capi
    from paper_1401_0763_gb300 import workloads as wl

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
    capi.load()
    stream = torch.cuda.Stream(device=dev)
    ctx = capi.Context(local, 0, stream)
    ctx.set_option(capi.SOR_OPT_TIMING, 1)
    ctx.set_option(capi.SOR_OPT_TEMPORAL_DEPTH, args.tdepth)

    u0_np = wl.random_edges(N, rank)
    w = capi.sor_omega_opt(N)
    kw = dict(omega=w, tol=-1.0, max_iters=ITERS, check_every=CHECK)
    u0 = torch.from_numpy(u0_np).to(dev)
    out = torch.empty_like(u0)
    torch.cuda.synchronize()

    def barrier():
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()

    def step(precision, src, dst):
        st, res = ctx.solve_raw(capi.make_params(N, precision=precision, **kw), src.data_ptr(), None, dst.data_ptr())
        if st != capi.SOR_OK:
            raise capi.SorError(st, ctx.last_error())
        return res.as_dict()

    # ---- device-resident FP64 (the headline) --------------------------------------------------------------
    for _ in range(args.warmup):
        step(capi.SOR_FP64, u0, out)
    ctx.reset_stats()
    barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with Clocks(local) as clk:
        ev0.record(stream)
        res = None
        for _ in range(args.steps):
            res = step(capi.SOR_FP64, u0, out)
        ev1.record(stream)
        torch.cuda.synchronize()
    barrier()
    ms = ev0.elapsed_time(ev1)
    st = ctx.stats()
    ms_max = max_over_ranks(ms, ws)
    lups_rank = float(N) * N * ITERS * args.steps
    value = aggregate_glups(lups_rank, ms_max, ws)
    launches = int(st["kernel_launches"])  # every kernel launch of the timed solves (graph replays included)
    sweep_ms_per_launch = st["sweep_ms"] / max(1, st["timed_launches"])
    lups_per_launch = float(N) * N / 2.0  # one colour phase updates half the cells
    fp64_tflops = lups_per_launch * FP64_FLOPS_PER_LUP / (sweep_ms_per_launch * 1e-3) / 1e12
    hbm_gbs_fp64 = lups_per_launch * HBM_BYTES_PER_LUP["f64"] / (sweep_ms_per_launch * 1e-3) / 1e9
    peaks, peaks_src = measured_peaks()
    check = {"iterations": res["iterations"], "final_maxdelta": res["final_maxdelta"],
             "final_resid_rel": res["final_resid_rel"]}
    # the FP64 peak, measured now on this GPU: independent FMA chains (2 flops each) and addition chains
    fma_rate = ctx.diag_fp64_rate(0)
    add_rate = ctx.diag_fp64_rate(1)
    fp64_peak_tflops = 2.0 * fma_rate / 1e12

    # ---- FP32 storage, same plate (secondary line item) -----------------------------------------------------
    for _ in range(max(1, args.warmup // 2)):
        step(capi.SOR_FP32, u0, out)
    ctx.reset_stats()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step(capi.SOR_FP32, u0, out)
    e1.record(stream)
    torch.cuda.synchronize()
    ms32 = e0.elapsed_time(e1)
    st32 = ctx.stats()
    per32 = st32["sweep_ms"] / max(1, st32["timed_launches"])
    # algorithmic bytes: 8 B per update of an unfused iteration (read + write each cell once); the fused
    # kernel moves fewer DRAM bytes (state in L2 at this size; see dram_bytes_per_update)
    fp32 = {"value": lups_rank / (ms32 * 1e-3) / 1e9, "unit": "GLUP/s", "ms_per_step": ms32 / args.steps,
            "algorithmic_gbs": lups_per_launch * HBM_BYTES_PER_LUP["f32"] / (per32 * 1e-3) / 1e9,
            "algorithmic_bytes_per_update": HBM_BYTES_PER_LUP["f32"],
            "dram_bytes_per_update": TB32_DRAM_BYTES_PER_UPDATE,
            "note": "the 68 MB FP32 state fits in L2: algorithmic_gbs is not an HBM measurement"}
    fp32["algorithmic_over_hbm_peak"] = fp32["algorithmic_gbs"] / peaks["hbm_gbs"]

    # ---- end to end: pinned host buffers, copies inside the timed region ------------------------------------
    h_u0 = torch.from_numpy(u0_np).pin_memory()
    h_out = torch.empty_like(h_u0).pin_memory()
    step(capi.SOR_FP64, h_u0, h_out)
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e2 = torch.cuda.Event(enable_timing=True)
    e3 = torch.cuda.Event(enable_timing=True)
    e2.record(stream)
    for _ in range(args.steps):
        step(capi.SOR_FP64, h_u0, h_out)
    e3.record(stream)
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(max(e2.elapsed_time(e3), 1e3 * (time.perf_counter() - t0)), ws)
    e2e = {"value": aggregate_glups(lups_rank, e2e_ms, ws), "unit": "GLUP/s",
           "h2d_bytes_per_step": int(h_u0.numel() * 8), "d2h_bytes_per_step": int(h_out.numel() * 8)}
    assert np.isfinite(h_out.numpy()).all()

    # ---- CPU baseline: the oracle on a bounded sample (rank 0, N=1 only) ------------------------------------
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        import cpu_baseline
        v, dt = oracle_sample(args.cpu_iters)
        va, dta, threads = allcore_sample(args.allcore_iters)
        cpu = {"value": v, "unit": "GLUP/s", "cores": 1, "kind": "oracle",
               "sample": f"4096^2 plate, {args.cpu_iters} iterations ({dt:.1f} s, single thread)",
               "host_cores": cpu_baseline.host_cores(), "os_cpu_count": os.cpu_count(),
               "allcore": {"value": va, "unit": "GLUP/s", "cores": threads,
                           "kind": "threaded red-black twin of the oracle (bitwise equal to it)",
                           "sample": f"4096^2 plate, {args.allcore_iters} iterations ({dta:.1f} s)"}}

    ctx.close()
    if rank == 0:
        clocks = clk.summary()
        line = {
            "metric": METRIC, "value": value, "unit": "GLUP/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n": N, "iterations": ITERS, "check_every": CHECK,
                       "l2": "inputs larger than L2 (134 MB natural in + 136 MB colour-split state + 134 MB out; "
                             "no flush)", "parallelism": "replicas" if ws > 1 else "single GPU"},
            "roofline": {"bound": "alu", "achieved": fp64_tflops, "peak": fp64_peak_tflops, "unit": "TFLOP/s",
                         "frac": fp64_tflops / fp64_peak_tflops,
                         "traffic": FAST64_DRAM_BYTES_PER_LAUNCH,
                         "traffic_unit": "bytes per launch of 50 iterations (dram read + write, ncu)",
                         "traffic_algorithmic": 16.0 * N * N * CHECK,
                         "kernel": "k_fast_chain<false> (a chunk of 50 iterations per launch; "
                                   "achieved from the per-phase CUDA-event time)",
                         "peak_source": "measured on this GPU by sor_diag_fp64_rate: independent FP64 FMA chains, "
                                        "2 flops per FMA (of measured)",
                         "fp64_fma_ops_per_s": fma_rate, "fp64_add_ops_per_s": add_rate,
                         "nominal_peak": NOMINAL_FP64_TFLOPS, "frac_of_nominal": fp64_tflops / NOMINAL_FP64_TFLOPS,
                         "hbm_gbs": hbm_gbs_fp64, "hbm_frac": hbm_gbs_fp64 / peaks["hbm_gbs"],
                         "hbm_peak_source": peaks_src},
            "fp32": fp32,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": launches,
            "clocks": {k: v for k, v in clocks.items() if k in ("sm_mhz", "sm_max_mhz", "reasons")},
            "check": check,
        }
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


# ---------------------------------------------------------------------------------------------------------------
# other workloads (one JSON line each, selected with --workload; the default line is above)
# ---------------------------------------------------------------------------------------------------------------

def _pct(xs, q):
    import numpy as np
    return float(np.percentile(np.asarray(xs), q)) if len(xs) else None


def workload_plate256(args, ctx, capi, wl):
    """258x258 plate, top edge 100, w_opt, stop on max|change| < 1e-8 checked every iteration."""
    import numpy as np
    n = 256
    u0 = np.ascontiguousarray(wl.heat_plate(n, 100.0))
    out = np.empty_like(u0)
    lines = {}
    # the default (one launch on a cooperative grid of many SMs, bands exchanging edge rows point to point and
    # the stop test decided behind the sweeps), the same grid with a grid-wide barrier per colour phase, one
    # thread-block cluster, and the chunked multi-CTA path; all evaluate the update in the oracle's exact order
    for name, small in (("fp64", 1), ("fp64_gridbar", 3), ("fp64_cluster", 2), ("fp64_chunked", 0)):
        ctx.set_option(capi.SOR_OPT_CLUSTER, small)
        kw = dict(omega=capi.sor_omega_opt(n), tol=1e-8, max_iters=5000, check_every=1,
                  flags=capi.SOR_FLAG_EXACT_ORDER)
        for _ in range(args.warmup):
            ctx.solve(u0, out=out, **kw)
        t0 = time.perf_counter()
        dev = []
        for _ in range(args.steps):
            _, res = ctx.solve(u0, out=out, **kw)
            dev.append(res["device_s"])
        dt = (time.perf_counter() - t0) / args.steps
        lines[name] = {"solve_ms": 1e3 * dt, "device_ms": 1e3 * float(np.median(dev)), "solves_per_s": 1.0 / dt,
                       "iterations": res["iterations"], "glups": n * n * res["iterations"] / dt / 1e9,
                       "converged": res["converged"]}
    ctx.set_option(capi.SOR_OPT_CLUSTER, 1)
    return {"metric": "time to solution, 258x258 heat plate to max|change| < 1e-8", "value": lines["fp64"]["solve_ms"],
            "unit": "ms", "higher_is_better": False, "detail": lines,
            "config": {"workload": "258x258 plate, top 100, w_opt, K=1, cap 5000, host buffers, exact order"}}


def workload_poisson4096(args, ctx, capi, wl):
    """Poisson -Laplace(u) = f with the 8-Gaussian source, zero edges: FP32 sweeps + FP64 defect correction
    (20 sweeps per correction) versus plain FP64 SOR with the residual test every 20 iterations, to the same
    relative residual ||f - Au|| / ||f||.  The 1e-10 target is below what an FP64 solution can reach beyond
    N ~ 1024 (the floor grows like (N+1)^2), so the 4098^2 plate is run to 1e-7 and 1e-8 and the 1e-10 target
    on 1026^2; both solvers stop at their floor (stall window of 50 residual tests)."""
    import torch
    cases = [(4096, 1e-7), (4096, 1e-8), (1024, 1e-10)]
    detail = {}
    for n, tol in cases:
        u0_np, f_np = wl.poisson_problem(n, args.seed)
        u0 = torch.from_numpy(u0_np).cuda()
        f = torch.from_numpy(f_np).cuda()
        out = torch.empty_like(u0)
        w = capi.sor_omega_opt(n)
        runs = {"fp32_refine": dict(precision=capi.SOR_FP32_REFINE, omega=w, tol=tol, max_iters=400000,
                                    inner_sweeps=20, stall_window=50),
                "fp64_plain": dict(precision=capi.SOR_FP64, omega=w, tol=tol, max_iters=400000, check_every=20,
                                   stop=capi.SOR_STOP_RESID_REL, stall_window=50)}
        key = f"n{n}_tol{tol:g}"
        detail[key] = {}
        for name, kw in runs.items():
            ctx.solve(u0, f, out=out, **dict(kw, max_iters=200))  # warm-up: workspace, graphs
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            _, res = ctx.solve(u0, f, out=out, **kw)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            rec = {"time_to_solution_s": dt, "sweeps": res["iterations"], "outer_steps": res["outer_steps"],
                   "final_resid_rel": res["final_resid_rel"], "converged": res["converged"],
                   "glups": float(n) * n * res["iterations"] / dt / 1e9}
            detail[key][name] = rec
        r, p = detail[key]["fp32_refine"], detail[key]["fp64_plain"]
        detail[key]["speedup_refine_vs_plain"] = p["time_to_solution_s"] / r["time_to_solution_s"]
    head = detail["n4096_tol1e-07"]
    return {"metric": "time to solution, 4098^2 Poisson (8 Gaussians) to relative residual 1e-7 "
                      "(and 1e-8; 1026^2 to 1e-10)",
            "value": head["fp32_refine"]["time_to_solution_s"], "unit": "s", "higher_is_better": False,
            "detail": detail,
            "config": {"workload": "zero edges, f = 8-Gaussian sum (seeded), w_opt, inner 20 FP32 sweeps, "
                                   "stall window 50"}}


def workload_batch512(args, ctx, capi, wl):
    """512 heat plates, interior side log-uniform in [64, 1024], random edges, FP32 sweeps + FP64 defect
    correction to a 1e-10 relative residual, all submitted at once to the batching scheduler."""
    import numpy as np
    count = args.count or 512
    sizes = wl.batch_sizes(count, args.seed)
    reqs = []
    for k, n in enumerate(sizes):
        n = int(n)
        u0 = np.ascontiguousarray(wl.random_edges(n, args.seed * 1000 + k))
        reqs.append((n, u0, np.empty_like(u0)))
    kw = dict(precision=capi.SOR_FP32_REFINE, tol=1e-10, max_iters=1000000, inner_sweeps=20)
    best = None
    for rep in range(max(1, args.steps // 2) + 1):  # first repetition warms up
        t0 = time.perf_counter()
        tickets = [ctx.submit(u0, None, out=o, omega=capi.sor_omega_opt(n), **kw)[0] for n, u0, o in reqs]
        lat, sweeps, conv = [], 0, 0
        for (n, _, _), t in zip(reqs, tickets):
            st, res = ctx.wait(t, 600.0)
            if st != capi.SOR_OK:
                raise capi.SorError(st, ctx.last_error())
            lat.append(res["latency_s"])
            sweeps += res["iterations"] * n * n
            conv += res["converged"]
        dt = time.perf_counter() - t0
        if rep > 0 and (best is None or dt < best[0]):
            best = (dt, lat, sweeps, conv)
    dt, lat, lups, conv = best
    cpu = None
    if not args.no_cpu_baseline:
        import oracle
        oracle.build()
        done, t_all, cells = 0, 0.0, 0.0
        for n, u0, _ in reqs:
            t = time.perf_counter()
            r = oracle.refine(u0, oracle.omega_opt(n), inner_sweeps=20, tol=1e-10, max_outer=100000)
            t_all += time.perf_counter() - t
            done += 1
            cells += float(n) ** 2 * r["sweeps"]
            if t_all > args.cpu_budget_s:
                break
        cpu = {"value": done / t_all, "unit": "solves/s", "cores": 1, "kind": "oracle",
               "sweep_glups": cells / t_all / 1e9,
               "sample": f"the oracle's defect correction on the first {done} plates of the batch "
                         f"(N = {[int(x[0]) for x in reqs[:done]]}), {t_all:.1f} s"}
    return {"metric": "solves/s, 512 heat plates (N log-uniform 64..1024) to 1e-10 relative residual",
            "value": count / dt, "unit": "solves/s", "higher_is_better": True,
            "detail": {"makespan_s": dt, "converged": conv, "count": count, "glups": lups / dt / 1e9,
                       "latency_p50_s": _pct(lat, 50), "latency_p99_s": _pct(lat, 99)},
            "cpu_baseline": cpu,
            "config": {"workload": f"{count} plates, seed {args.seed}, FP32 sweeps + FP64 correction, inner 20"}}


def _accuracy(recs):
    """How the requests ended: converged below their tolerance, or stopped by the stall rule at the
    attainable floor (FP64 storage cannot hold a relative residual much below ~8 eps max|u| / max|h^2 f|,
    which grows like (N+1)^2), with the worst final relative residuals."""
    conv = [r for r in recs if r["converged"]]
    stalled = [r for r in recs if not r["converged"]]
    out = {"requests": len(recs), "converged": len(conv), "stopped_by_stall_rule": len(stalled)}
    if conv:
        out["worst_converged_resid_over_tol"] = max(r["resid"] / r["tol"] for r in conv)
    if stalled:
        w = max(stalled, key=lambda r: r["resid"])
        out["worst_stalled"] = {"final_resid_rel": w["resid"], "tol": w["tol"], "n": w["n"]}
        out["stalled_n_min"] = min(r["n"] for r in stalled)
        out["stalled_tol_max"] = max(r["tol"] for r in stalled)
    return out


def workload_serve(args, ctx, capi, wl):
    """Poisson arrivals of solve requests (N log-uniform 128..4096, tolerance log-uniform 1e-10..1e-6,
    Gaussian-sum source, random edges) at a mean rate, served by continuous batching (FP32 sweeps + FP64
    defect correction) under a 150 GB budget, against one-at-a-time plain FP64 solves on the same GPU.

    Open loop: request k is due at its scheduled arrival t_k; the client submits it once it is due and
    fewer than --outstanding requests are in the library, and its latency is completion - t_k, so time
    spent waiting for a place counts like time in the server's own queue.  Inputs are generated just
    before submission by a pool of threads running ahead (10,000 requests of up to 4098^2 do not fit in
    host memory at once).  The one-at-a-time arm serves the first --fp64-sample requests in arrival order
    with blocking plain FP64 solves (residual test every 20 iterations), in real time from the same
    scheduled arrivals.  Both arms report how each request ended (see _accuracy)."""
    import concurrent.futures as cf

    import numpy as np
    count = args.count or 1000
    rate = args.rate
    limit = max(1, args.outstanding)
    reqs = wl.request_stream(count, rate, args.seed)

    def prep(k):
        u0, f = wl.request_inputs(reqs[k])
        return np.ascontiguousarray(u0), np.ascontiguousarray(f)

    ahead = min(count, max(8, min(limit, 48)))
    pool = cf.ThreadPoolExecutor(max_workers=args.gen_threads)
    futs = {k: pool.submit(prep, k) for k in range(ahead)}
    next_prep = ahead
    outstanding = {}
    recs = [None] * count
    t0 = time.perf_counter()
    k = 0
    while k < count or outstanding:
        progressed = False
        for t in list(outstanding):
            st, res = ctx.poll(t)
            if st == capi.SOR_NOT_READY:
                continue
            if st != capi.SOR_OK:
                raise capi.SorError(st, ctx.last_error())
            kk, t_sub = outstanding.pop(t)
            r = reqs[kk]
            done = t_sub + res["latency_s"]
            recs[kk] = {"latency": done - r.arrival_s, "done": done, "converged": bool(res["converged"]),
                        "resid": res["final_resid_rel"], "tol": r.tol, "n": r.n, "sweeps": res["iterations"]}
            progressed = True
        now = time.perf_counter() - t0
        if k < count and len(outstanding) < limit and reqs[k].arrival_s <= now:
            u0, f = futs.pop(k).result()
            if next_prep < count:
                futs[next_prep] = pool.submit(prep, next_prep)
                next_prep += 1
            t_sub = time.perf_counter() - t0
            ticket, _ = ctx.submit(u0, f, precision=capi.SOR_FP32_REFINE, omega=capi.sor_omega_opt(reqs[k].n),
                                   tol=reqs[k].tol, max_iters=2000000, inner_sweeps=20, stall_window=50)
            outstanding[ticket] = (k, t_sub)
            k += 1
            progressed = True
        if not progressed:
            time.sleep(0.0005)
    pool.shutdown()
    lat = [r["latency"] for r in recs]
    makespan = max(r["done"] for r in recs) - reqs[0].arrival_s
    cells = sum(float(r["n"]) ** 2 * r["sweeps"] for r in recs)
    served = {"p50_s": _pct(lat, 50), "p99_s": _pct(lat, 99), "max_s": max(lat),
              "achieved_solves_per_s": count / makespan, "makespan_s": makespan,
              "offered_rate_per_s": rate, "offered_span_s": reqs[-1].arrival_s - reqs[0].arrival_s,
              "sweep_glups": cells / makespan / 1e9, "accuracy": _accuracy(recs),
              "outstanding_limit": limit}
    # one at a time, plain FP64 with the residual test every 20 iterations, real time
    sub = min(count, args.fp64_sample)
    recs64 = []
    pool = cf.ThreadPoolExecutor(max_workers=args.gen_threads)
    futs = {kk: pool.submit(prep, kk) for kk in range(min(sub, 8))}
    for kk in range(min(sub, 8)):
        futs[kk].result()  # inputs of the first requests ready before the clock starts
    t0 = time.perf_counter()
    busy = 0.0
    for kk, r in enumerate(reqs[:sub]):
        now = time.perf_counter() - t0
        if r.arrival_s > now:
            time.sleep(r.arrival_s - now)
        u0, f = futs.pop(kk).result()
        if kk + 8 < sub:
            futs[kk + 8] = pool.submit(prep, kk + 8)
        ts = time.perf_counter()
        _, res = ctx.solve(u0, f, precision=capi.SOR_FP64, omega=capi.sor_omega_opt(r.n), tol=r.tol,
                           max_iters=2000000, check_every=20, stop=capi.SOR_STOP_RESID_REL, stall_window=50)
        te = time.perf_counter()
        busy += te - ts
        recs64.append({"latency": te - t0 - r.arrival_s, "done": te - t0, "converged": bool(res["converged"]),
                       "resid": res["final_resid_rel"], "tol": r.tol, "n": r.n, "sweeps": res["iterations"]})
    pool.shutdown()
    lat64 = [r["latency"] for r in recs64]
    span64 = recs64[-1]["done"] - reqs[0].arrival_s
    fp64 = {"p50_s": _pct(lat64, 50), "p99_s": _pct(lat64, 99), "achieved_solves_per_s": sub / span64,
            "requests": sub, "mean_service_s": busy / sub, "accuracy": _accuracy(recs64),
            "note": "the first requests of the same stream, served in arrival order by blocking solves"}
    # the same first requests through the batching arm, for a like-for-like capacity figure
    head = recs[:sub]
    served["first_requests_mean_latency_s"] = float(np.mean([r["latency"] for r in head]))
    cpu = None
    if not args.no_cpu_baseline:
        cpu = _oracle_requests(reqs, wl, args.cpu_budget_s)
    return {"metric": "p99 latency of served solves (Poisson arrivals) to their tolerance",
            "value": served["p99_s"], "unit": "s", "higher_is_better": False,
            "detail": {"continuous_batching_fp32_refine": served, "one_at_a_time_fp64": fp64,
                       "offered_rate_per_s": rate, "requests": count},
            "cpu_baseline": cpu,
            "config": {"workload": f"{count} requests, rate {rate}/s, seed {args.seed}, budget 150 GB, "
                                   f"at most {limit} outstanding in the library"}}


def _oracle_requests(reqs, wl, budget_s):
    """The oracle's defect correction (FP32 sweeps, FP64 residual and correction, one host core) on the
    first requests of the stream with N <= 1024, in order, until about budget_s seconds have passed."""
    import oracle
    oracle.build()
    done, cells, t_all, ns = 0, 0.0, 0.0, []
    for r in reqs:
        if r.n > 1024:
            continue
        u0, f = wl.request_inputs(r)
        w = oracle.omega_opt(r.n)
        t = time.perf_counter()
        res = oracle.refine(u0, w, f=f, inner_sweeps=20, tol=r.tol, max_outer=100000, stall_window=50)
        t_all += time.perf_counter() - t
        done += 1
        cells += float(r.n) ** 2 * res["sweeps"]
        ns.append(r.n)
        if t_all > budget_s:
            break
    return {"value": done / t_all if t_all else None, "unit": "solves/s", "cores": 1, "kind": "oracle",
            "sweep_glups": cells / t_all / 1e9 if t_all else None,
            "sample": f"the first {done} requests with N <= 1024 (N = {ns}), {t_all:.1f} s"}


def workload_paper(args, ctx, capi, wl):
    """The paper's own experiment (Section 3.4, Section 4): 4096x4096 plate, north edge 1.0, the others 0,
    w = 0.376, stop when max|change| < 1e-5 checked every K = 4000 iterations, at most 50000 iterations,
    FP64.  Table 1's times (unnamed multicore host) are context: the speedup is reported against them."""
    import json as _json
    import torch
    n = 4096
    with open(os.path.join(ROOT, "tests", "golden", "paper_constants.json")) as fh:
        pc = _json.load(fh)
    u0 = torch.from_numpy(wl.heat_plate(n, pc["north_boundary"])).cuda()
    out = torch.empty_like(u0)
    kw = dict(omega=pc["omega"], tol=pc["epsilon"], max_iters=pc["max_iterations"], check_every=pc["K"])
    ctx.solve(u0, out=out, **dict(kw, max_iters=pc["K"]))  # warm-up: workspace, graphs
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    _, res = ctx.solve(u0, out=out, **kw)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    table = {row["threads"]: row["time_s"] for row in pc["table1"]}
    best = min(table[8].values())
    return {"metric": "time to solution of the paper's 4096^2 heat plate (w = 0.376, eps = 1e-5, K = 4000)",
            "value": dt, "unit": "s", "higher_is_better": False,
            "detail": {"iterations": res["iterations"], "converged": res["converged"],
                       "final_maxdelta": res["final_maxdelta"], "glups": float(n) * n * res["iterations"] / dt / 1e9,
                       "paper_table1_best_8_threads_s": best, "speedup_vs_paper_best": best / dt,
                       "paper_table1_serial_chapel_s": table[1]["chapel"]},
            "config": {"workload": "4096^2 interior, north 1.0, w 0.376, eps 1e-5, K 4000, cap 50000, FP64"}}


def workload_plate16384(args, ctx, capi, wl):
    """The default plate scaled to 16386^2 (16384^2 interior): the colour-split state (2.1 GB FP64, 1.1 GB
    FP32) is far larger than the 129 MB L2, so the FP32 line is a clean HBM measurement.  200 iterations with
    max|change| every 50, device-resident inputs, FP64 (default path) and FP32 (fused depth 6)."""
    import numpy as np
    import torch
    n, iters = 16384, 200
    u0 = torch.from_numpy(wl.random_edges(n, args.seed)).cuda()
    out = torch.empty_like(u0)
    w = capi.sor_omega_opt(n)
    lines = {}
    for name, prec in (("fp64", capi.SOR_FP64), ("fp32", capi.SOR_FP32)):
        kw = dict(precision=prec, omega=w, tol=-1.0, max_iters=iters, check_every=50)
        for _ in range(args.warmup):
            ctx.solve(u0, out=out, **dict(kw, max_iters=50))
        torch.cuda.synchronize()
        dev = []
        t0 = time.perf_counter()
        for _ in range(args.steps):
            _, res = ctx.solve(u0, out=out, **kw)
            dev.append(res["device_s"])
        torch.cuda.synchronize()
        dt = (time.perf_counter() - t0) / args.steps
        lup = float(n) * n * iters
        lines[name] = {"glups": lup / float(np.median(dev)) / 1e9, "glups_call": lup / dt / 1e9,
                       "solve_s": dt, "iterations": res["iterations"]}
    peaks, src = measured_peaks()
    hbm = float(peaks.get("hbm_gbs") or 6800.0)
    ach64 = FP64_FLOPS_PER_LUP * lines["fp64"]["glups"] / 1e3
    lines["fp64"]["roofline"] = {"bound": "alu", "achieved": ach64, "peak": NOMINAL_FP64_TFLOPS, "unit": "TFLOP/s",
                                 "frac": ach64 / NOMINAL_FP64_TFLOPS, "kernel": "k_fast_chain<false>",
                                 "hbm_frac": HBM_BYTES_PER_LUP["f64"] * lines["fp64"]["glups"] / hbm}
    lines["fp32"]["roofline"] = {"bound": "hbm", "achieved": HBM_BYTES_PER_LUP["f32"] * lines["fp32"]["glups"],
                                 "peak": hbm, "unit": "GB/s",
                                 "frac": HBM_BYTES_PER_LUP["f32"] * lines["fp32"]["glups"] / hbm,
                                 "kernel": "k_sweep_tb<6,0>", "peak_source": src,
                                 "note": "8 B per update is the unfused traffic; the fused kernel moves less"}
    return {"metric": "red-black SOR GLUP/s, 16386^2 plate (state far above L2)", "value": lines["fp64"]["glups"],
            "unit": "GLUP/s", "higher_is_better": True, "dtype": "f64", "detail": lines,
            "config": {"workload": "16386^2 plate, random edges U[0,100], w_opt, 200 iterations, max|change| every 50",
                       "l2": "colour-split state 2.1 GB (FP64) / 1.1 GB (FP32), far above the 129 MB L2"}}


def workload_cube256(args, ctx, capi, wl):
    """3D red-black SOR (7-point stencil, the paper's next step, Section 5): 258^3 cube, shell values
    i.i.d. U[0, 100], interior 0, f = 0, w_opt, 1000 iterations with max|change| every 50, device-resident
    inputs.  Lines: FP64 default (rescaled unknowns, shared pair sums, within 1e-12 of the oracle), FP64
    exact order and FP32 (both bitwise equal to the oracle); FP32 at each cube depth (iterations fused per
    blocked launch, 1 and 2; the default 0 = one data-flow launch per run of iterations).  The
    oracle is timed on 10 iterations of the same cube on one host core."""
    import numpy as np
    import torch

    import oracle
    n, iters = 256, 1000
    u0_np = wl.random_shell(n, args.seed)
    u0 = torch.from_numpy(u0_np).cuda()
    out = torch.empty_like(u0)
    w = capi.sor_omega_opt(n)
    lines = {}
    for name, prec, flags, depth in (("fp64", capi.SOR_FP64, 0, 0),
                                     ("fp64_exact", capi.SOR_FP64, capi.SOR_FLAG_EXACT_ORDER, 0),
                                     ("fp32", capi.SOR_FP32, 0, 0), ("fp32_blocked1", capi.SOR_FP32, 0, 1),
                                     ("fp32_blocked2", capi.SOR_FP32, 0, 2)):
        ctx.set_option(capi.SOR_OPT_CUBE_DEPTH, depth)
        kw = dict(precision=prec, omega=w, tol=0.0, max_iters=iters, check_every=50, flags=flags)
        for _ in range(args.warmup):
            ctx.solve3d(u0, out=out, **dict(kw, max_iters=100))
        torch.cuda.synchronize()
        dev = []
        t0 = time.perf_counter()
        for _ in range(args.steps):
            _, res = ctx.solve3d(u0, out=out, **kw)
            dev.append(res["device_s"])
        torch.cuda.synchronize()
        dt = (time.perf_counter() - t0) / args.steps
        lup = float(n) ** 3 * iters
        lines[name] = {"glups": lup / float(np.median(dev)) / 1e9, "glups_call": lup / dt / 1e9,
                       "solve_s": dt, "iterations": res["iterations"]}
    ctx.set_option(capi.SOR_OPT_CUBE_DEPTH, 0)
    # FP64: 8 algorithmic flops per update ((1-w)u + (w/6)(sum of six neighbours): 5 adds, 2 multiplies,
    # 1 add); the default kernel issues 5 FP64 operations per update for them, the exact one 8
    for name, kern in (("fp64", "k_f3_flow"), ("fp64_exact", "k_3_flow<double>")):
        ach = 8.0 * lines[name]["glups"] / 1e3
        lines[name]["roofline"] = {"bound": "alu", "achieved": ach, "peak": NOMINAL_FP64_TFLOPS, "unit": "TFLOP/s",
                                   "frac": ach / NOMINAL_FP64_TFLOPS, "kernel": kern}
    # FP32: 8 B per update (read + write once per iteration) against measured HBM
    peaks, src = measured_peaks()
    hbm = float(peaks.get("hbm_gbs") or 6800.0)
    lines["fp32"]["roofline"] = {"bound": "hbm", "achieved": 8.0 * lines["fp32"]["glups"], "peak": hbm,
                                 "unit": "GB/s", "frac": 8.0 * lines["fp32"]["glups"] / hbm,
                                 "kernel": "k_3_flow<float>", "peak_source": src,
                                 "note": "unfused-equivalent bytes; the 69 MB FP32 state is L2-resident"}
    cpu = None
    if not args.no_cpu_baseline:
        k = 10
        t0 = time.perf_counter()
        oracle.sor3d_f64(u0_np, w, max_iters=k, check_every=50, tol=0.0)
        ct = time.perf_counter() - t0
        cpu = {"value": float(n) ** 3 * k / ct / 1e9, "unit": "GLUP/s", "cores": 1, "kind": "oracle",
               "sample": f"{k} FP64 iterations of the same 258^3 cube"}
    return {"metric": "3D red-black SOR GLUP/s (258^3 cube, 7-point stencil)", "value": lines["fp64"]["glups"],
            "unit": "GLUP/s", "higher_is_better": True, "dtype": "f64", "detail": lines, "cpu_baseline": cpu,
            "config": {"workload": "258^3 cube, shell U[0,100], w_opt, 1000 iterations, max|change| every 50",
                       "l2": "colour-split FP64 state 2 x 85 MB, above the 129 MB L2"}}


def workload_cube512(args, ctx, capi, wl):
    """FP32 red-black SOR on a 514^3 cube (state 0.6 GB per buffer pair, far above L2), shell U[0, 100],
    interior 0, f = 0, w_opt, 200 iterations with max|change| every 50, device-resident inputs, at each cube
    depth (0 = default, one data-flow launch per run of iterations; 1 and 2 = blocked sweeps)."""
    import numpy as np
    import torch
    n, iters = 512, 200
    u0 = torch.from_numpy(wl.random_shell(n, args.seed)).cuda()
    out = torch.empty_like(u0)
    w = capi.sor_omega_opt(n)
    lines = {}
    for name, depth in (("fp32", 0), ("fp32_blocked1", 1), ("fp32_blocked2", 2)):
        ctx.set_option(capi.SOR_OPT_CUBE_DEPTH, depth)
        kw = dict(precision=capi.SOR_FP32, omega=w, tol=0.0, max_iters=iters, check_every=50)
        for _ in range(args.warmup):
            ctx.solve3d(u0, out=out, **dict(kw, max_iters=50))
        torch.cuda.synchronize()
        dev = []
        for _ in range(args.steps):
            _, res = ctx.solve3d(u0, out=out, **kw)
            dev.append(res["device_s"])
        lup = float(n) ** 3 * iters
        g = lup / float(np.median(dev)) / 1e9
        lines[name] = {"glups": g, "device_s": float(np.median(dev)), "iterations": res["iterations"],
                       "unfused_equiv_gbs": 8.0 * g}
    ctx.set_option(capi.SOR_OPT_CUBE_DEPTH, 0)
    peaks, src = measured_peaks()
    hbm = float(peaks.get("hbm_gbs") or 6800.0)
    return {"metric": "FP32 3D red-black SOR GLUP/s (514^3 cube, 7-point stencil)", "value": lines["fp32"]["glups"],
            "unit": "GLUP/s", "higher_is_better": True, "dtype": "f32", "detail": lines,
            "roofline": {"bound": "hbm", "achieved": 8.0 * lines["fp32"]["glups"], "peak": hbm, "unit": "GB/s",
                         "frac": 8.0 * lines["fp32"]["glups"] / hbm, "kernel": "k_3_flow<float>",
                         "peak_source": src, "note": "unfused-equivalent bytes (8 per update)"},
            "config": {"workload": "514^3 cube, shell U[0,100], w_opt, 200 iterations, max|change| every 50",
                       "l2": "FP32 colour arrays 2 x 0.3 GB per buffer pair, far above the 129 MB L2"}}


def workload_cubepoisson(args, ctx, capi, wl):
    """3D Poisson on the 258^3 cube (zero shell, f = sum of 8 Gaussians, seeded) to a relative residual of
    1e-10: FP32 sweeps + FP64 defect correction (20 sweeps per correction, bitwise equal to the oracle)
    versus plain FP64 SOR (the default rescaled path) with the residual test every 20 iterations.  The
    oracle is timed on one outer step of its defect correction on the same cube, on one host core."""
    import numpy as np
    import torch

    import oracle
    n, tol = 256, 1e-10
    u0_np = np.zeros((n + 2,) * 3)
    f_np = wl.gaussian_source3(n, args.seed)
    u0 = torch.from_numpy(u0_np).cuda()
    f = torch.from_numpy(f_np).cuda()
    out = torch.empty_like(u0)
    w = capi.sor_omega_opt(n)
    runs = {"fp32_refine": dict(precision=capi.SOR_FP32_REFINE, omega=w, tol=tol, max_iters=40000, inner_sweeps=20),
            "fp64_plain": dict(precision=capi.SOR_FP64, omega=w, tol=tol, max_iters=40000, check_every=20,
                               stop=capi.SOR_STOP_RESID_REL)}
    detail = {}
    for name, kw in runs.items():
        for _ in range(args.warmup):
            ctx.solve3d(u0, f, out=out, **dict(kw, max_iters=200))
        torch.cuda.synchronize()
        times = []
        for _ in range(args.steps):
            t0 = time.perf_counter()
            _, res = ctx.solve3d(u0, f, out=out, **kw)
            torch.cuda.synchronize()
            times.append(time.perf_counter() - t0)
        dt = float(np.median(times))
        detail[name] = {"time_to_solution_s": dt, "device_s": res["device_s"], "sweeps": res["iterations"],
                        "outer_steps": res["outer_steps"], "final_resid_rel": res["final_resid_rel"],
                        "converged": res["converged"], "glups": float(n) ** 3 * res["iterations"] / dt / 1e9}
    detail["speedup_refine_vs_plain"] = (detail["fp64_plain"]["time_to_solution_s"] /
                                         detail["fp32_refine"]["time_to_solution_s"])
    cpu = None
    if not args.no_cpu_baseline:
        t0 = time.perf_counter()
        oracle.refine3d(u0_np, w, f=f_np, inner_sweeps=20, tol=-1.0, max_outer=1)
        ct = time.perf_counter() - t0
        cpu = {"value": float(n) ** 3 * 20 / ct / 1e9, "unit": "GLUP/s", "cores": 1, "kind": "oracle",
               "sample": "one outer step (residual, 20 FP32 sweeps, correction) of the same cube"}
    return {"metric": "time to solution, 258^3 Poisson cube (8 Gaussians) to relative residual 1e-10",
            "value": detail["fp32_refine"]["time_to_solution_s"], "unit": "s", "higher_is_better": False,
            "dtype": "f64", "detail": detail, "cpu_baseline": cpu,
            "config": {"workload": "258^3 cube, zero shell, f = 8-Gaussian sum (seeded), w_opt, inner 20 FP32 "
                                   "sweeps; plain FP64 tests the residual every 20 iterations"}}


def workload_ninepoisson(args, ctx, capi, wl):
    """Poisson with the compact 9-point stencil and four-colour SOR: 1026^2 plate, zero edges, f = sum of
    8 Gaussians (seeded), to a relative residual of 1e-9: FP32 four-colour sweeps + FP64 defect correction
    (20 sweeps per correction, bitwise equal to the oracle) versus plain FP64 four-colour SOR (the default
    shared-triple path) with the residual test every 20 iterations.  The oracle is timed on one outer step
    of its defect correction on the same plate, on one host core."""
    import numpy as np
    import torch

    import oracle
    n, tol = 1024, 1e-9
    u0_np, f_np = wl.poisson_problem(n, args.seed)
    u0 = torch.from_numpy(u0_np).cuda()
    f = torch.from_numpy(f_np).cuda()
    out = torch.empty_like(u0)
    w = capi.sor_omega_opt(n)
    runs = {"fp32_refine": dict(precision=capi.SOR_FP32_REFINE, omega=w, tol=tol, max_iters=60000, inner_sweeps=20),
            "fp64_plain": dict(precision=capi.SOR_FP64, omega=w, tol=tol, max_iters=60000, check_every=20,
                               stop=capi.SOR_STOP_RESID_REL)}
    detail = {}
    for name, kw in runs.items():
        for _ in range(args.warmup):
            ctx.solve9(u0, f, out=out, **dict(kw, max_iters=200))
        torch.cuda.synchronize()
        times = []
        for _ in range(args.steps):
            t0 = time.perf_counter()
            _, res = ctx.solve9(u0, f, out=out, **kw)
            torch.cuda.synchronize()
            times.append(time.perf_counter() - t0)
        dt = float(np.median(times))
        detail[name] = {"time_to_solution_s": dt, "device_s": res["device_s"], "sweeps": res["iterations"],
                        "outer_steps": res["outer_steps"], "final_resid_rel": res["final_resid_rel"],
                        "converged": res["converged"], "glups": float(n) * n * res["iterations"] / dt / 1e9}
    detail["speedup_refine_vs_plain"] = (detail["fp64_plain"]["time_to_solution_s"] /
                                         detail["fp32_refine"]["time_to_solution_s"])
    cpu = None
    if not args.no_cpu_baseline:
        t0 = time.perf_counter()
        oracle.refine9(u0_np, w, f=f_np, inner_sweeps=20, tol=-1.0, max_outer=1)
        ct = time.perf_counter() - t0
        cpu = {"value": float(n) * n * 20 / ct / 1e9, "unit": "GLUP/s", "cores": 1, "kind": "oracle",
               "sample": "one outer step (residual, 20 FP32 four-colour sweeps, correction) of the same plate"}
    return {"metric": "time to solution, 1026^2 Poisson plate, 9-point four-colour SOR, relative residual 1e-9",
            "value": detail["fp32_refine"]["time_to_solution_s"], "unit": "s", "higher_is_better": False,
            "dtype": "f64", "detail": detail, "cpu_baseline": cpu,
            "config": {"workload": "1026^2 plate, zero edges, f = 8-Gaussian sum (seeded), w = 2/(1+sin pi h), "
                                   "inner 20 FP32 sweeps; plain FP64 tests the residual every 20 iterations"}}


def workload_ninepoint4096(args, ctx, capi, wl):
    """Four-colour SOR on the compact 9-point stencil (multi-colour SOR, Section 3.1): the 4098^2 plate of
    the default workload (random edges U[0, 100], f = 0, w_opt), 1000 iterations with max|change| every 50,
    device-resident inputs.  Lines: FP64 default (shared north / south triples, within 1e-12 of the oracle),
    FP64 exact order and FP32 (both bitwise equal to the oracle).  The oracle is timed on 10 iterations of
    the same plate on one host core."""
    import numpy as np
    import torch

    import oracle
    n, iters = 4096, 1000
    u0_np = wl.random_edges(n, args.seed)
    u0 = torch.from_numpy(u0_np).cuda()
    out = torch.empty_like(u0)
    w = capi.sor_omega_opt(n)
    lines = {}
    for name, prec, flags in (("fp64", capi.SOR_FP64, 0), ("fp64_exact", capi.SOR_FP64, capi.SOR_FLAG_EXACT_ORDER),
                              ("fp32", capi.SOR_FP32, 0)):
        kw = dict(precision=prec, omega=w, tol=0.0, max_iters=iters, check_every=50, flags=flags)
        for _ in range(args.warmup):
            ctx.solve9(u0, out=out, **dict(kw, max_iters=100))
        torch.cuda.synchronize()
        dev = []
        t0 = time.perf_counter()
        for _ in range(args.steps):
            _, res = ctx.solve9(u0, out=out, **kw)
            dev.append(res["device_s"])
        torch.cuda.synchronize()
        dt = (time.perf_counter() - t0) / args.steps
        lup = float(n) * n * iters
        lines[name] = {"glups": lup / float(np.median(dev)) / 1e9, "glups_call": lup / dt / 1e9,
                       "solve_s": dt, "iterations": res["iterations"]}
    # FP64: 11 algorithmic flops per update (6 adds for the eight neighbours, 1 multiply by 4, 1 add,
    # 2 multiplies, 1 add); the default kernel issues 7 FP64 operations per update for them, the exact one 11
    for name, kern in (("fp64", "k_9_flow<double,FAST>"), ("fp64_exact", "k_9_flow<double,EXACT>")):
        ach = 11.0 * lines[name]["glups"] / 1e3
        lines[name]["roofline"] = {"bound": "alu", "achieved": ach, "peak": NOMINAL_FP64_TFLOPS, "unit": "TFLOP/s",
                                   "frac": ach / NOMINAL_FP64_TFLOPS, "kernel": kern}
    peaks, src = measured_peaks()
    hbm = float(peaks.get("hbm_gbs") or 6800.0)
    lines["fp32"]["roofline"] = {"bound": "hbm", "achieved": 8.0 * lines["fp32"]["glups"], "peak": hbm,
                                 "unit": "GB/s", "frac": 8.0 * lines["fp32"]["glups"] / hbm,
                                 "kernel": "k_9_flow<float,EXACT>", "peak_source": src}
    cpu = None
    if not args.no_cpu_baseline:
        k = 10
        t0 = time.perf_counter()
        oracle.sor9_f64(u0_np, w, max_iters=k, check_every=50, tol=0.0)
        ct = time.perf_counter() - t0
        cpu = {"value": float(n) * n * k / ct / 1e9, "unit": "GLUP/s", "cores": 1, "kind": "oracle",
               "sample": f"{k} FP64 iterations of the same 4098^2 plate"}
    return {"metric": "four-colour 9-point SOR GLUP/s (4098^2 plate)", "value": lines["fp64"]["glups"],
            "unit": "GLUP/s", "higher_is_better": True, "dtype": "f64", "detail": lines, "cpu_baseline": cpu,
            "config": {"workload": "4098^2 plate, random edges U[0,100], w_opt, 1000 iterations, max|change| every 50",
                       "l2": "4 quarter arrays of 34 MB FP64 (134 MB in all), above the 129 MB L2"}}


def workload_block4096(args, ctx, capi, wl):
    """Block two-colour SOR (the block-parallel SOR of Section 3.1: blocks of by x bx cells coloured (I + J)
    mod 2, colour 0 first, row-major order inside a block) on the 4098^2 plate of the default workload
    (random edges U[0, 100], f = 0, w_opt), 1000 iterations with max|change| every 50, device-resident inputs,
    FP64 in the exact order (bitwise equal to the oracle), for six block shapes, and in FP32 for two.  The oracle is
    timed on 10 iterations of the same plate on one host core."""
    import numpy as np
    import torch

    import oracle
    n, iters = 4096, 1000
    u0_np = wl.random_edges(n, args.seed)
    u0 = torch.from_numpy(u0_np).cuda()
    out = torch.empty_like(u0)
    w = capi.sor_omega_opt(n)
    lines = {}
    for by, bx in ((32, 32), (32, 64), (32, 128), (16, 64), (16, 128), (8, 64)):
        kw = dict(block_rows=by, block_cols=bx, precision=capi.SOR_FP64, omega=w, tol=0.0, max_iters=iters,
                  check_every=50)
        for _ in range(args.warmup):
            ctx.solve_block(u0, out=out, **dict(kw, max_iters=100))
        torch.cuda.synchronize()
        dev = []
        t0 = time.perf_counter()
        for _ in range(args.steps):
            _, res = ctx.solve_block(u0, out=out, **kw)
            dev.append(res["device_s"])
        torch.cuda.synchronize()
        dt = (time.perf_counter() - t0) / args.steps
        lup = float(n) * n * iters
        glups = lup / float(np.median(dev)) / 1e9
        # 6 algorithmic FP64 flops per update (3 adds of the neighbours, 2 multiplies, 1 add), all issued
        ach = 6.0 * glups / 1e3
        # columns of a warp segment's run of blocks (the library's default choice)
        k = max(1, 128 // bx)
        if (k * bx) / (k * bx + by - 1.0) < 1.15 * bx / (bx + by - 1.0):
            k = 1
        run_cols = k * bx
        lines[f"{by}x{bx}"] = {"glups": glups, "glups_call": lup / dt / 1e9, "solve_s": dt,
                               "iterations": res["iterations"], "wavefront_lane_use": run_cols / (run_cols + by - 1.0),
                               "roofline": {"bound": "alu", "achieved": ach, "peak": NOMINAL_FP64_TFLOPS,
                                            "unit": "TFLOP/s", "frac": ach / NOMINAL_FP64_TFLOPS,
                                            "kernel": "k_blk_phase<false,*>"}}
    best = max(lines, key=lambda k: lines[k]["glups"])
    # the same iterations in FP32 storage and arithmetic (bitwise equal to the FP32 oracle)
    for by, bx in ((16, 128), (32, 128)):
        kw = dict(block_rows=by, block_cols=bx, precision=capi.SOR_FP32, omega=w, tol=0.0, max_iters=iters,
                  check_every=50)
        for _ in range(args.warmup):
            ctx.solve_block(u0, out=out, **dict(kw, max_iters=100))
        torch.cuda.synchronize()
        dev = []
        for _ in range(args.steps):
            _, res = ctx.solve_block(u0, out=out, **kw)
            dev.append(res["device_s"])
        lines[f"fp32_{by}x{bx}"] = {
            "glups": float(n) * n * iters / float(np.median(dev)) / 1e9, "iterations": res["iterations"],
            "hbm_gbs_unfused": 8.0 * float(n) * n * iters / float(np.median(dev)) / 1e9,
            "note": "FP32 storage, blocks staged in shared memory; device time of the iterations (the rounding of "
                    "u0 to FP32 and the widening of the result excluded)"}
    cpu = None
    if not args.no_cpu_baseline:
        k = 10
        t0 = time.perf_counter()
        oracle.sor_block_f64(u0_np, w, by=32, bx=128, max_iters=k, check_every=50, tol=0.0)
        ct = time.perf_counter() - t0
        cpu = {"value": float(n) * n * k / ct / 1e9, "unit": "GLUP/s", "cores": 1, "kind": "oracle",
               "sample": f"{k} iterations of the same 4098^2 plate, blocks of 32 x 128"}
    return {"metric": "block two-colour SOR GLUP/s (4098^2 plate)", "value": lines[best]["glups"],
            "unit": "GLUP/s", "higher_is_better": True, "dtype": "f64", "detail": lines, "best_shape": best,
            "cpu_baseline": cpu,
            "config": {"workload": "4098^2 plate, random edges U[0,100], w_opt, 1000 iterations, max|change| every "
                                   "50, blocks of 32 x 32, 32 x 64, 32 x 128, 16 x 64, 16 x 128 and 8 x 64 cells",
                       "l2": "one 134 MB FP64 array, above the 129 MB L2"}}


def workload_fp64rate(args, ctx, capi, wl):
    """The FP64 peak of this GPU as sor_diag_fp64_rate measures it (independent chains of FP64 FMAs and of
    additions on a full-occupancy grid, CUDA-event timed), repeated `steps` times, next to the nominal rate."""
    import torch
    props = torch.cuda.get_device_properties(0)
    fma = [ctx.diag_fp64_rate(0) for _ in range(max(1, args.steps))]
    add = [ctx.diag_fp64_rate(1) for _ in range(max(1, args.steps))]
    nominal = props.multi_processor_count * 2 * 2.07e9
    return {"metric": "FP64 lane operations per second (independent chains, whole GPU)",
            "value": max(fma), "unit": "ops/s", "higher_is_better": True, "dtype": "f64",
            "detail": {"fma_ops_per_s": fma, "add_ops_per_s": add, "fma_tflops": 2.0 * max(fma) / 1e12,
                       "nominal_ops_per_s": nominal, "fma_frac_of_nominal": max(fma) / nominal,
                       "add_frac_of_nominal": max(add) / nominal, "sms": props.multi_processor_count},
            "config": {"workload": "8 blocks x 256 threads per SM, 8 chains per thread, 16384 steps per chain"}}


WORKLOADS = {"paper": workload_paper, "fp64rate": workload_fp64rate, "plate256": workload_plate256, "poisson4096": workload_poisson4096, "batch512": workload_batch512,
             "serve": workload_serve, "cube256": workload_cube256, "ninepoint4096": workload_ninepoint4096,
             "cubepoisson": workload_cubepoisson, "ninepoisson": workload_ninepoisson,
             "plate16384": workload_plate16384, "cube512": workload_cube512, "block4096": workload_block4096}


def run_workload(args):
    import torch

    from paper_1401_0763_gb300 import capi
    from paper_1401_0763_gb300 import workloads as wl
    capi.load()
    budget = 150 << 30 if args.workload == "serve" else 0
    with capi.Context(0, budget) as ctx:
        ctx.set_option(capi.SOR_OPT_TEMPORAL_DEPTH, args.tdepth)
        line = WORKLOADS[args.workload](args, ctx, capi, wl)
        torch.cuda.synchronize()
    line.update({"n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "data": "synthetic",
                 "workload_key": args.workload})
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-iters", type=int, default=150)
    ap.add_argument("--allcore-iters", type=int, default=200, help="iterations of the all-core CPU sample")
    ap.add_argument("--ref-iters", type=int, default=50)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--tdepth", type=int, default=0, help="FP32 iterations fused per tile pass (0 = library default)")
    ap.add_argument("--workload", default="plate4096", choices=["plate4096"] + sorted(WORKLOADS),
                    help="plate4096 is the default benchmark line; the others print their own line")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--count", type=int, default=0, help="batch512 / serve: number of grids or requests")
    ap.add_argument("--rate", type=float, default=50.0, help="serve: mean arrival rate per second")
    ap.add_argument("--fp64-sample", type=int, default=100, help="serve: requests served one at a time in FP64")
    ap.add_argument("--outstanding", type=int, default=96, help="serve: most requests in the library at once")
    ap.add_argument("--gen-threads", type=int, default=4, help="serve: threads generating request inputs")
    ap.add_argument("--cpu-budget-s", type=float, default=20.0, help="batch512 / serve: oracle sample time")
    args = ap.parse_args()
    ws, rank, local = dist_env()
    if args.impl == "reference":
        return run_reference(args, ws, rank)
    from paper_1401_0763_gb300 import _build
    _build.build()
    if args.workload != "plate4096":
        return run_workload(args) if rank == 0 else 0
    return run_ours(args, ws, rank, local)


if __name__ == "__main__":
    sys.exit(main())
