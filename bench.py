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
NOMINAL_FP64_TFLOPS = 1.25  # GB300 FP64 (non-tensor) nominal rate


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
    ms_max = ms
    if ws > 1:
        import torch.distributed as dist
        t = torch.tensor([ms], dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_max = float(t.item())
    lups_rank = float(N) * N * ITERS * args.steps
    value = ws * lups_rank / (ms_max * 1e-3) / 1e9
    launches = int(st["sweep_launches"]) + 3 * args.steps  # + pack, final residual, unpack per solve
    sweep_ms_per_launch = st["sweep_ms"] / max(1, st["timed_launches"])
    lups_per_launch = float(N) * N / 2.0  # one colour phase updates half the cells
    fp64_tflops = lups_per_launch * FP64_FLOPS_PER_LUP / (sweep_ms_per_launch * 1e-3) / 1e12
    hbm_gbs_fp64 = lups_per_launch * HBM_BYTES_PER_LUP["f64"] / (sweep_ms_per_launch * 1e-3) / 1e9
    peaks, peaks_src = measured_peaks()
    check = {"iterations": res["iterations"], "final_maxdelta": res["final_maxdelta"],
             "final_resid_rel": res["final_resid_rel"]}

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
    fp32 = {"value": lups_rank / (ms32 * 1e-3) / 1e9, "unit": "GLUP/s", "ms_per_step": ms32 / args.steps,
            "sweep_hbm_gbs": lups_per_launch * HBM_BYTES_PER_LUP["f32"] / (per32 * 1e-3) / 1e9}
    fp32["sweep_hbm_frac"] = fp32["sweep_hbm_gbs"] / peaks["hbm_gbs"]

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
    e2e_ms = max(e2.elapsed_time(e3), 1e3 * (time.perf_counter() - t0))
    if ws > 1:
        import torch.distributed as dist
        t = torch.tensor([e2e_ms], dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_ms = float(t.item())
    e2e = {"value": ws * lups_rank / (e2e_ms * 1e-3) / 1e9, "unit": "GLUP/s",
           "h2d_bytes_per_step": int(h_u0.numel() * 8), "d2h_bytes_per_step": int(h_out.numel() * 8)}
    assert np.isfinite(h_out.numpy()).all()

    # ---- CPU baseline: the oracle on a bounded sample (rank 0, N=1 only) ------------------------------------
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        v, dt = oracle_sample(args.cpu_iters)
        cpu = {"value": v, "unit": "GLUP/s", "cores": 1, "kind": "oracle",
               "sample": f"4096^2 plate, {args.cpu_iters} iterations ({dt:.1f} s, single thread)"}

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
            "roofline": {"bound": "alu", "achieved": fp64_tflops, "peak": NOMINAL_FP64_TFLOPS, "unit": "TFLOP/s",
                         "frac": fp64_tflops / NOMINAL_FP64_TFLOPS, "traffic": None,
                         "kernel": "k_sweep<double> (one colour phase)",
                         "peak_source": "nominal GB300 FP64 rate (recipe); probe measured 1.20",
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


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-iters", type=int, default=150)
    ap.add_argument("--ref-iters", type=int, default=50)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--tdepth", type=int, default=0, help="FP32 iterations fused per tile pass (0 = library default)")
    args = ap.parse_args()
    ws, rank, local = dist_env()
    if args.impl == "reference":
        return run_reference(args, ws, rank)
    from paper_1401_0763_gb300 import _build
    _build.build()
    return run_ours(args, ws, rank, local)


if __name__ == "__main__":
    sys.exit(main())
