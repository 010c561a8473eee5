"""Benchmark of the periodic 1D heat stencil (Eq. 2, Section 2) on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--form auto|plain|persist|tblock]
                    [--T depth] [--dtype f64|f32c] [--workload ring-2^28-f64|...] [--impl ours|reference]

One bench step is one pass of the whole hot path over one batch of synthetic
input: load the initial state from a device-resident copy (heat_set_device),
advance nt steps (heat_run), take the FP64 conservation sum (heat_sum).  The
metric is GLUP/s = ring points x time steps / second (the paper's "cells
processed per second", Section 6).  Rank 0 prints one JSON line.

Under torchrun (N > 1) every rank runs its own independent replica of the
workload on its own GPU (the ring is not sharded across GPUs): weak scaling, no
data-path collective; `value` is all ranks' point-steps over the slowest rank's
time.  ``--impl reference`` times the CPU oracle (single thread) on a bounded
sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "FP64 GLUP/s (ring point-steps per second)"
METRIC_F32C = "binary32-compensated GLUP/s (ring point-steps per second)"
UNIT = "GLUP/s"

# name -> (nx, np, nt, k, dt, dx, initial condition, dtype)
WORKLOADS = {
    # np=256 partitions x nx=2^20 points (N = 2^28, 2.1 GB per binary64 buffer), nt=1000, r=0.25,
    # u0 = U[0,1) from PCG64 seed 0 plus the Fourier mode m=3 of amplitude 1
    "ring-2^28-f64": dict(nx=1 << 20, np=256, nt=1000, k=0.25, dt=1.0, dx=1.0, init="uniform+mode3", dtype="f64"),
    # the paper's shape (Section 6): 1e6 nodes, 1000 steps, u0[g] = g
    "ring-1e6-f64": dict(nx=250000, np=4, nt=1000, k=0.25, dt=1.0, dx=1.0, init="ramp", dtype="f64"),
    # np=4 x nx=1000, nt=100, k=0.5 (r=0.5), u0[g] = g
    "ring-4000-f64": dict(nx=1000, np=4, nt=100, k=0.5, dt=1.0, dx=1.0, init="ramp", dtype="f64"),
    # profiling case: np=32 x nx=2^20 (N = 2^25, 268 MB per buffer, still larger than L2), nt=20
    "ring-2^25-f64": dict(nx=1 << 20, np=32, nt=20, k=0.25, dt=1.0, dx=1.0, init="uniform+mode3", dtype="f64"),
    # binary32 state with the compensated update, same ring as the first, r = 0.25
    "ring-2^28-f32c": dict(nx=1 << 20, np=256, nt=1000, k=0.25, dt=1.0, dx=1.0, init="modes1,7,64", dtype="f32c"),
}
DEFAULT_WORKLOAD = "ring-2^28-f64"

# DP instructions per point-step of the binary64 update (exact reading: fma, add, mul, add;
# fused reading: fma, add, fma); binary32-compensated: about 14 FP32 operations.
DP_OPS = {0: 4, 1: 3}


def initial_state(w: dict) -> np.ndarray:
    from paper_2307_01117_gb300 import workloads
    n = w["nx"] * w["np"]
    if w["init"] == "ramp":
        return workloads.ramp(n, w["dx"])
    if w["init"] == "uniform+mode3":
        return workloads.uniform_plus_mode(n, seed=0, m=3)
    if w["init"].startswith("modes"):
        return workloads.modes(n, [int(m) for m in w["init"][5:].split(",")])
    raise ValueError(w["init"])


def peaks() -> dict:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return {"hbm_gbs": float(d["hbm_gbs"]), "sm_max_mhz": float(d.get("sm_max_mhz", 2070.0)), "src": "measured"}
    return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0, "src": "fallback"}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines: list[str] = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
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
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def profile_traffic(kernel: str, workload: str, src_files: list[str]) -> float | None:
    """DRAM bytes per launch from the committed ncu summary, if the kernel source
    is unchanged since it was taken."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        rec = json.load(f).get(f"{kernel}@{workload}")
    if not rec:
        return None
    h = hashlib.sha256()
    for s in src_files:
        with open(os.path.join(ROOT, s), "rb") as f:
            h.update(f.read())
    if rec.get("source_sha256") != h.hexdigest():
        return None
    return float(rec["dram_bytes_per_launch"])


def cpu_baseline(w: dict, seconds: float = 12.0) -> dict:
    """The CPU oracle, as it stands, single-threaded on a bounded sample of the
    workload: the first 2^22 points of the ring's initial state treated as a
    ring of its own, stepped until about `seconds` have passed."""
    import oracle
    n = min(w["nx"] * w["np"], 1 << 22)
    w2 = dict(w)
    w2["nx"], w2["np"] = n, 1
    u0 = initial_state(w2)
    r = oracle.coef(w["k"], w["dt"], w["dx"])
    t0 = time.perf_counter()
    oracle.run(u0[: min(n, 1 << 16)], r, 2)
    steps, total = 0, 0.0
    chunk = 4
    u = u0
    while total < seconds:
        t0 = time.perf_counter()
        if w["dtype"] == "f32c":
            u = oracle.run_f32c(u, np.float32(r), chunk, 1)
        else:
            u = oracle.run(u, r, chunk)
        total += time.perf_counter() - t0
        steps += chunk
    return {"value": n * steps / total / 1e9, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{n} points x {steps} steps ({'binary32 compensated' if w['dtype'] == 'f32c' else 'binary64'}), "
                      f"{total:.1f} s on 1 host core"}


def run_reference(args, w: dict, rank: int, world: int) -> None:
    if rank != 0:
        return
    cb = cpu_baseline(w, seconds=max(2.0, 2.0 * args.steps))
    line = {"impl": "reference", "metric": METRIC, "value": cb["value"], "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": None, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64" if w["dtype"] == "f64" else "f32",
            "data": "synthetic", "config": {"workload": args.workload, **{k: w[k] for k in ("nx", "np", "nt", "k")}},
            "cpu_baseline": cb, "e2e": {"value": cb["value"], "unit": UNIT, "h2d_bytes_per_step": 0,
                                        "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main() -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS))
    ap.add_argument("--form", default="auto", choices=["auto", "plain", "persist", "tblock"])
    ap.add_argument("--T", type=int, default=0)
    ap.add_argument("--arith", default="exact", choices=["exact", "fma"])
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    w = dict(WORKLOADS[args.workload])

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        run_reference(args, w, rank, world)
        return 0

    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    from paper_2307_01117_gb300 import build as hbuild
    from paper_2307_01117_gb300 import heat as H
    if not os.path.exists(H.LIB_PATH):
        hbuild.build()

    n = w["nx"] * w["np"]
    nt = w["nt"]
    arith = H.HEAT_ARITH_FMA if args.arith == "fma" else H.HEAT_ARITH_EXACT
    u0 = initial_state(w)
    stream = torch.cuda.Stream()
    u0_dev = torch.from_numpy(u0).to(f"cuda:{local}")
    h = H.Heat(w["nx"], w["np"], w["k"], w["dt"], w["dx"], dtype=w["dtype"], form=args.form, T=args.T,
               arith=arith, stream=stream)
    ctx = h.ctx

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()

    def step(ev=None):
        H.heat_set_device(ctx, u0_dev)
        if ev is not None:
            ev[0].record(stream)
        H.heat_run(ctx, nt)
        if ev is not None:
            ev[1].record(stream)
        return H.heat_sum(ctx)   # synchronises the stream

    for _ in range(args.warmup):
        step()
    barrier()

    clocks = ClockSampler(local)
    clocks.start()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    t_start, t_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    t_start.record(stream)
    for i in range(args.steps):
        step(evs[i])
    t_end.record(stream)
    barrier()
    clk = clocks.stop()
    ms_total = t_start.elapsed_time(t_end)
    run_ms = [a.elapsed_time(b) for a, b in evs]

    ms_max = ms_total
    if dist is not None:
        t = torch.tensor([ms_total], device=f"cuda:{local}")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_max = float(t.item())
    ms_per_step = ms_max / args.steps
    point_steps = float(n) * nt
    value = world * point_steps * args.steps / (ms_max * 1e-3) / 1e9

    # which kernel dominates and how long one launch takes (CUDA events on the ctx stream)
    last = H.heat_last_run(ctx)
    form_used = last["form"]
    launches_per_run = max(1, last["launches"])
    kernel_ms = statistics.mean(run_ms) / launches_per_run
    pk = peaks()
    steps_per_launch = nt / launches_per_run
    units = float(n) * steps_per_launch          # point-steps per launch
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    kname = {("plain", "f64"): "k_plain_f64", ("plain", "f32c"): "k_plain_f32c", ("persist", "f64"): "k_persist",
             ("persist", "f32c"): "k_persist", ("tblock", "f64"): "k_tblock", ("tblock", "f32c"): "k_tblock"}[
        (form_used, w["dtype"])]
    srcs = {"k_plain_f64": ["k_plain.cu"], "k_plain_f32c": ["k_plain.cu"], "k_persist": ["k_persist.cu"],
            "k_tblock": ["k_tblock.cu"]}[kname]
    srcs = [f"paper_2307_01117_gb300/csrc/{x}" for x in srcs] + ["paper_2307_01117_gb300/csrc/stencil_ops.cuh"]
    # algorithmic HBM bytes: each point read once and written once per launch, whatever the steps per launch
    # (one-step forms: 16 B per point-step in binary64; forms that keep T steps on chip: 16/T)
    elem = 8.0 if w["dtype"] == "f64" else 4.0
    alg_bytes = 2.0 * elem * float(n) * (steps_per_launch if form_used == "persist" else 1.0)
    hbm_achieved = alg_bytes / (kernel_ms * 1e-3) / 1e9
    roof_hbm = {"bound": "hbm", "achieved": hbm_achieved, "peak": pk["hbm_gbs"], "unit": "GB/s",
                "frac": hbm_achieved / pk["hbm_gbs"], "peak_src": pk["src"], "alg_bytes_per_launch": alg_bytes}
    if w["dtype"] == "f64":
        dp_ops = DP_OPS[arith] * units
        # DP pipe: 2 lane-operations per clock per SM (GB300 nominal 1.25 TFLOP/s FP64 with FMA = 2 flops)
        dp_peak = 2.0 * sms * pk["sm_max_mhz"] * 1e6 / 1e9
        achieved = dp_ops / (kernel_ms * 1e-3) / 1e9
        roofline = {"bound": "alu", "achieved": achieved, "peak": dp_peak, "unit": "G DP-op/s",
                    "frac": achieved / dp_peak,
                    "peak_src": f"2 DP ops/clk/SM x {sms} SMs x {pk['sm_max_mhz']:.0f} MHz (max SM clock)",
                    "alg_ops_per_launch": dp_ops}
    else:
        roofline = dict(roof_hbm)
    roofline["traffic"] = profile_traffic(kname, args.workload, srcs)
    roofline["kernel"] = kname
    roofline["launch_ms"] = kernel_ms

    # end to end through the C ABI with host buffers: H2D of u0, run, sum, D2H of the state
    e2e = None
    if not args.no_e2e:
        host_in = torch.empty(n, dtype=torch.float64, pin_memory=True).numpy()
        host_in[:] = u0
        host_out = torch.empty(n, dtype=torch.float64, pin_memory=True).numpy()
        H.heat_set(ctx, host_in)
        H.heat_run(ctx, nt)
        H.heat_get(ctx, host_out)
        barrier()
        k_e2e = max(1, min(args.steps, 3))
        t0 = time.perf_counter()
        for _ in range(k_e2e):
            H.heat_set(ctx, host_in)
            H.heat_run(ctx, nt)
            H.heat_sum(ctx)
            H.heat_get(ctx, host_out)
        barrier()
        dt_e2e = time.perf_counter() - t0
        if dist is not None:
            t = torch.tensor([dt_e2e], device=f"cuda:{local}")
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            dt_e2e = float(t.item())
        e2e = {"value": world * point_steps * k_e2e / dt_e2e / 1e9, "unit": UNIT, "h2d_bytes_per_step": n * 8,
               "d2h_bytes_per_step": n * 8, "steps": k_e2e}

    cb = None
    if rank == 0 and not args.no_cpu_baseline:
        cb = cpu_baseline(w)

    launches = args.steps * (launches_per_run + 2)  # stencil launches + the two reduction kernels
    if rank == 0:
        line = {
            "metric": METRIC if w["dtype"] == "f64" else METRIC_F32C, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64" if w["dtype"] == "f64" else "f32", "data": "synthetic",
            "config": {"workload": args.workload, "nx": w["nx"], "np": w["np"], "N": n, "nt": nt, "k": w["k"],
                       "dt": w["dt"], "dx": w["dx"], "init": w["init"], "form": form_used, "T": last["T"],
                       "segments": last["segments"] if form_used != "plain" else None,
                       "arith": args.arith, "l2": "inputs larger than L2 (no flush needed)" if n * 8 > 2 * 135e6
                       else "L2-resident ring", "parallelism": "replicas" if world > 1 else "single GPU"},
            "roofline": roofline, "roofline_hbm": roof_hbm, "cpu_baseline": cb, "e2e": e2e,
            "gpu_launches": launches, "clocks": clk,
        }
        print(json.dumps(line), flush=True)
    h.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
