"""Benchmark of the periodic 1D heat stencil (Eq. 2, Section 2) on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
                    [--form auto|plain|persist|tblock|cluster|persist_tb] [--T depth] [--arith exact|fma]
                    [--layout 0|1] [--split L] [--emul S] [--k K] [--impl ours|reference]
                    [--no-e2e] [--no-cpu-baseline] [--rate R] [--duration S] [--tick STEPS]

Workloads (all synthetic, seeded; the paper's own workload is synthetic too):
  ring-2^28-f64   (default) one ring, np = 256 x nx = 2^20, nt = 1000, r = 0.25,
                  u0 = U[0,1) + sin(2 pi 3 g / N)
  ring-1e6-f64    the paper's shape (Section 6): 10^6 points, 1000 steps, u0 = g
  ring-4000-f64   np = 4 x nx = 1000, nt = 100, r = 0.5, u0 = g
  ring-2^25-f64   profiling case (still larger than L2); ring-2^25-f32c likewise
  ring-2^28-f32c  binary32 compensated state, u0 = sum of modes 1, 7, 64
  batch-4096-f64  4096 independent rings, N log-uniform in [1e3, 1e6], np in
                  {1,2,4,8,16}, nt uniform in [100, 5000], r uniform in
                  [0.05, 0.5], u0 = U[-1,1) (seed 1), one persistent launch
  batch-256-f64   the first 256 rings of the same table
  batch-prof-f64  the same 256 rings with nt uniform in [100, 300] (profiling case)
  precision-2^28  binary32 compensated vs binary64 on the 2^28-point ring, nt = 10000,
                  u0 = modes 1, 7, 64; errors against a binary64 run and the closed form
  serve-100, serve-2000
                  Poisson request streams (100 or 2000 requests/s), N log-uniform in
                  [1e4, 1e7], nt uniform in [100, 2000], r uniform in [0.05, 0.5],
                  binary64 / binary32 compensated 50/50, 120 GB state budget; one
                  step = one arrival window; p50/p99 latency beside GLUP/s

One bench step is one pass of the whole hot path over one batch of input:
load the initial state from a device-resident copy, advance every ring its nt
steps, take the FP64 conservation sum (single ring) or synchronise (batch).
value = ring point-steps / second (GLUP/s, the paper's "cells processed per
second", Section 6), timed with CUDA events on the work's stream, 3+ warm-ups,
inputs larger than L2.  `e2e` is the same metric through the C ABI with host
buffers: every step's initial state is copied in from pinned host memory and
its final state read back inside the timed region (single rings: two contexts
on two streams take the steps in turn, so one context's copies run while the
other advances its ring).  `cpu_baseline` is the CPU oracle,
single-threaded, on a bounded sample; `cpu_threaded` is the paper's parallel
algorithm (one host thread per segment, SPSC ghost queues) on every host core,
on the same sample.  Binary64 ring lines also carry `plain`: the plain
one-step-per-launch kernel on the same ring in the same run (GLUP/s, its HBM
fraction at 16 B per point-step and its FP64-unit fraction); the default line
also carries `serving`: a 10 s window of 100 requests/s through the
continuous-batching server (p50/p99 latency, GLUP/s, backlog).

Under torchrun (N > 1) every rank runs its own independent replica on its own
GPU (replicas only: the ring is not sharded across GPUs): weak scaling, no
data-path collective; `value` is all ranks' point-steps over the slowest rank's
time.  ``--impl reference`` times the CPU oracle (single thread, on the host)
instead: W short warm-up samples, then K timed bounded samples of the workload
(about 2 s each); only rank 0 runs it.  Rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

UNIT = "GLUP/s"
METRIC = {"f64": "FP64 GLUP/s (ring point-steps per second)",
          "f32c": "binary32-compensated GLUP/s (ring point-steps per second)"}

WORKLOADS = {
    "ring-2^28-f64": dict(kind="ring", nx=1 << 20, np=256, nt=1000, k=0.25, dt=1.0, dx=1.0, init="uniform+mode3",
                          dtype="f64"),
    "ring-1e6-f64": dict(kind="ring", nx=250000, np=4, nt=1000, k=0.25, dt=1.0, dx=1.0, init="ramp", dtype="f64"),
    "ring-4000-f64": dict(kind="ring", nx=1000, np=4, nt=100, k=0.5, dt=1.0, dx=1.0, init="ramp", dtype="f64"),
    "ring-2^25-f64": dict(kind="ring", nx=1 << 20, np=32, nt=20, k=0.25, dt=1.0, dx=1.0, init="uniform+mode3",
                          dtype="f64"),
    "ring-2^25-f32c": dict(kind="ring", nx=1 << 20, np=32, nt=64, k=0.25, dt=1.0, dx=1.0, init="modes1,7,64",
                           dtype="f32c"),
    "ring-2^28-f32c": dict(kind="ring", nx=1 << 20, np=256, nt=1000, k=0.25, dt=1.0, dx=1.0, init="modes1,7,64",
                           dtype="f32c"),
    "batch-4096-f64": dict(kind="batch", count=4096, seed=1, dtype="f64"),
    # Poisson arrivals, N log-uniform in [1e4, 1e7], nt uniform in [100, 2000], r uniform in [0.05, 0.5],
    # binary64 or binary32-compensated 50/50, 120 GB state budget; one step = one arrival window
    "serve-2000": dict(kind="serve", rate=2000.0, duration=60.0, budget=120e9, seed=2, dtype="f64"),
    "serve-100": dict(kind="serve", rate=100.0, duration=30.0, budget=120e9, seed=2, dtype="f64"),
    "batch-256-f64": dict(kind="batch", count=256, seed=1, dtype="f64"),
    # profiling case: 256 rings of the same size law, nt uniform in [100, 300]
    "batch-prof-f64": dict(kind="batch", count=256, seed=1, dtype="f64", nt_lo=100, nt_hi=300),
    # binary32 compensated vs binary64 on np=256 x nx=2^20 (N = 2^28), nt = 10000, r = 0.25,
    # u0 = sum of modes 1, 7, 64: timed binary32 runs, then errors against a binary64 run
    # and the closed form sum_m lambda_m^nt sin(2 pi m g / N)
    "precision-2^28": dict(kind="precision", nx=1 << 20, np=256, nt=10000, k=0.25, dt=1.0, dx=1.0,
                           init="modes1,7,64", dtype="f32c", modes=(1, 7, 64)),
}
DEFAULT_WORKLOAD = "ring-2^28-f64"

# FP64-unit instructions per point-step: exact reading fma, add, mul, add; fused reading fma, add, fma
DP_OPS = {"exact": 4, "fma": 3}


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
        sm, smax, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
                power.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "power_w_median": statistics.median(power) if power else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def is_pow2(r: float) -> bool:
    m, _ = np.frexp(abs(r))
    return r != 0.0 and m == 0.5


ALU_OPS_SRC = ["paper_2307_01117_gb300/csrc/dp_emul.cuh", "paper_2307_01117_gb300/csrc/tb_core.cuh"]


def alu_ops(kind: str) -> float | None:
    """ALU-pipe instructions per point-step of the integer-pipe binary64 routine
    ("pow2": r = 2^k, "general"), measured with ncu on an all-integer launch and
    recorded in profiles/alu_ops.json; None if the routine changed since."""
    p = os.path.join(ROOT, "profiles", "alu_ops.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        rec = json.load(f).get(kind)
    if not rec:
        return None
    h = hashlib.sha256()
    for s in ALU_OPS_SRC:
        with open(os.path.join(ROOT, s), "rb") as f:
            h.update(f.read())
    return float(rec["alu_inst_per_point_step"]) if rec.get("source_sha256") == h.hexdigest() else None


def profile_traffic(kernel: str, workload: str, src_files: list[str]) -> float | None:
    """DRAM bytes per launch from the committed ncu summary (profiles/traffic.json),
    if the kernel's source is unchanged since the counters were taken."""
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


# ---------------------------------------------------------------------------------------------
# Replicas (N > 1): every rank runs the same workload on its own GPU

def reduce_max(x: float, dist, device) -> float:
    """Maximum of x over the ranks (x itself without a process group)."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(point_steps_per_step: float, steps: int, ms_max: float, world: int) -> float:
    """Whole-job GLUP/s: all ranks' point-steps over the slowest rank's time."""
    return world * point_steps_per_step * steps / (ms_max * 1e-3) / 1e9


# ---------------------------------------------------------------------------------------------
# CPU oracle baseline

def host_cpu() -> str:
    """The host CPU's model (from /proc/cpuinfo where it is there) and core count."""
    seen = {}
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if ":" in line:
                    key, val = (x.strip() for x in line.split(":", 1))
                    seen.setdefault(key.lower(), val)
    except OSError:
        pass
    import platform
    model = seen.get("model name") or " ".join(
        f"{k} {seen[k]}" for k in ("cpu implementer", "cpu part") if k in seen)
    return f"{model or platform.processor() or platform.machine()} ({platform.machine()}), {os.cpu_count()} cores"


def cpu_baseline(w: dict, seconds: float = 12.0) -> dict:
    """The CPU oracle, as it stands, single-threaded on a bounded sample of the
    workload, stepped until about `seconds` have passed."""
    import oracle
    if w["kind"] == "batch":
        from paper_2307_01117_gb300 import workloads
        specs = workloads.ring_table(w["count"], seed=w["seed"], nt_lo=w.get("nt_lo", 100), nt_hi=w.get("nt_hi", 5000))
        done_pts, total, rings = 0, 0.0, 0
        for spec in specs:
            if total >= seconds:
                break
            u0 = workloads.ring_initial(spec)
            t0 = time.perf_counter()
            oracle.run(u0, spec.r, spec.nt)
            total += time.perf_counter() - t0
            done_pts += spec.n * spec.nt
            rings += 1
        return {"value": done_pts / total / 1e9, "unit": UNIT, "cores": 1, "kind": "oracle", "host": host_cpu(),
                "sample": f"the first {rings} rings of the table, all their steps, {total:.1f} s on 1 host core"}
    n = min(w["nx"] * w["np"], 1 << 22)
    w2 = dict(w)
    w2["nx"], w2["np"] = n, 1
    u = initial_state(w2)
    r = oracle.coef(w["k"], w["dt"], w["dx"])
    steps, total, chunk = 0, 0.0, 4
    while total < seconds:
        t0 = time.perf_counter()
        if w["dtype"] == "f32c":
            u = oracle.run_f32c(u, np.float32(r), chunk, 1)
        else:
            u = oracle.run(u, r, chunk)
        total += time.perf_counter() - t0
        steps += chunk
    return {"value": n * steps / total / 1e9, "unit": UNIT, "cores": 1, "kind": "oracle", "host": host_cpu(),
            "sample": f"a ring of {n} points with the workload's initial-state recipe x {steps} steps "
                      f"({'binary32 compensated' if w['dtype'] == 'f32c' else 'binary64'}), {total:.1f} s on 1 host core"}


def cpu_threaded(w: dict, seconds: float = 8.0) -> dict | None:
    """The paper's parallel algorithm on every host core (oracle/heat_threaded.c:
    one thread per segment, mutex/condition-variable SPSC ghost queues, Section 2)
    on the same bounded sample as cpu_baseline; binary64 ring workloads only."""
    if w["kind"] not in ("ring",) or w["dtype"] != "f64":
        return None
    import oracle
    cores = os.cpu_count() or 1
    n = min(w["nx"] * w["np"], 1 << 22) // cores * cores
    w2 = dict(w)
    w2["nx"], w2["np"] = n, 1
    u = initial_state(w2)
    r = oracle.coef(w["k"], w["dt"], w["dx"])
    steps, total, chunk = 0, 0.0, 16
    while total < seconds:
        t0 = time.perf_counter()
        u = oracle.run_threaded(u, cores, r, chunk)
        total += time.perf_counter() - t0
        steps += chunk
    return {"value": n * steps / total / 1e9, "unit": UNIT, "cores": cores, "host": host_cpu(),
            "kind": "threaded SPSC-queue stepper (Section 2): one thread per segment",
            "sample": f"a ring of {n} points with the workload's initial-state recipe, {cores} segments x "
                      f"{steps} steps (binary64), {total:.1f} s on {cores} host cores"}


def cpu_report() -> dict:
    """CPU baselines on the paper-shaped configurations, each run in full: the
    oracle single-threaded on C0 (10^6 points x 1000 steps, u0 = g, r = 1/4; the
    paper's Fig. 3 workload, Section 6) and on C1 (np = 4 x nx = 1000, 100 steps,
    r = 1/2), and the threaded SPSC-queue stepper (Section 2) on C0 at the
    paper's thread counts 2, 20 and 40 (Section 5's T_average) and at the host's
    core count; counts above the core count oversubscribe the host."""
    import oracle
    from paper_2307_01117_gb300 import workloads
    out = {"host": host_cpu(), "cores": os.cpu_count()}

    def timed(fn):
        t0 = time.perf_counter()
        fn()
        return time.perf_counter() - t0

    u0 = workloads.ramp(10**6)
    t = timed(lambda: oracle.run(u0, 0.25, 1000))
    out["C0_oracle"] = {"N": 10**6, "nt": 1000, "threads": 1, "seconds": t, "glups": 1e9 / t / 1e9}
    u1 = workloads.ramp(4000)
    t = timed(lambda: oracle.run(u1, 0.5, 100))
    out["C1_oracle"] = {"N": 4000, "nt": 100, "threads": 1, "seconds": t, "glups": 4e5 / t / 1e9}
    rows = []
    for th in sorted({2, 20, 40, os.cpu_count() or 1}):
        n = 10**6 // th * th      # equal segments
        u = workloads.ramp(n)
        t = timed(lambda: oracle.run_threaded(u, th, 0.25, 1000))
        rows.append({"threads": th, "N": n, "nt": 1000, "seconds": t, "glups": n * 1000 / t / 1e9,
                     "oversubscribed": th > (os.cpu_count() or 1)})
    out["C0_threaded"] = rows
    return out


def _oracle_units(w: dict):
    """Endless stream of small pieces of the workload for the CPU oracle, each a
    call returning the point-steps it advanced, and a description of the sample:
    single rings take 4 steps at a time on a ring of min(N, 2^22) points built
    with the workload's initial-state recipe; batches and request streams visit
    their rings in table or arrival order, up to 32 steps each, then start over."""
    import oracle
    from paper_2307_01117_gb300 import workloads
    if w["kind"] in ("ring", "precision"):
        n = min(w["nx"] * w["np"], 1 << 22)
        w2 = dict(w)
        w2["nx"], w2["np"] = n, 1
        state = {"u": initial_state(w2)}
        r = oracle.coef(w["k"], w["dt"], w["dx"])
        f32 = w["dtype"] == "f32c"

        def unit():
            u = state["u"]
            state["u"] = oracle.run_f32c(u, np.float32(r), 4, 1) if f32 else oracle.run(u, r, 4)
            return 4 * n
        desc = (f"a ring of {n} points with the workload's initial-state recipe, 4 steps at a time "
                f"({'binary32 compensated' if f32 else 'binary64'})")
        while True:
            yield unit, desc
    if w["kind"] == "batch":
        specs = workloads.ring_table(w["count"], seed=w["seed"], nt_lo=w.get("nt_lo", 100), nt_hi=w.get("nt_hi", 5000))
        rings = [(s.n, s.nt, s.r, s.seed, False, lambda s=s: workloads.ring_initial(s)) for s in specs]
        desc = "the rings of the batch table in order, up to 32 of each ring's steps (binary64)"
    else:
        reqs = workloads.request_stream(w["rate"], w["duration"], seed=w["seed"])
        rings = [(q.n, q.nt, q.r, q.seed, q.f32c, lambda q=q: workloads.uniform(q.n, q.seed, -1.0, 1.0)) for q in reqs]
        desc = ("the requests of the arrival stream in order, up to 32 of each request's steps "
                "(binary64 or binary32 compensated as requested; u0 = U[-1,1) drawn on the host)")
    while True:
        for n, nt, r, _, f32, init in rings:
            steps = min(nt, 32)

            def unit(n=n, r=r, f32=f32, init=init, steps=steps):
                u = init()
                if f32:
                    oracle.run_f32c(u, np.float32(r), steps, 1)
                else:
                    oracle.run(u, r, steps)
                return n * steps
            yield unit, desc


def _oracle_samples(w: dict, count: int, seconds: float, units=None):
    """`count` samples of at least `seconds` each: (point-steps, seconds) per sample."""
    units = units or _oracle_units(w)
    out, desc = [], ""
    for _ in range(count):
        done, t0 = 0, time.perf_counter()
        while True:
            unit, desc = next(units)
            done += unit()
            if time.perf_counter() - t0 >= seconds:
                break
        out.append((done, time.perf_counter() - t0))
    return out, desc, units


def reference_config(args, w: dict) -> dict:
    """The workload as the GPU arm's `config` names it, without device state."""
    if w["kind"] in ("ring", "precision"):
        n = w["nx"] * w["np"]
        return {"workload": args.workload, "nx": w["nx"], "np": w["np"], "N": n, "nt": w["nt"], "k": w["k"],
                "dt": w["dt"], "dx": w["dx"], "init": w["init"], "arith": args.arith}
    if w["kind"] == "batch":
        return {"workload": args.workload, "rings": w["count"], "seed": w["seed"],
                "nt_range": [w.get("nt_lo", 100), w.get("nt_hi", 5000)]}
    return {"workload": args.workload, "rate_req_s": w["rate"], "window_s": w["duration"], "seed": w["seed"]}


def run_reference(args, w: dict, rank: int) -> None:
    """--impl reference: the CPU oracle as it stands, single-threaded on the host,
    on bounded samples of the workload: W warm-up samples of about 0.2 s, then K
    timed samples of about 2 s (one per bench step).  Under torchrun only rank 0
    runs it."""
    if rank != 0:
        return
    _, _, units = _oracle_samples(w, args.warmup, 0.2)
    samples, desc, _ = _oracle_samples(w, args.steps, 2.0, units)
    pts = sum(p for p, _ in samples)
    secs = sum(t for _, t in samples)
    value = pts / secs / 1e9
    cb = {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "host": host_cpu(),
          "sample": f"{desc}; {args.warmup} warm-up samples, then {args.steps} timed samples of about 2 s "
                    f"({pts:.3g} point-steps in {secs:.1f} s on 1 host core)"}
    line = {"impl": "reference", "metric": METRIC[w["dtype"]], "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if w["dtype"] == "f64" else "f32", "data": "synthetic",
            "config": reference_config(args, w), "cpu_baseline": cb,
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------------------------
# Runners, one per workload kind: step(events), e2e_prepare/e2e_run, kernel_info, config.

class RingRunner:
    """One ring: a step loads u0 from a device copy, runs nt steps and takes the sum."""
    E2E_COPIES = "beside the steps: two contexts on two streams take the steps in turn"

    def __init__(self, args, w, H, torch, local, stream):
        self.args, self.w, self.H, self.torch, self.stream = args, w, H, torch, stream
        self.n = w["nx"] * w["np"]
        self.nt = w["nt"]
        self.point_steps = float(self.n) * self.nt
        self.u0 = initial_state(w)
        self.u0_dev = torch.from_numpy(self.u0).to(f"cuda:{local}")
        self.h = self._context(stream)
        self.h2 = None

    def _context(self, stream):
        args, w, H = self.args, self.w, self.H
        arith = H.HEAT_ARITH_FMA if args.arith == "fma" else H.HEAT_ARITH_EXACT
        h = H.Heat(w["nx"], w["np"], w["k"], w["dt"], w["dx"], dtype=w["dtype"], form=args.form, T=args.T,
                   arith=arith, stream=stream)
        if args.layout >= 0:
            H.heat_set_layout(h.ctx, args.layout)
        if args.split:
            H.heat_set_split(h.ctx, args.split)
        if args.emul >= 0:
            H.heat_set_emulation(h.ctx, args.emul)
        return h

    def step(self, ev=None):
        H, ctx = self.H, self.h.ctx
        H.heat_set_device(ctx, self.u0_dev)
        if ev is not None:
            ev[0].record(self.stream)
        H.heat_run(ctx, self.nt)
        if ev is not None:
            ev[1].record(self.stream)
        H.heat_sum(ctx)  # synchronises the stream

    def e2e_prepare(self):
        # two contexts on two streams take the steps in turn: while one advances
        # its ring, the other's result is read back and its next input copied
        # in; an event keeps the two contexts' steps in order on the device
        torch = self.torch
        self.host_in = torch.empty(self.n, dtype=torch.float64, pin_memory=True).numpy()
        self.host_in[:] = self.u0
        self.host_out = [torch.empty(self.n, dtype=torch.float64, pin_memory=True).numpy() for _ in range(2)]
        if self.h2 is None:
            self.stream2 = torch.cuda.Stream()
            self.h2 = self._context(self.stream2)
        self.pipe = [(self.h, self.stream), (self.h2, self.stream2)]
        self.done = [torch.cuda.Event(), torch.cuda.Event()]

    def e2e_run(self, k):
        H, prev = self.H, None
        for i in range(k):
            x = i & 1
            h, s = self.pipe[x]
            H.heat_set(h.ctx, self.host_in)           # host -> device, beside the other context's steps
            if prev is not None:
                s.wait_event(self.done[prev])
            H.heat_run(h.ctx, self.nt)
            self.done[x].record(s)
            if prev is not None:
                self._e2e_finish(prev)                # device -> host, beside this context's steps
            prev = x
        self._e2e_finish(prev)

    def e2e_agree(self):
        """Both contexts advanced the same input: their read-back states agree bitwise."""
        a, b = (o.view(np.uint64) for o in self.host_out)
        return bool(np.array_equal(a, b))

    def _e2e_finish(self, x):
        ctx = self.pipe[x][0].ctx
        self.H.heat_sum(ctx)
        self.H.heat_get(ctx, self.host_out[x])

    def e2e_bytes(self):
        return self.n * 8, self.n * 8

    def kernel_info(self, run_ms):
        last = self.H.heat_last_run(self.h.ctx)
        form = last["form"]
        launches = max(1, last["launches"])
        # the flag-queue form at depth T > 1 runs k_queue (T-point messages)
        name = {"plain": "k_plain_f64" if self.w["dtype"] == "f64" else "k_plain_f32c",
                "persist": "k_queue" if last["T"] > 1 else "k_persist",
                "tblock": "k_tblock", "cluster": "k_cluster", "persist_tb": "k_wave"}[form]
        src = {"k_plain_f64": "k_plain.cu", "k_plain_f32c": "k_plain.cu", "k_persist": "k_persist.cu",
               "k_queue": "k_queue.cu", "k_tblock": "k_tblock.cu", "k_cluster": "k_cluster.cu",
               "k_wave": "k_wave.cu"}[name]
        srcs = [f"paper_2307_01117_gb300/csrc/{src}", "paper_2307_01117_gb300/csrc/stencil_ops.cuh"]
        if name in ("k_tblock", "k_cluster", "k_wave", "k_queue"):
            srcs.append("paper_2307_01117_gb300/csrc/tb_core.cuh")
        if name in ("k_tblock", "k_wave", "k_queue"):
            srcs.append("paper_2307_01117_gb300/csrc/dp_emul.cuh")
        if name in ("k_wave", "k_queue"):
            srcs.append("paper_2307_01117_gb300/csrc/wave_core.cuh")
        steps_per_launch = self.nt / launches
        elem = 8.0 if self.w["dtype"] == "f64" else 4.0
        # every point read once and written once per launch; the persistent form
        # streams the ring through HBM once per step
        # (the cluster form keeps the ring in shared memory: one read and one write per launch;
        # the persistent temporal-blocking form reads and writes the ring once per T-step level)
        passes = {"persist": -(-steps_per_launch // max(1, last["T"])),
                  "persist_tb": -(-steps_per_launch // max(1, last["T"]))}.get(form, 1.0)
        alg_bytes = 2.0 * elem * self.n * passes
        r = self.w["k"] * self.w["dt"] / (self.w["dx"] * self.w["dx"])
        return {"kernel": name, "src": srcs, "launches": launches, "launch_ms": statistics.mean(run_ms) / launches,
                "point_steps_per_launch": self.n * steps_per_launch, "alg_bytes_per_launch": alg_bytes,
                "form": form, "T": last["T"], "segments": last["segments"] if form != "plain" else None,
                "emul_share": self.H.heat_get_emulation(self.h.ctx)
                if form in ("tblock", "persist_tb") or name == "k_queue" else 0,
                "r_pow2": is_pow2(r),
                # FP64-unit operations per point-step: for r = 2^k every form but the strided
                # temporal-blocking layout multiplies by moving the exponent on the integer pipes
                "dp_ops": 3 if (not (form == "tblock" and self.args.layout == 0) and self.args.arith == "exact"
                                and is_pow2(r)) else DP_OPS[self.args.arith]}

    def config(self):
        w = self.w
        return {"workload": self.args.workload, "nx": w["nx"], "np": w["np"], "N": self.n, "nt": self.nt,
                "k": w["k"], "dt": w["dt"], "dx": w["dx"], "init": w["init"], "arith": self.args.arith,
                "split": self.args.split, "emul_share_of_32": self.H.heat_get_emulation(self.h.ctx),
                "l2": "inputs larger than L2 (no flush needed)" if self.n * 8 > 2 * 135e6 else "L2-resident ring"}

    def close(self):
        self.h.close()
        if self.h2 is not None:
            self.h2.close()


class BatchRunner:
    """Many rings in one batch: a step restores their initial states and runs one
    batch launch that advances every ring its nt steps."""
    E2E_COPIES = "beside the launches: two batches on two streams take the steps in turn"

    def __init__(self, args, w, H, torch, local, stream):
        from paper_2307_01117_gb300 import workloads
        self.args, self.w, self.H, self.torch, self.stream = args, w, H, torch, stream
        self.specs = workloads.ring_table(w["count"], seed=w["seed"], nt_lo=w.get("nt_lo", 100),
                                          nt_hi=w.get("nt_hi", 5000))
        self.inits = [workloads.ring_initial(s) for s in self.specs]
        self.n_total = sum(s.n for s in self.specs)
        self.point_steps = float(sum(s.n * s.nt for s in self.specs))
        dt = H.HEAT_F64 if w["dtype"] == "f64" else H.HEAT_F32C
        self.b = H.heat_batch_create(sum(s.n + 64 for s in self.specs), dt)
        H.heat_batch_set_stream(self.b, stream)
        self.ids = [H.heat_batch_add(self.b, s.nx, s.np_, s.r, 1.0, 1.0, s.nt, u) for s, u in
                    zip(self.specs, self.inits)]
        if args.emul >= 0:
            H.heat_batch_set_emulation(self.b, args.emul)
        if args.T:
            H.heat_batch_set_tuning(self.b, args.T, 0)
            self.tuned = (args.T, 0)
        else:
            self.tuned = H.heat_batch_autotune(self.b)
        H.heat_batch_save(self.b)

    def step(self, ev=None):
        H = self.H
        H.heat_batch_restore(self.b)
        if ev is not None:
            ev[0].record(self.stream)
        H.heat_batch_run(self.b, 0)
        if ev is not None:
            ev[1].record(self.stream)
        H.heat_batch_sync(self.b)

    def e2e_prepare(self):
        # two batches on two streams take the steps in turn: while one runs its
        # launch, the other's results are read back and its next inputs copied
        # in; an event keeps the two batches' launches in order on the device
        torch, H = self.torch, self.H
        self.host_in = [torch.from_numpy(u).pin_memory().numpy() for u in self.inits]
        self.host_out = [[torch.empty(s.n, dtype=torch.float64, pin_memory=True).numpy() for s in self.specs]
                         for _ in range(2)]
        if getattr(self, "b2", None) is None:
            self.stream2 = torch.cuda.Stream()
            dt = H.HEAT_F64 if self.w["dtype"] == "f64" else H.HEAT_F32C
            self.b2 = H.heat_batch_create(sum(s.n + 64 for s in self.specs), dt)
            H.heat_batch_set_stream(self.b2, self.stream2)
            H.heat_batch_set_tuning(self.b2, *self.tuned)
            if self.args.emul >= 0:
                H.heat_batch_set_emulation(self.b2, self.args.emul)
            self.ids2 = []
        self.pipe = [[self.b, self.stream, self.ids], [self.b2, self.stream2, self.ids2]]
        self.done = [torch.cuda.Event(), torch.cuda.Event()]

    def e2e_run(self, k):
        H, prev = self.H, None
        for i in range(k):
            x = i & 1
            b, s, ids = self.pipe[x]
            for rid in ids:
                H.heat_batch_remove(b, rid)
            # host -> device, beside the other batch's launch
            ids[:] = [H.heat_batch_add(b, sp.nx, sp.np_, sp.r, 1.0, 1.0, sp.nt, u) for sp, u in
                      zip(self.specs, self.host_in)]
            if prev is not None:
                s.wait_event(self.done[prev])
            H.heat_batch_run(b, 0)
            self.done[x].record(s)
            if prev is not None:
                self._e2e_finish(prev)                # device -> host, beside this batch's launch
            prev = x
        self._e2e_finish(prev)
        self.ids = self.pipe[0][2]

    def _e2e_finish(self, x):
        b, _, ids = self.pipe[x]
        for rid, sp, out in zip(ids, self.specs, self.host_out[x]):
            self.H.heat_batch_get(b, rid, sp.n, out)

    def e2e_bytes(self):
        return self.n_total * 8, self.n_total * 8

    def e2e_agree(self):
        """Both batches advanced the same inputs: their read-back states agree bitwise."""
        return all(np.array_equal(a.view(np.uint64), c.view(np.uint64))
                   for a, c in zip(self.host_out[0], self.host_out[1]))

    def kernel_info(self, run_ms):
        T = self.tuned[0]
        elem = 8.0 if self.w["dtype"] == "f64" else 4.0
        # every point read and written once per T-step level
        level_points = sum(-(-s.nt // T) * s.n for s in self.specs)
        return {"kernel": "k_batch", "src": ["paper_2307_01117_gb300/csrc/k_batch.cu",
                                             "paper_2307_01117_gb300/csrc/tb_core.cuh",
                                             "paper_2307_01117_gb300/csrc/dp_emul.cuh",
                                             "paper_2307_01117_gb300/csrc/wave_core.cuh",
                                             "paper_2307_01117_gb300/csrc/stencil_ops.cuh"],
                "launches": 1, "launch_ms": statistics.mean(run_ms), "point_steps_per_launch": self.point_steps,
                "alg_bytes_per_launch": 2.0 * elem * level_points, "form": "batch", "T": T,
                "segments": self.tuned[1],
                # the library's adaptive split (-1) unless --emul set a share
                "emul_share": (self.args.emul if self.args.emul >= 0 else -1)
                if self.w["dtype"] == "f64" and self.args.arith == "exact" else 0,
                "r_pow2": all(is_pow2(s.r) for s in self.specs)}

    def config(self):
        ns = [s.n for s in self.specs]
        return {"workload": self.args.workload, "rings": len(self.specs), "points": self.n_total,
                "point_steps": self.point_steps, "n_min": min(ns), "n_max": max(ns),
                "nt_range": [min(s.nt for s in self.specs), max(s.nt for s in self.specs)],
                "tuning": {"T": self.tuned[0], "window_points": self.tuned[1]},
                "l2": "inputs larger than L2 (no flush needed)"}

    def close(self):
        self.H.heat_batch_destroy(self.b)
        if getattr(self, "b2", None) is not None:
            self.H.heat_batch_destroy(self.b2)


class PrecisionRunner(RingRunner):
    """Timed binary32-compensated runs; afterwards one binary64 run of the same ring
    and the closed form give the error report."""

    def accuracy(self):
        torch, H, w = self.torch, self.H, self.w
        n, nt = self.n, self.nt
        # binary32 result of one run
        self.step()
        f32 = torch.empty(n, dtype=torch.float64, device=self.u0_dev.device)
        H.heat_get_device(self.h.ctx, f32)
        # binary64 result (exact reading, default form)
        with H.Heat(w["nx"], w["np"], w["k"], w["dt"], w["dx"], dtype="f64", stream=self.stream) as h64:
            H.heat_set_device(h64.ctx, self.u0_dev)
            H.heat_run(h64.ctx, nt)
            f64 = torch.empty_like(f32)
            H.heat_get_device(h64.ctx, f64)
            h64.sync()
        torch.cuda.synchronize()
        # closed form in binary64: sum_m lambda_m^nt sin(2 pi m g / N), phase reduced as (m g) mod N
        r = w["k"] * w["dt"] / (w["dx"] * w["dx"])
        g = torch.arange(n, dtype=torch.int64, device=f32.device)
        exact = torch.zeros_like(f32)
        for m in w["modes"]:
            lam_n = float(np.exp(nt * np.log1p(-4.0 * r * np.sin(np.pi * m / n) ** 2)))
            exact += lam_n * torch.sin((2.0 * np.pi / n) * ((m * g) % n).to(torch.float64))
        del g
        d = f32 - f64
        rms = float(torch.sqrt(torch.mean(f64 * f64)))
        amax = float(torch.max(torch.abs(f64)))
        ulp32 = float(np.spacing(np.float32(amax)))
        T = H.heat_last_run(self.h.ctx)["T"]
        return {
            "binary32_vs_binary64": {"max_abs": float(torch.max(torch.abs(d))),
                                     "l2_rel": float(torch.sqrt(torch.mean(d * d))) / rms},
            "binary64_vs_closed_form_max_abs": float(torch.max(torch.abs(f64 - exact))),
            "binary32_vs_closed_form_max_abs": float(torch.max(torch.abs(f32 - exact))),
            "initial_rounding_max_abs": float(torch.max(torch.abs(self.u0_dev - self.u0_dev.float().double()))),
            "bound_binary32": (nt / T + 2) * ulp32, "bound_rule": "(nt/T + 2) ulp32(max|u|)", "T": T,
            "max_abs_u": amax, "decay_mode64": float(np.exp(nt * np.log1p(-4.0 * r * np.sin(np.pi * 64 / n) ** 2))),
        }


class ServeRunner:
    """One step = one window of Poisson arrivals replayed in real time through the
    continuous-batching server (not drained at the window's end: unfinished
    requests count as backlog)."""
    E2E_COPIES = None

    def __init__(self, args, w, H, torch, local, stream):
        from paper_2307_01117_gb300 import serve, workloads
        self.args, self.w, self.H, self.torch, self.stream = args, w, H, torch, stream
        self.serve, self.workloads = serve, workloads
        self.rate = args.rate or w["rate"]
        self.duration = args.duration or w["duration"]
        self.windows = []
        self.k = 0
        self.point_steps = 0.0

    def _window(self, duration, seed):
        reqs = self.workloads.request_stream(rate=self.rate, duration=duration, seed=seed)
        if self.args.server == "kernel":
            srv = self.serve.KernelServer(budget_bytes=self.w["budget"], stream=self.stream)
        else:
            srv = self.serve.HeatServer(budget_bytes=self.w["budget"], tick_steps=self.args.tick, stream=self.stream)
        try:
            return srv.serve(reqs, duration=duration)
        finally:
            srv.close()

    def step(self, ev=None):
        if ev is None:   # warm-up: a short window
            self._window(min(2.0, self.duration), self.w["seed"] + 1000 + self.k)
            self.k += 1
            return
        ev[0].record(self.stream)
        st = self._window(self.duration, self.w["seed"] + len(self.windows))
        ev[1].record(self.stream)
        self.windows.append(st)
        self.point_steps = st.summary()["completed_point_steps"]

    def e2e_prepare(self):
        pass

    def e2e_run(self, k):
        pass

    def e2e_bytes(self):
        return 0, 0

    def kernel_info(self, run_ms):
        # kernel server: `ticks` counts server-kernel launches (both dtypes);
        # runs: one launch per arena and run
        ticks = max(1, sum(st.ticks for st in self.windows))
        ps = sum(st.gpu_point_steps for st in self.windows)
        per_window = max(1, ticks // max(1, len(self.windows)))
        kernel, src = (("k_serve", "k_serve.cu") if self.args.server == "kernel" else ("k_batch", "k_batch.cu"))
        return {"kernel": kernel, "src": [f"paper_2307_01117_gb300/csrc/{src}",
                                          "paper_2307_01117_gb300/csrc/tb_core.cuh",
                                          "paper_2307_01117_gb300/csrc/dp_emul.cuh"],
                "launches": per_window, "launch_ms": statistics.mean(run_ms) / per_window,
                "point_steps_per_launch": ps / ticks, "alg_bytes_per_launch": 0.0, "form": "serve",
                "T": None, "segments": None}

    def latency(self):
        done = [d for st in self.windows for d in st.done]
        lat = np.array([d.latency for d in done]) if done else np.zeros(0)
        s = [st.summary() for st in self.windows]
        return {"p50_s": float(np.percentile(lat, 50)) if lat.size else None,
                "p99_s": float(np.percentile(lat, 99)) if lat.size else None,
                "rate_req_s": self.rate, "window_s": self.duration,
                "submitted": sum(x["submitted"] for x in s), "completed": sum(x["completed"] for x in s),
                "backlog_at_window_end": sum(x["backlog"] for x in s),
                "advanced_glups": statistics.mean(x["advanced_glups"] for x in s),
                "max_inflight": max(x["max_inflight"] for x in s), "ticks": sum(x["ticks"] for x in s)}

    def config(self):
        return {"workload": self.args.workload, "rate_req_s": self.rate, "window_s": self.duration,
                "budget_bytes": self.w["budget"], "server": self.args.server,
                "tick_steps": self.args.tick if self.args.server == "runs" else None,
                "requests": "N log-uniform [1e4, 1e7], nt uniform [100, 2000], r uniform [0.05, 0.5], "
                            "binary64 / binary32-compensated 50/50, u0 = U[-1,1) drawn on the device (kernel server: "
                            "views into a pool drawn once)",
                "l2": "inputs larger than L2 (no flush needed)"}

    def close(self):
        pass


# ---------------------------------------------------------------------------------------------
# Sub-records of the default line: the plain one-step-per-launch kernel on the same
# ring, and a short serving window

def plain_subrecord(args, w, H, torch, local, stream, sms: int, pk: dict, probe: dict | None,
                    steps: int = 2) -> dict:
    """The same ring advanced by the plain form (one launch per step): GLUP/s with
    its HBM fraction (16 B per point-step, binary64) and its FP64-unit fraction,
    timed like the headline (CUDA events around heat_run, one warm-up step that
    also captures the run's CUDA graph)."""
    r = w["k"] * w["dt"] / (w["dx"] * w["dx"])
    n, nt = w["nx"] * w["np"], w["nt"]
    u0 = torch.from_numpy(initial_state(w)).to(f"cuda:{local}")
    with H.Heat(w["nx"], w["np"], w["k"], w["dt"], w["dx"], dtype=w["dtype"], form="plain", stream=stream) as h:
        ms = []
        for i in range(steps + 1):
            H.heat_set_device(h.ctx, u0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            H.heat_run(h.ctx, nt)
            e1.record(stream)
            h.sync()
            if i:
                ms.append(e0.elapsed_time(e1))
        launches = H.heat_last_run(h.ctx)["launches"]
    del u0
    glups = n * nt / (statistics.mean(ms) * 1e-3) / 1e9
    elem = 8.0 if w["dtype"] == "f64" else 4.0
    dp_ops = 3 if (args.arith == "exact" and is_pow2(r)) else DP_OPS[args.arith]
    f_peak = 2.0 * sms * pk["sm_max_mhz"] * 1e6 / dp_ops / 1e9
    hbm_gbs = glups * 2 * elem
    f_meas = (1e-9 / (1.0 / probe["dfma_lane_ops_per_s"] + (dp_ops - 1) / probe["dadd_lane_ops_per_s"])
              if probe else None)
    return {"kernel": "k_plain_f64" if w["dtype"] == "f64" else "k_plain_f32c", "form": "plain",
            "value": glups, "unit": UNIT, "steps": steps, "launches_per_step": launches,
            "hbm": {"achieved": hbm_gbs, "peak": pk["hbm_gbs"], "unit": "GB/s", "frac": hbm_gbs / pk["hbm_gbs"],
                    "bytes_per_point_step": 2 * elem},
            "fp64_unit": {"achieved": glups, "peak": f_peak, "unit": "GLUP/s", "frac": glups / f_peak,
                          "peak_measured": f_meas, "frac_measured": glups / f_meas if f_meas else None,
                          "fp64_ops_per_point_step": dp_ops} if w["dtype"] == "f64" else None,
            "headline_over_plain": None}


def serving_subrecord(stream, server: str, rate: float = 100.0, duration: float = 10.0, tick: int = 256,
                      budget: float = 120e9) -> dict:
    """A short serving window (Poisson arrivals replayed in real time through the
    continuous-batching server, not drained): p50/p99 latency, GLUP/s, backlog."""
    from paper_2307_01117_gb300 import serve, workloads
    srv = (serve.KernelServer(budget_bytes=budget, stream=stream) if server == "kernel"
           else serve.HeatServer(budget_bytes=budget, tick_steps=tick, stream=stream))
    try:
        srv.serve(workloads.request_stream(rate=rate, duration=2.0, seed=1002), duration=2.0)   # warm-up
        st = srv.serve(workloads.request_stream(rate=rate, duration=duration, seed=2), duration=duration)
    finally:
        srv.close()
    s = st.summary()
    return {"rate_req_s": rate, "window_s": duration, "server": server,
            "tick_steps": tick if server == "runs" else None, "budget_bytes": budget,
            "p50_s": s["p50_s"], "p99_s": s["p99_s"], "submitted": s["submitted"], "completed": s["completed"],
            "backlog_at_window_end": s["backlog"], "completed_glups": s["completed_glups"],
            "advanced_glups": s["advanced_glups"], "max_inflight": s["max_inflight"],
            "requests": "N log-uniform [1e4, 1e7], nt uniform [100, 2000], r uniform [0.05, 0.5], "
                        "binary64 / binary32-compensated 50/50 (seed 2)"}


# ---------------------------------------------------------------------------------------------

def main() -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS))
    ap.add_argument("--form", default="auto", choices=["auto", "plain", "persist", "tblock", "cluster", "persist_tb"])
    ap.add_argument("--T", type=int, default=0)
    ap.add_argument("--arith", default="exact", choices=["exact", "fma"])
    ap.add_argument("--layout", type=int, default=-1, help="temporal-blocking register layout (0 strided, 1 contiguous)")
    ap.add_argument("--split", type=int, default=0)
    ap.add_argument("--k", type=float, default=0.0, help="ring workloads: override the diffusivity k (r = k dt/dx^2)")
    ap.add_argument("--emul", type=int, default=-1,
                    help="binary64 tiles of 32 on the integer pipes (-1: the library's choice)")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--rate", type=float, default=0.0, help="serving workloads: arrivals per second")
    ap.add_argument("--duration", type=float, default=0.0, help="serving workloads: window length (s)")
    ap.add_argument("--tick", type=int, default=256, help="serving workloads: steps per run (--server runs)")
    ap.add_argument("--server", default="kernel", choices=["kernel", "runs"],
                    help="serving: requests join one running kernel (kernel) or queued batch runs (runs)")
    ap.add_argument("--cpu-report", action="store_true",
                    help="print the CPU baselines on the paper-shaped configurations (no GPU) and exit")
    ap.add_argument("--no-plain", action="store_true", help="leave out the plain-form sub-record")
    ap.add_argument("--no-serving", action="store_true", help="leave out the serving sub-record")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    w = dict(WORKLOADS[args.workload])
    if args.k and w["kind"] in ("ring", "precision"):
        w["k"] = args.k

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        run_reference(args, w, rank)
        return 0
    if args.cpu_report:
        if rank == 0:
            print(json.dumps({"cpu_report": cpu_report()}), flush=True)
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

    stream = torch.cuda.Stream()
    runner = {"ring": RingRunner, "batch": BatchRunner, "serve": ServeRunner,
              "precision": PrecisionRunner}[w["kind"]](args, w, H, torch, local, stream)

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()

    def max_over_ranks(x: float) -> float:
        return reduce_max(x, dist, torch.device("cuda", local))

    for _ in range(args.warmup):
        runner.step()
    barrier()

    clocks = ClockSampler(local)
    clocks.start()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    t_start, t_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    t_start.record(stream)
    for i in range(args.steps):
        runner.step(evs[i])
    t_end.record(stream)
    barrier()
    clk = clocks.stop()
    ms_max = max_over_ranks(t_start.elapsed_time(t_end))
    run_ms = [a.elapsed_time(b) for a, b in evs]
    value = replica_throughput(runner.point_steps, args.steps, ms_max, world)

    # the dominant kernel: algorithmic work per launch over its average launch time
    ki = runner.kernel_info(run_ms)
    pk = peaks()
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    # measured issue rates of the FP64 unit and the integer ALU pipes (probe
    # kernels, CUDA events), beside the nominal 2 and 64 lane-ops/clk/SM
    probe = None
    if w["dtype"] == "f64" and w["kind"] != "serve":
        probe = H.heat_probe_pipes(stream)
        probe["nominal_dp_lane_ops_per_s"] = 2.0 * sms * pk["sm_max_mhz"] * 1e6
        probe["nominal_alu_lane_ops_per_s"] = 64.0 * sms * pk["sm_max_mhz"] * 1e6
    launch_s = ki["launch_ms"] * 1e-3
    hbm = ki["alg_bytes_per_launch"] / launch_s / 1e9
    roof_hbm = {"bound": "hbm", "achieved": hbm, "peak": pk["hbm_gbs"], "unit": "GB/s", "frac": hbm / pk["hbm_gbs"],
                "peak_src": "measured (MEASURED_PEAKS.json hbm_gbs)" if pk["src"] == "measured" else "fallback",
                "alg_bytes_per_launch": ki["alg_bytes_per_launch"]}
    if w["kind"] == "serve":
        roofline = {"bound": "alu", "achieved": None, "peak": None, "unit": "G DP-op/s", "frac": None,
                    "note": "mixed binary64 / binary32 requests; the ring and batch lines carry the kernel rooflines"}
    elif w["dtype"] == "f64":
        # binary64: the FP64 unit's ceiling (2 DP ops/clk/SM) at 4 (exact) or 3 (fused)
        # DP ops per point-step, plus -- when a share of the tiles runs on the integer
        # pipes -- the ALU pipes' ceiling (64 lanes/clk/SM) at the integer routine's ALU
        # instructions per point-step (ncu, profiles/alu_ops.json)
        sm_hz = pk["sm_max_mhz"] * 1e6
        dp_ops = ki.get("dp_ops", DP_OPS[args.arith])
        f_peak = 2.0 * sms * sm_hz / dp_ops / 1e9
        achieved = ki["point_steps_per_launch"] / launch_s / 1e9
        share = ki.get("emul_share", 0)
        roofline = {"bound": "alu", "achieved": achieved, "unit": "GLUP/s", "fp64_unit_peak": f_peak,
                    "fp64_ops_per_point_step": dp_ops, "emul_share_of_32": share}
        # the same ceilings from the probe's measured rates: one fused multiply-add
        # and dp_ops - 1 adds (or multiplies, issued like adds) per point-step
        f_meas = 1e-9 / (1.0 / probe["dfma_lane_ops_per_s"] + (dp_ops - 1) / probe["dadd_lane_ops_per_s"])
        roofline["fp64_unit_peak_measured"] = f_meas
        if share:
            a_ops = alu_ops("pow2" if ki.get("r_pow2") else "general")
            i_peak = 64.0 * sms * sm_hz / a_ops / 1e9 if a_ops else None
            peak = f_peak + i_peak if i_peak else None
            i_meas = probe["alu_lane_ops_per_s"] / a_ops / 1e9 if a_ops else None
            roofline.update({
                "peak": peak, "frac": achieved / peak if peak else None, "int_pipes_peak": i_peak,
                "int_pipes_peak_measured": i_meas,
                "peak_measured": f_meas + i_meas if i_meas else None,
                "frac_measured": achieved / (f_meas + i_meas) if i_meas else None,
                "alu_inst_per_int_point_step": a_ops,
                "peak_src": f"FP64 unit: 2 DP ops/clk/SM x {sms} SMs x {pk['sm_max_mhz']:.0f} MHz / "
                            f"{dp_ops} per point-step, plus ALU pipes: 64 lanes/clk/SM x {sms} SMs x "
                            f"{pk['sm_max_mhz']:.0f} MHz / {a_ops} ALU instructions per integer point-step "
                            f"(ncu-measured, profiles/alu_ops.json)"})
        else:
            roofline.update({
                "peak": f_peak, "frac": achieved / f_peak, "peak_measured": f_meas, "frac_measured": achieved / f_meas,
                "peak_src": f"FP64 unit: 2 DP ops/clk/SM x {sms} SMs x {pk['sm_max_mhz']:.0f} MHz max SM clock "
                            f"/ {dp_ops} DP ops per point-step (GB300 nominal 1.25 TFLOP/s FP64)"})
    else:
        # binary32 compensated: 13 FP32 operations per point-step (two fused differences
        # and their adds, the sum, the product, TwoSum's six, the correction add)
        ops = 13.0 * ki["point_steps_per_launch"]
        fp32_peak = 128.0 * sms * pk["sm_max_mhz"] * 1e6 / 1e12
        achieved = ops / launch_s / 1e12
        roofline = {"bound": "alu", "achieved": achieved, "peak": fp32_peak, "unit": "T FP32-op/s",
                    "frac": achieved / fp32_peak,
                    "peak_src": f"FP32 pipe: 128 ops/clk/SM x {sms} SMs x {pk['sm_max_mhz']:.0f} MHz max SM clock",
                    "alg_ops_per_launch": ops}
    roofline["traffic"] = profile_traffic(ki["kernel"], args.workload, ki["src"])
    roofline["kernel"] = ki["kernel"]
    roofline["launch_ms"] = ki["launch_ms"]
    roofline["launches_per_step"] = ki["launches"]

    e2e = None
    if not args.no_e2e and w["kind"] != "serve":
        runner.e2e_prepare()
        runner.e2e_run(2)
        barrier()
        k_e2e = max(1, min(args.steps, 5))
        t0 = time.perf_counter()
        runner.e2e_run(k_e2e)
        barrier()
        dt_e2e = max_over_ranks(time.perf_counter() - t0)
        bi, bo = runner.e2e_bytes()
        e2e = {"value": world * runner.point_steps * k_e2e / dt_e2e / 1e9, "unit": UNIT, "h2d_bytes_per_step": bi,
               "d2h_bytes_per_step": bo, "steps": k_e2e, "copies": runner.E2E_COPIES,
               "contexts_agree_bitwise": runner.e2e_agree()}

    # the default line carries the plain kernel on the same ring and a short
    # serving window beside the headline (outside its timed region)
    plain = serving = None
    if w["kind"] == "ring" and w["dtype"] == "f64" and not args.no_plain and ki["form"] != "plain":
        plain = plain_subrecord(args, w, H, torch, local, stream, sms, pk, probe)
        plain["headline_over_plain"] = value / plain["value"]
    if args.workload == DEFAULT_WORKLOAD and not args.no_serving:
        serving = serving_subrecord(stream, args.server)

    cb = ct = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and w["kind"] != "serve":
        cb = cpu_baseline(w)
        ct = cpu_threaded(w)

    launches = args.steps * (ki["launches"] + (2 if w["kind"] in ("ring", "precision") else 0))
    if rank == 0:
        cfg = runner.config()
        cfg.update({"form": ki["form"], "T": ki["T"], "segments": ki["segments"],
                    "parallelism": "replicas" if world > 1 else "single GPU"})
        line = {
            "metric": METRIC[w["dtype"]], "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64" if w["dtype"] == "f64" else "f32", "data": "synthetic",
            "config": cfg, "roofline": roofline, "roofline_hbm": roof_hbm, "cpu_baseline": cb, "cpu_threaded": ct,
            "e2e": e2e,
            "gpu_launches": launches, "clocks": clk,
        }
        if probe is not None:
            line["pipe_probe"] = probe
        if plain is not None:
            line["plain"] = plain
        if serving is not None:
            line["serving"] = serving
        if w["kind"] == "precision":
            line["accuracy"] = runner.accuracy()
        if w["kind"] == "serve":
            line["latency"] = runner.latency()
            line["metric"] = "serving: completed GLUP/s with p50/p99 request latency"
        print(json.dumps(line), flush=True)
    runner.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
