"""Continuous-batching server for heat solves (Section 2's problem as requests).

Requests (ring size, steps, coefficient, binary64 or binary32-compensated) are
admitted into two device arenas (the batched-ring runtime, heat_batch_* in
include/heat.h) as space frees up: admission is by free device memory under a
byte budget, and a request's state stays resident on the device from admission
to completion.  Each run advances all admitted requests of an arena by up to
`tick_steps` steps in one persistent launch, so requests that arrive while
others are running join the next run and their work overlaps on the device.

The loop never waits for the device.  Each arena keeps up to `max_queued_runs`
runs queued on its stream (one running, the next behind it), so the GPU has
its next run while the host admits arrivals and collects results.  When a run
that finishes a request is queued, the request's final state is copied, on the
same stream, to a device buffer and from there to pinned host memory, an event
is recorded behind the copy, and the request's arena space is released at
once (every later use of that space is queued behind the copy on the same
stream).  The host polls those events; latency runs from a request's arrival
to the moment the host sees its result in host memory.  Device errors (a
bounded wait that ran out) surface at the end of serve(), when both arenas are
synchronised.

The arenas split the budget by the expected byte share of the request mix
(binary64 points cost 16 bytes in two buffers, binary32 points 8: a 50/50 mix
by count puts one third of the bytes in binary32).  With `tick_steps` a
multiple of the binary32 block depth T, each result is bitwise the one the
request gets alone (binary64: heat_run; binary32: the temporal-blocking form
with block depth T).
"""
from __future__ import annotations

import collections
import time
from dataclasses import dataclass, field

import numpy as np

from . import heat as H
from .workloads import Request


@dataclass
class Done:
    index: int
    t_arrive: float
    t_admit: float
    t_done: float
    n: int
    nt: int
    f32c: bool

    @property
    def latency(self) -> float:
        return self.t_done - self.t_arrive


@dataclass
class ServeStats:
    done: list = field(default_factory=list)
    submitted: int = 0
    rejected_too_large: int = 0
    wall_s: float = 0.0
    ticks: int = 0
    max_inflight: int = 0
    gpu_point_steps: float = 0.0

    def summary(self) -> dict:
        lat = np.array([d.latency for d in self.done]) if self.done else np.zeros(0)
        ps = float(sum(d.n * d.nt for d in self.done))
        return {
            "submitted": self.submitted, "completed": len(self.done),
            "backlog": self.submitted - len(self.done) - self.rejected_too_large,
            "rejected_too_large": self.rejected_too_large,
            "p50_s": float(np.percentile(lat, 50)) if lat.size else None,
            "p99_s": float(np.percentile(lat, 99)) if lat.size else None,
            "mean_s": float(lat.mean()) if lat.size else None,
            "completed_point_steps": ps,
            "completed_glups": ps / self.wall_s / 1e9 if self.wall_s > 0 else None,
            "advanced_glups": self.gpu_point_steps / self.wall_s / 1e9 if self.wall_s > 0 else None,
            "wall_s": self.wall_s, "ticks": self.ticks, "max_inflight": self.max_inflight,
        }


class HeatServer:
    """budget_bytes: device memory for ring state (both arenas, both buffers)."""

    def __init__(self, budget_bytes: float, tick_steps: int = 256, lookahead: int = 64, f32c_share: float = 1 / 3,
                 T64: int = 0, T32: int = 16, stream=None, init_fn=None, ctas64: int = 3, ctas32: int = 2,
                 max_queued_runs: int = 2):
        import torch
        self.torch = torch
        self.tick_steps = int(tick_steps)
        self.lookahead = int(lookahead)
        self.max_queued_runs = max(1, int(max_queued_runs))
        # binary64 points cost 16 bytes (two buffers), binary32 points 8 bytes
        cap32 = max(1, int(budget_bytes * f32c_share) // 8)
        cap64 = max(1, int(budget_bytes * (1 - f32c_share)) // 16)
        self.caps = {False: cap64, True: cap32}
        self.batch = {False: H.heat_batch_create(cap64, H.HEAT_F64), True: H.heat_batch_create(cap32, H.HEAT_F32C)}
        # one stream per arena: the binary64 batch (FP64 unit) and the binary32
        # batch (FP32 and integer pipes) run side by side, each capped so that
        # both fit on every SM
        self.stream = stream if stream is not None else torch.cuda.Stream()
        self.stream32 = torch.cuda.Stream()
        H.heat_batch_set_stream(self.batch[False], self.stream)
        H.heat_batch_set_stream(self.batch[True], self.stream32)
        if ctas64 or ctas32:
            H.heat_batch_set_ctas_per_sm(self.batch[False], ctas64)
            H.heat_batch_set_ctas_per_sm(self.batch[True], ctas32)
        if T64:
            H.heat_batch_set_tuning(self.batch[False], T64, 0)
        H.heat_batch_set_tuning(self.batch[True], T32, 0)
        if self.tick_steps % T32:
            raise ValueError("tick_steps must be a multiple of the binary32 block depth")
        self.init_fn = init_fn or self._device_uniform
        self._reset_queues()

    def _reset_queues(self) -> None:
        self.queue: collections.deque = collections.deque()
        self.inflight: dict = {}   # (f32c, ring id) -> (index, request, t_admit)
        self.runs: dict = {False: collections.deque(), True: collections.deque()}  # events behind queued runs
        self.pending: list = []    # result copies in flight: (event, host array, index, request, t_admit)
        self.results: dict = {}    # index -> host array (when keep_results)

    # -- device specifics (stream-ordered work and events) ----------------------------------------

    def _arena_stream(self, f32: bool):
        return self.stream32 if f32 else self.stream

    def _device_uniform(self, req: Request):
        torch = self.torch
        g = torch.Generator(device="cuda")
        g.manual_seed(req.seed)
        return torch.empty(req.n, dtype=torch.float64, device="cuda").uniform_(-1.0, 1.0, generator=g)

    def _mark(self, f32: bool):
        """An event recorded now on the arena's stream."""
        ev = self.torch.cuda.Event()
        ev.record(self._arena_stream(f32))
        return ev

    def _result_copy(self, f32: bool, rid: int, n: int):
        """Queue a finished ring's state to pinned host memory on the arena's
        stream (device buffer, then host); returns (host array, event)."""
        torch = self.torch
        s = self._arena_stream(f32)
        with torch.cuda.stream(s):          # the buffer belongs to the stream that uses it
            dev = torch.empty(n, dtype=torch.float64, device="cuda")
        H.heat_batch_get_device(self.batch[f32], rid, dev, n)
        host = torch.empty(n, dtype=torch.float64, pin_memory=True)
        with torch.cuda.stream(s):
            host.copy_(dev, non_blocking=True)
        return host.numpy(), self._mark(f32)

    # ---------------------------------------------------------------------------------------------

    def close(self):
        for b in self.batch.values():
            H.heat_batch_destroy(b)
        self.batch = {}

    def submit(self, index: int, req: Request, stats: ServeStats) -> None:
        stats.submitted += 1
        if req.n + 64 > self.caps[req.f32c]:
            stats.rejected_too_large += 1
            return
        self.queue.append((index, req))

    def _admit(self, now: float) -> None:
        kept = collections.deque()
        looked = 0
        while self.queue and looked < self.lookahead:
            index, req = self.queue.popleft()
            looked += 1
            b = self.batch[req.f32c]
            with self.torch.cuda.stream(self._arena_stream(req.f32c)):  # the copy's stream
                u = self.init_fn(req)
            try:
                rid = H.heat_batch_add_device(b, req.n, 1, req.r, 1.0, 1.0, req.nt, u)
            except H.HeatError as e:
                if e.code != H.HEAT_ENOMEM:
                    raise
                kept.append((index, req))   # no room yet: keep its place
                continue
            self.inflight[(req.f32c, rid)] = (index, req, now)
        kept.extend(self.queue)
        self.queue = kept

    def _collect(self, t0: float, stats: ServeStats, keep_results: bool) -> None:
        """Record the requests whose results have reached host memory."""
        still = []
        for ev, host, index, req, t_admit in self.pending:
            if ev.query():
                stats.done.append(Done(index, req.t_arrive, t_admit, time.perf_counter() - t0, req.n, req.nt,
                                       req.f32c))
                if keep_results:
                    self.results[index] = host
            else:
                still.append((ev, host, index, req, t_admit))
        self.pending = still

    def _launch(self, f32: bool, stats: ServeStats) -> bool:
        """Queue one run of the arena if it has work and room in its run queue;
        queue the result copies of the requests the run finishes."""
        runs = self.runs[f32]
        while runs and runs[0].query():
            runs.popleft()
        if len(runs) >= self.max_queued_runs:
            return False
        b = self.batch[f32]
        H.heat_batch_run(b, self.tick_steps)
        ps = H.heat_batch_info(b)["last_point_steps"]
        if ps == 0:
            return False
        stats.gpu_point_steps += ps
        stats.ticks += 1
        finished = [key for key in self.inflight
                    if key[0] == f32 and H.heat_batch_query(b, key[1])[1] == 0]
        for key in finished:
            index, req, t_admit = self.inflight.pop(key)
            host, ev = self._result_copy(f32, key[1], req.n)
            # the space is free for rings admitted later: their copies and runs
            # are queued behind this copy on the same stream
            H.heat_batch_remove(b, key[1])
            self.pending.append((ev, host, index, req, t_admit))
        runs.append(self._mark(f32))
        return True

    def tick(self, t0: float, stats: ServeStats, keep_results: bool = False) -> int:
        """Collect finished results, admit arrivals, queue a run on each arena
        that has room for one.  Returns the number of requests in flight."""
        self._collect(t0, stats, keep_results)
        self._admit(time.perf_counter() - t0)
        stats.max_inflight = max(stats.max_inflight, len(self.inflight))
        launched = False
        for f32 in (False, True):
            launched |= self._launch(f32, stats)
        if not launched and (self.inflight or self.pending):
            time.sleep(2e-4)   # the device is busy with queued runs
        return len(self.inflight) + len(self.pending)

    def serve(self, requests: list[Request], duration: float | None = None, drain: bool = False,
              keep_results: bool = False) -> ServeStats:
        """Replay `requests` (arrival times in seconds from the start) in real time.
        Stops at `duration` (default: the last arrival) unless drain is set, in
        which case it runs until every admitted or queued request is done."""
        self._finish_leftovers()
        stats = ServeStats()
        self._reset_queues()
        reqs = sorted(enumerate(requests), key=lambda x: x[1].t_arrive)
        horizon = duration if duration is not None else (reqs[-1][1].t_arrive if reqs else 0.0)
        t0 = time.perf_counter()
        nxt = 0
        while True:
            now = time.perf_counter() - t0
            while nxt < len(reqs) and reqs[nxt][1].t_arrive <= now and reqs[nxt][1].t_arrive <= horizon:
                self.submit(reqs[nxt][0], reqs[nxt][1], stats)
                nxt += 1
            arrivals_left = nxt < len(reqs) and reqs[nxt][1].t_arrive <= horizon
            if now >= horizon and not drain:
                break
            if not self.queue and not self.inflight and not self.pending:
                if not arrivals_left:
                    break
                time.sleep(max(0.0, min(0.01, reqs[nxt][1].t_arrive - now)))
                continue
            self.tick(t0, stats, keep_results)
        stats.wall_s = time.perf_counter() - t0
        for b in self.batch.values():      # report a device error of the window, if any
            H.heat_batch_sync(b)
        return stats

    def _finish_leftovers(self) -> None:
        """Run the requests a previous window left in flight to completion and
        release their space, outside any window's clock and statistics."""
        self.queue.clear()
        scratch = ServeStats()
        t0 = time.perf_counter()
        while self.inflight or self.pending:
            self.tick(t0, scratch)


class KernelServer:
    """Continuous batching inside one running kernel per dtype (heat_server_* in
    include/heat.h): a request is admitted into its server's arena and slot
    table and published to the running server kernel, whose warps take it up at
    once -- no launch boundary, no host tick.  The host only admits, polls the
    host-mapped completion words and moves finished states to pinned host
    memory (device copy on the server's copy stream, then a host copy behind an
    event), so latency runs from arrival to the result in host memory.

    Admission is by free device memory under a byte budget (binary64 and
    binary32 servers split it by the expected byte share of the request mix,
    as HeatServer does), with a bounded lookahead past requests that do not fit
    yet.  Each result is bitwise the request's solo result (binary64:
    heat_run; binary32: the temporal-blocking form with the server's depth)."""

    def __init__(self, budget_bytes: float, lookahead: int = 64, f32c_share: float = 1 / 3, T64: int = 0,
                 T32: int = 16, stream=None, init_fn=None, ctas64: int = 4, ctas32: int = 2,
                 max_requests: int = 4096):
        import torch
        self.torch = torch
        self.lookahead = int(lookahead)
        cap32 = max(1, int(budget_bytes * f32c_share) // 8)
        cap64 = max(1, int(budget_bytes * (1 - f32c_share)) // 16)
        self.caps = {False: cap64, True: cap32}
        self.srv = {False: H.heat_server_create(cap64, H.HEAT_F64, max_requests, T64, ctas64)}
        try:
            self.srv[True] = H.heat_server_create(cap32, H.HEAT_F32C, max_requests, T32, ctas32)
        except Exception:
            H.heat_server_destroy(self.srv[False])
            raise
        self.stream = stream if stream is not None else torch.cuda.Stream()
        self.init_fn = init_fn or self._pool_view
        self._pool = None
        if init_fn is None:
            self._draw_pool(1 << 24)
        self._reset_queues()

    def _reset_queues(self) -> None:
        self.queue: collections.deque = collections.deque()
        self.inflight: dict = {}   # (f32c, request id) -> (index, request, t_admit, device input)
        self.pending: list = []    # result copies in flight: (event, host array, index, request, t_admit)
        self.results: dict = {}

    def _draw_pool(self, n: int) -> None:
        torch = self.torch
        g = torch.Generator(device="cuda")
        g.manual_seed(12345)
        with torch.cuda.stream(self.stream):
            self._pool = torch.empty(n, dtype=torch.float64, device="cuda").uniform_(-1.0, 1.0, generator=g)
        self.stream.synchronize()

    def _pool_view(self, req: Request):
        """The default initial state: U[-1, 1) values, a view into a pool drawn
        once on the device at a seed-given offset.  Drawing each request's values
        would launch a kernel per request, and beside the running server kernels
        such a launch waits for room on the SMs."""
        if req.n > self._pool.numel():
            self._draw_pool(req.n)
        off = (req.seed * 2654435761) % (self._pool.numel() - req.n + 1)
        return self._pool[off:off + req.n]

    def close(self):
        for s in self.srv.values():
            H.heat_server_destroy(s)
        self.srv = {}

    def submit(self, index: int, req: Request, stats: ServeStats) -> None:
        stats.submitted += 1
        if req.n + 64 > self.caps[req.f32c]:
            stats.rejected_too_large += 1
            return
        self.queue.append((index, req))

    # -- device specifics ---------------------------------------------------------------------

    def _input(self, req: Request):
        """The request's initial state on the device, complete (the server's copy
        stream does not wait for other streams)."""
        with self.torch.cuda.stream(self.stream):
            u = self.init_fn(req)
        self.stream.synchronize()
        return u

    def _fetch(self, f32: bool, rid: int, n: int):
        """Queue a completed request's state to pinned host memory: the server's
        device copy, then a host copy behind an event; returns (host array,
        event, device buffer).  The device buffer is written on the server's copy
        stream, which torch's allocator does not see: the caller keeps it until
        the event has fired."""
        torch = self.torch
        s = self.srv[f32]
        with torch.cuda.stream(self.stream):
            dev = torch.empty(n, dtype=torch.float64, device="cuda")
            landed = torch.cuda.Event()
            landed.record(self.stream)      # creates the event; the server records it again behind its copy
        H.heat_server_get_device(s, rid, dev, n, landed)
        host = torch.empty(n, dtype=torch.float64, pin_memory=True)
        with torch.cuda.stream(self.stream):
            self.stream.wait_event(landed)
            host.copy_(dev, non_blocking=True)
            done = torch.cuda.Event()
            done.record(self.stream)
        return host.numpy(), done, dev

    # ------------------------------------------------------------------------------------------

    def _admit(self, now: float) -> None:
        kept = collections.deque()
        looked = 0
        while self.queue and looked < self.lookahead:
            index, req = self.queue.popleft()
            looked += 1
            u = self._input(req)
            try:
                rid = H.heat_server_submit(self.srv[req.f32c], req.n, req.r, 1.0, 1.0, req.nt, u)
            except H.HeatError as e:
                if e.code != H.HEAT_ENOMEM:
                    raise
                kept.append((index, req))   # no room yet: keep its place
                continue
            self.inflight[(req.f32c, rid)] = (index, req, now, u)
        kept.extend(self.queue)
        self.queue = kept

    def _drain(self, f32: bool) -> None:
        """Move the requests the server reports complete to pinned host memory."""
        s = self.srv[f32]
        for rid in H.heat_server_poll(s):
            index, req, t_admit, _ = self.inflight.pop((f32, rid))
            host, done, dev = self._fetch(f32, rid, req.n)
            H.heat_server_release(s, rid)       # the space is reused behind the copy on the server's stream
            self.pending.append((done, host, index, req, t_admit, dev))

    def _finish_leftovers(self) -> None:
        """Let the requests a previous window left in flight complete and release
        them, outside any window's clock and statistics."""
        self.queue.clear()
        scratch = ServeStats()
        t0 = time.perf_counter()
        while self.inflight or self.pending:
            for f32 in (False, True):
                self._drain(f32)
            self._collect(t0, scratch, False)
            time.sleep(2e-4)

    def _collect(self, t0: float, stats: ServeStats, keep_results: bool) -> None:
        still = []
        for item in self.pending:
            ev, host, index, req, t_admit, _ = item
            if ev.query():   # the device buffer goes back to the allocator only now
                stats.done.append(Done(index, req.t_arrive, t_admit, time.perf_counter() - t0, req.n, req.nt,
                                       req.f32c))
                if keep_results:
                    self.results[index] = host
            else:
                still.append(item)
        self.pending = still

    def serve(self, requests: list[Request], duration: float | None = None, drain: bool = False,
              keep_results: bool = False) -> ServeStats:
        """Replay `requests` (arrival times in seconds from the start) in real time;
        the same contract as HeatServer.serve."""
        self._finish_leftovers()
        stats = ServeStats()
        self._reset_queues()
        reqs = sorted(enumerate(requests), key=lambda x: x[1].t_arrive)
        horizon = duration if duration is not None else (reqs[-1][1].t_arrive if reqs else 0.0)
        ps0 = sum(H.heat_server_info(s)["point_steps"] for s in self.srv.values())
        launches0 = sum(H.heat_server_info(s)["launches"] for s in self.srv.values())
        t0 = time.perf_counter()
        nxt = 0
        while True:
            now = time.perf_counter() - t0
            while nxt < len(reqs) and reqs[nxt][1].t_arrive <= now and reqs[nxt][1].t_arrive <= horizon:
                self.submit(reqs[nxt][0], reqs[nxt][1], stats)
                nxt += 1
            arrivals_left = nxt < len(reqs) and reqs[nxt][1].t_arrive <= horizon
            if now >= horizon and not drain:
                break
            if not self.queue and not self.inflight and not self.pending:
                if not arrivals_left:
                    break
                time.sleep(max(0.0, min(0.01, reqs[nxt][1].t_arrive - now)))
                continue
            self._admit(now)
            stats.max_inflight = max(stats.max_inflight, len(self.inflight))
            for f32 in (False, True):
                self._drain(f32)
            self._collect(t0, stats, keep_results)
            time.sleep(2e-4)
        stats.wall_s = time.perf_counter() - t0
        stats.gpu_point_steps = sum(H.heat_server_info(s)["point_steps"] for s in self.srv.values()) - ps0
        stats.ticks = sum(H.heat_server_info(s)["launches"] for s in self.srv.values()) - launches0
        return stats
