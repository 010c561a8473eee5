"""Host logic of the continuous-batching server (paper_2307_01117_gb300/serve.py)
on the CPU: admission by arena space with a bounded lookahead, requests that
wait for space keep their place, late arrivals join the next tick, oversized
requests are rejected.  The heat_batch_* calls are replaced by a fake that keeps
step counts and arena occupancy only (no device, no stencil arithmetic); its
runs and result copies count as complete as soon as they are queued."""
import contextlib
import time
import types

import numpy as np
import pytest

from paper_2307_01117_gb300 import serve
from paper_2307_01117_gb300.workloads import Request


class FakeError(RuntimeError):
    def __init__(self, code):
        super().__init__(code)
        self.code = code


ENOMEM = -2


class FakeBatches:
    """Arena occupancy in 64-point units; each run advances every ring by up to
    max_steps and sleeps `tick_s` (a stand-in for the launch)."""

    def __init__(self, caps, tick_s=0.0):
        self.caps, self.tick_s = caps, tick_s
        self.rings = {b: {} for b in caps}
        self.next_id = {b: 0 for b in caps}
        self.last = {b: 0 for b in caps}
        self.runs = 0

    def _len(self, n):
        return -(-(n + 64) // 64) * 64

    def heat_batch_add_device(self, b, nx, np_, k, dt, dx, nt, u):
        n = nx * np_
        assert len(u) == n
        if sum(r["len"] for r in self.rings[b].values()) + self._len(n) > self.caps[b]:
            raise FakeError(ENOMEM)
        rid = self.next_id[b]
        self.next_id[b] += 1
        self.rings[b][rid] = {"n": n, "len": self._len(n), "left": nt, "done": 0}
        return rid

    def heat_batch_run(self, b, max_steps):
        ps = 0
        for r in self.rings[b].values():
            s = min(r["left"], max_steps)
            r["left"] -= s
            r["done"] += s
            ps += s * r["n"]
        self.last[b] = ps
        self.runs += ps > 0            # runs that had work
        if self.tick_s:
            time.sleep(self.tick_s)

    def heat_batch_info(self, b):
        return {"last_point_steps": self.last[b]}

    def heat_batch_sync(self, b):
        pass

    def heat_batch_query(self, b, rid):
        r = self.rings[b][rid]
        return r["done"], r["left"]

    def heat_batch_get(self, b, rid, n):
        return np.zeros(n)

    def heat_batch_remove(self, b, rid):
        del self.rings[b][rid]


def make_server(monkeypatch, cap_points, tick_steps=16, lookahead=64, tick_s=0.0):
    fake = FakeBatches({"b64": cap_points, "b32": cap_points}, tick_s)
    ns = types.SimpleNamespace(HeatError=FakeError, HEAT_ENOMEM=ENOMEM,
                               **{k: getattr(fake, k) for k in dir(fake) if k.startswith("heat_batch_")})
    monkeypatch.setattr(serve, "H", ns)
    srv = object.__new__(serve.HeatServer)
    srv.torch = types.SimpleNamespace(cuda=types.SimpleNamespace(stream=lambda s: contextlib.nullcontext()))
    srv.tick_steps, srv.lookahead = tick_steps, lookahead
    srv.caps = {False: cap_points, True: cap_points}
    srv.batch = {False: "b64", True: "b32"}
    srv.stream = srv.stream32 = None
    srv.init_fn = lambda req: np.zeros(req.n)
    srv.max_queued_runs = 2
    srv._reset_queues()
    # the fake's runs and copies are complete when queued
    srv._mark = lambda f32: READY
    srv._result_copy = lambda f32, rid, n: (np.zeros(n), READY)
    return srv, fake


READY = types.SimpleNamespace(query=lambda: True)


def req(t, n, nt, f32c=False, seed=0):
    return Request(t_arrive=t, n=n, nt=nt, r=0.25, f32c=f32c, seed=seed)


def test_requests_wait_for_space_and_all_complete(monkeypatch):
    srv, fake = make_server(monkeypatch, cap_points=10_000)
    reqs = [req(0.0, 4000, 48) for _ in range(5)]        # two fit at a time (2 x 4096 points)
    st = srv.serve(reqs, drain=True)
    assert len(st.done) == 5 and st.max_inflight == 2 and not srv.queue and not srv.inflight
    order = [d.index for d in sorted(st.done, key=lambda d: d.t_done)]
    assert order[:2] == [0, 1] and sorted(order) == [0, 1, 2, 3, 4]   # waiting requests kept their places
    assert st.ticks == 3 * 3                                          # 48 steps = 3 ticks of 16, three waves
    assert all(r == {} for r in fake.rings.values())                  # every arena slot released


def test_lookahead_admits_a_small_request_behind_one_that_does_not_fit(monkeypatch):
    srv, fake = make_server(monkeypatch, cap_points=10_000)
    st = serve.ServeStats()
    for i, r in enumerate([req(0.0, 6000, 32), req(0.0, 6000, 32), req(0.0, 1000, 32)]):
        srv.submit(i, r, st)
    srv._admit(0.0)
    admitted = sorted(idx for idx, _, _ in srv.inflight.values())
    assert admitted == [0, 2] and [i for i, _ in srv.queue] == [1]


def test_lookahead_is_bounded(monkeypatch):
    srv, fake = make_server(monkeypatch, cap_points=10_000, lookahead=2)
    st = serve.ServeStats()
    for i, r in enumerate([req(0.0, 9000, 32), req(0.0, 9000, 32), req(0.0, 100, 32)]):
        srv.submit(i, r, st)
    srv._admit(0.0)
    # the first fills the arena, the second does not fit, the third is beyond the lookahead
    assert sorted(idx for idx, _, _ in srv.inflight.values()) == [0]
    assert [i for i, _ in srv.queue] == [1, 2]


def test_oversized_requests_are_rejected(monkeypatch):
    srv, fake = make_server(monkeypatch, cap_points=10_000)
    st = srv.serve([req(0.0, 10_000, 16), req(0.0, 100, 16)], drain=True)
    assert st.rejected_too_large == 1 and [d.index for d in st.done] == [1]
    assert st.summary()["backlog"] == 0


def test_late_arrival_joins_the_next_tick_beside_a_running_request(monkeypatch):
    srv, fake = make_server(monkeypatch, cap_points=100_000, tick_s=0.002)
    reqs = [req(0.0, 2000, 16 * 60), req(0.03, 2000, 16)]   # the first runs about 60 ticks (0.12 s)
    st = srv.serve(reqs, drain=True)
    done = {d.index: d for d in st.done}
    assert st.max_inflight == 2
    assert done[1].t_admit < done[0].t_done                   # admitted while the first still ran
    assert done[1].t_done < done[0].t_done                     # and finished first
    assert st.gpu_point_steps == 2000 * 16 * 60 + 2000 * 16


def test_binary32_requests_use_their_own_arena(monkeypatch):
    srv, fake = make_server(monkeypatch, cap_points=5_000)
    st = srv.serve([req(0.0, 4000, 16), req(0.0, 4000, 16, f32c=True)], drain=True)
    assert st.max_inflight == 2 and len(st.done) == 2
    assert {d.f32c for d in st.done} == {False, True}


class Flag:
    """A stand-in for a CUDA event that the test completes by hand."""

    def __init__(self):
        self.ready = False

    def query(self):
        return self.ready


def test_runs_queue_ahead_and_results_count_when_their_copy_lands(monkeypatch):
    srv, fake = make_server(monkeypatch, cap_points=100_000)
    runs, copies = [], []
    srv._mark = lambda f32: runs.append(Flag()) or runs[-1]
    srv._result_copy = lambda f32, rid, n: (np.zeros(n), copies.append(Flag()) or copies[-1])
    st = serve.ServeStats()
    srv.submit(0, req(0.0, 1000, 16 * 5), st)
    srv.submit(1, req(0.0, 1000, 16), st)
    srv.tick(0.0, st)
    srv.tick(0.0, st)
    assert fake.runs == 2 and len(runs) == 2              # two runs queued, none complete yet
    srv.tick(0.0, st)
    assert fake.runs == 2                                 # the run queue is full: the host does not wait, it skips
    assert len(copies) == 1 and not st.done               # request 1 finished in run 1; its copy is in flight
    assert fake.rings["b64"].keys() == {0}                # and its space was released when the copy was queued
    runs[0].ready = True
    srv.tick(0.0, st)
    assert fake.runs == 3 and not st.done
    copies[0].ready = True
    srv.tick(0.0, st)
    assert [d.index for d in st.done] == [1]


# --- the kernel server's host logic (KernelServer), against a fake heat_server_* ----------

class FakeServers:
    """Slots and arena occupancy only; a request completes after `polls_to_finish`
    polls of its server (a stand-in for the running kernel)."""

    def __init__(self, caps, slots=4, polls_to_finish=2):
        self.caps, self.slots, self.polls_to_finish = caps, slots, polls_to_finish
        self.live = {s: {} for s in caps}
        self.submitted, self.released = [], []

    def heat_server_submit(self, s, n, k, dt, dx, nt, u):
        used = sum(r["n"] for r in self.live[s].values())
        free = [i for i in range(self.slots) if i not in self.live[s]]
        if not free or used + n > self.caps[s]:
            raise FakeError(ENOMEM)
        rid = free[0]
        self.live[s][rid] = {"n": n, "polls": 0, "reported": False}
        self.submitted.append((s, rid, n))
        return rid

    def heat_server_poll(self, s):
        out = []
        for rid, r in self.live[s].items():
            r["polls"] += 1
            if r["polls"] >= self.polls_to_finish and not r["reported"]:
                r["reported"] = True
                out.append(rid)
        return out

    def heat_server_release(self, s, rid):
        assert self.live[s][rid]["reported"]
        del self.live[s][rid]
        self.released.append((s, rid))

    def heat_server_info(self, s):
        return {"point_steps": 0, "in_flight": len(self.live[s]), "running": True, "launches": 1}


def make_kernel_server(monkeypatch, cap_points, slots=4, lookahead=64):
    fake = FakeServers({"s64": cap_points, "s32": cap_points}, slots)
    ns = types.SimpleNamespace(HeatError=FakeError, HEAT_ENOMEM=ENOMEM,
                               **{k: getattr(fake, k) for k in dir(fake) if k.startswith("heat_server_")})
    monkeypatch.setattr(serve, "H", ns)
    srv = object.__new__(serve.KernelServer)
    srv.lookahead = lookahead
    srv.caps = {False: cap_points, True: cap_points}
    srv.srv = {False: "s64", True: "s32"}
    srv._input = lambda req: np.zeros(req.n)
    srv._fetch = lambda f32, rid, n: (np.zeros(n), READY, None)
    srv._reset_queues()
    return srv, fake


def test_kernel_server_admits_by_space_and_slots_and_releases_every_request(monkeypatch):
    srv, fake = make_kernel_server(monkeypatch, cap_points=10_000, slots=2)
    reqs = [req(0.0, 4000, 48) for _ in range(5)] + [req(0.0, 100, 48, f32c=True)]
    st = srv.serve(reqs, drain=True)
    assert len(st.done) == 6 and st.max_inflight >= 2
    assert not srv.queue and not srv.inflight and not srv.pending
    assert all(v == {} for v in fake.live.values())
    assert sorted(fake.released) == sorted((s, rid) for s, rid, _ in fake.submitted)
    order = [d.index for d in sorted((d for d in st.done if not d.f32c), key=lambda d: d.t_done)]
    assert order[:2] == [0, 1] and sorted(order) == [0, 1, 2, 3, 4]   # waiting requests kept their places


def test_kernel_server_lookahead_admits_a_small_request_behind_a_large_one(monkeypatch):
    srv, fake = make_kernel_server(monkeypatch, cap_points=10_000, slots=8)
    st = serve.ServeStats()
    for i, r in enumerate([req(0.0, 6000, 32), req(0.0, 6000, 32), req(0.0, 1000, 32)]):
        srv.submit(i, r, st)
    srv._admit(0.0)
    assert sorted(idx for idx, *_ in srv.inflight.values()) == [0, 2] and [i for i, _ in srv.queue] == [1]


def test_kernel_server_rejects_oversized_requests(monkeypatch):
    srv, fake = make_kernel_server(monkeypatch, cap_points=10_000)
    st = srv.serve([req(0.0, 10_000, 16), req(0.0, 100, 16)], drain=True)
    assert st.rejected_too_large == 1 and [d.index for d in st.done] == [1]


def test_a_new_window_first_finishes_what_the_last_one_left_in_flight(monkeypatch):
    srv, fake = make_server(monkeypatch, cap_points=100_000, tick_s=0.002)
    st = srv.serve([req(0.0, 2000, 16 * 50)], duration=0.005)  # ends after a few runs, the request in flight
    assert st.submitted == 1 and not st.done and srv.inflight
    st2 = srv.serve([req(0.0, 1000, 16)], drain=True)
    assert [d.index for d in st2.done] == [0] and all(r == {} for r in fake.rings.values())


def test_kernel_server_window_finishes_the_last_windows_requests(monkeypatch):
    srv, fake = make_kernel_server(monkeypatch, cap_points=10_000)
    fake.polls_to_finish = 10**9                              # never completes within the first window
    srv.serve([req(0.0, 2000, 32)], duration=0.002)
    assert srv.inflight
    fake.polls_to_finish = 2
    st = srv.serve([req(0.0, 1000, 16)], drain=True)
    assert [d.index for d in st.done] == [0]
    assert all(v == {} for v in fake.live.values())


def test_kernel_server_default_inputs_are_pool_views():
    """The default initial state of a request is a view into one pool, at an
    offset set by the request's seed: no kernel launch per request, the same
    values for the same seed, always inside the pool."""
    import torch
    srv = object.__new__(serve.KernelServer)
    srv._pool = torch.arange(1000, dtype=torch.float64)
    for seed in range(50):
        for n in (1, 17, 999, 1000):
            v = srv._pool_view(req(0.0, n, 10, seed=seed))
            assert v.numel() == n and v.data_ptr() >= srv._pool.data_ptr()
            off = int(v[0].item())
            assert 0 <= off <= 1000 - n and torch.equal(v, srv._pool[off:off + n])
            assert torch.equal(v, srv._pool_view(req(0.0, n, 10, seed=seed)))
    offs = {int(srv._pool_view(req(0.0, 10, 10, seed=s))[0].item()) for s in range(50)}
    assert len(offs) > 40
