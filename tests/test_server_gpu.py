"""The request server (heat_server_*): continuous batching inside one running
kernel.  Requests submitted while others run join the running kernel (no new
launch), each result is bitwise the request's solo result, the kernel ends by
itself when idle and starts again on the next submission, and oversized or
invalid requests are refused."""
import time

import numpy as np
import pytest

import oracle
from paper_2307_01117_gb300 import heat as H
from paper_2307_01117_gb300 import workloads
from paper_2307_01117_gb300.workloads import Request

pytestmark = [pytest.mark.gpu, pytest.mark.timeout(180)]


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2307_01117_gb300 import build
    build.build()


def bits(a):
    return np.asarray(a).view(np.uint64)


def solo(req, T32=16):
    u0 = workloads.uniform(req.n, req.seed, -1, 1)
    if req.f32c:
        return oracle.run_f32c(u0.astype(np.float32), np.float32(req.r), req.nt, T32).astype(np.float64)
    return oracle.run(u0, req.r, req.nt)


def wait_for(s, want, limit_s=60.0):
    """Poll until `want` request ids have been reported."""
    got, t0 = [], time.time()
    while len(got) < want:
        got += H.heat_server_poll(s)
        assert time.time() - t0 < limit_s, "requests did not complete"
        time.sleep(1e-3)
    return got


def fetch(s, rid, n):
    import torch
    out = torch.empty(n, dtype=torch.float64, device="cuda")
    ev = torch.cuda.Event()
    ev.record()
    H.heat_server_get_device(s, rid, out, n, ev)
    ev.synchronize()
    return out.cpu().numpy()


def test_requests_join_the_running_kernel_and_match_their_solo_results():
    import torch
    s = H.heat_server_create(1 << 22, H.HEAT_F64, 64, 16, 4)
    try:
        H.heat_server_set_limits(s, 2_000_000_000, 500_000_000)
        long_req = Request(t_arrive=0, n=1_000_000, nt=3000, r=0.3, f32c=False, seed=7)
        u_long = torch.from_numpy(workloads.uniform(long_req.n, long_req.seed, -1, 1)).cuda()
        short_reqs = [Request(t_arrive=0, n=1000 + 977 * i, nt=17 + 13 * i, r=0.05 + 0.03 * i, f32c=False,
                              seed=100 + i) for i in range(12)]
        inputs = [torch.from_numpy(workloads.uniform(q.n, q.seed, -1, 1)).cuda() for q in short_reqs]
        torch.cuda.current_stream().synchronize()
        rid_long = H.heat_server_submit(s, long_req.n, long_req.r, 1.0, 1.0, long_req.nt, u_long)
        time.sleep(0.002)
        info = H.heat_server_info(s)
        assert info["running"] and info["launches"] == 1
        # submitted while the long request runs (it takes about 20 ms on its own)
        shorts = [(H.heat_server_submit(s, q.n, q.r, 1.0, 1.0, q.nt, u), q) for q, u in zip(short_reqs, inputs)]
        done = wait_for(s, len(shorts))
        # the short requests were admitted into the kernel already running the long one
        assert H.heat_server_info(s)["launches"] == 1
        assert rid_long not in done
        for rid, req in shorts:
            assert np.array_equal(bits(fetch(s, rid, req.n)), bits(solo(req))), req
            H.heat_server_release(s, rid)
        done = wait_for(s, 1)
        assert done == [rid_long]
        # the long request by light cones: tile edges and seeded points
        got = fetch(s, rid_long, long_req.n)
        idx = np.unique(np.concatenate([np.arange(0, long_req.n, 480)[:8], [long_req.n - 1],
                                        np.random.Generator(np.random.PCG64(1)).integers(0, long_req.n, 24)]))
        u0 = workloads.uniform(long_req.n, long_req.seed, -1, 1)
        assert np.array_equal(bits(got[idx]), bits(oracle.cone(u0, long_req.r, long_req.nt, idx)))
        H.heat_server_release(s, rid_long)
        assert H.heat_server_info(s)["in_flight"] == 0
    finally:
        H.heat_server_destroy(s)


def test_idle_kernel_ends_and_the_next_submission_starts_it_again():
    import torch
    s = H.heat_server_create(1 << 18, H.HEAT_F64, 8, 8, 2)
    try:
        H.heat_server_set_limits(s, 2_000_000_000, 20_000_000)   # 20 ms idle limit
        for round_ in range(2):
            req = Request(t_arrive=0, n=5000 + round_, nt=40, r=0.25, f32c=False, seed=3 + round_)
            u = torch.from_numpy(workloads.uniform(req.n, req.seed, -1, 1)).cuda()
            torch.cuda.current_stream().synchronize()
            rid = H.heat_server_submit(s, req.n, req.r, 1.0, 1.0, req.nt, u)
            assert wait_for(s, 1) == [rid]
            assert np.array_equal(bits(fetch(s, rid, req.n)), bits(solo(req)))
            H.heat_server_release(s, rid)
            t0 = time.time()
            while H.heat_server_info(s)["running"]:
                assert time.time() - t0 < 10.0
                time.sleep(0.005)
        assert H.heat_server_info(s)["launches"] == 2
    finally:
        H.heat_server_destroy(s)


@pytest.mark.parametrize("T32", [16, 32])
def test_binary32_requests_match_the_temporal_blocking_form(T32):
    import torch
    s = H.heat_server_create(1 << 20, H.HEAT_F32C, 16, T32, 2)
    try:
        reqs, ins = [], []
        for i in range(6):
            req = Request(t_arrive=0, n=700 + 5003 * i, nt=T32 * (1 + i) + i, r=0.1 + 0.07 * i, f32c=True,
                          seed=40 + i)
            u = torch.from_numpy(workloads.uniform(req.n, req.seed, -1, 1)).cuda()
            torch.cuda.current_stream().synchronize()
            ins.append(u)
            reqs.append((H.heat_server_submit(s, req.n, req.r, 1.0, 1.0, req.nt, u), req))
        wait_for(s, len(reqs))
        for rid, req in reqs:
            assert np.array_equal(fetch(s, rid, req.n), solo(req, T32)), req
            H.heat_server_release(s, rid)
    finally:
        H.heat_server_destroy(s)


def test_slots_are_reused_across_many_requests():
    """More requests than slots, each released on completion: slot generations
    keep every request's units apart."""
    import torch
    s = H.heat_server_create(1 << 18, H.HEAT_F64, 4, 12, 3)
    try:
        pending, checked, inputs = {}, 0, {}
        rng = np.random.Generator(np.random.PCG64(9))
        for i in range(40):
            req = Request(t_arrive=0, n=int(rng.integers(50, 20000)), nt=int(rng.integers(1, 90)),
                          r=float(rng.uniform(0.05, 0.5)), f32c=False, seed=500 + i)
            u = torch.from_numpy(workloads.uniform(req.n, req.seed, -1, 1)).cuda()
            torch.cuda.current_stream().synchronize()
            while True:
                try:
                    rid = H.heat_server_submit(s, req.n, req.r, 1.0, 1.0, req.nt, u)
                    break
                except H.HeatError as e:
                    assert e.code == H.HEAT_ENOMEM
                    for d in wait_for(s, 1):
                        dreq = pending.pop(d)
                        assert np.array_equal(bits(fetch(s, d, dreq.n)), bits(solo(dreq)))
                        H.heat_server_release(s, d)
                        checked += 1
            pending[rid] = req
            inputs[rid] = u
        for d in wait_for(s, len(pending)):
            dreq = pending.pop(d)
            assert np.array_equal(bits(fetch(s, d, dreq.n)), bits(solo(dreq)))
            H.heat_server_release(s, d)
            checked += 1
        assert checked == 40
    finally:
        H.heat_server_destroy(s)


def test_server_argument_errors():
    import torch
    s = H.heat_server_create(1 << 12, H.HEAT_F64, 2, 8, 1)
    try:
        u = torch.zeros(1 << 13, dtype=torch.float64, device="cuda")
        with pytest.raises(H.HeatError) as e:
            H.heat_server_submit(s, 0, 0.25, 1.0, 1.0, 10, u)
        assert e.value.code == H.HEAT_EINVAL
        with pytest.raises(H.HeatError) as e:
            H.heat_server_submit(s, 1 << 13, 0.25, 1.0, 1.0, 10, u)    # larger than the arena
        assert e.value.code == H.HEAT_ENOMEM
        with pytest.raises(H.HeatError) as e:
            H.heat_server_submit(s, 100, 0.25, 1.0, 0.0, 10, u)        # dx = 0
        assert e.value.code == H.HEAT_EINVAL
        assert H.heat_server_poll(s) == []
        with pytest.raises(H.HeatError) as e:
            H.heat_server_release(s, 0)                                 # nothing there
        assert e.value.code == H.HEAT_ESTATE
    finally:
        H.heat_server_destroy(s)


def test_kernel_server_results_alone_equal_results_in_the_mix():
    import torch
    from paper_2307_01117_gb300.serve import KernelServer
    reqs = workloads.request_stream(rate=60.0, duration=0.7, seed=5, n_lo=1e3, n_hi=4e4, nt_lo=20, nt_hi=300)
    assert len(reqs) >= 20
    srv = KernelServer(budget_bytes=2.5e6, T32=16, max_requests=64,
                       init_fn=lambda req: torch.from_numpy(workloads.uniform(req.n, req.seed, -1, 1)).cuda())
    try:
        st = srv.serve(reqs, drain=True, keep_results=True)
    finally:
        srv.close()
    s = st.summary()
    assert s["completed"] + s["rejected_too_large"] == len(reqs)
    assert st.max_inflight >= 2
    for d in st.done:
        req = reqs[d.index]
        assert np.array_equal(bits(srv.results[d.index]), bits(solo(req))), (d.index, req)
