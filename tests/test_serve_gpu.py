"""Serving loop: requests admitted by free arena space, batched while others run,
each result bitwise the one the request gets alone."""
import numpy as np
import pytest

import oracle
from paper_2307_01117_gb300 import heat as H
from paper_2307_01117_gb300 import workloads
from paper_2307_01117_gb300.workloads import Request

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2307_01117_gb300 import build
    build.build()


def host_init(req):
    return workloads.uniform(req.n, req.seed, -1, 1)


def test_results_alone_equal_results_in_the_mix():
    import torch
    from paper_2307_01117_gb300.serve import HeatServer
    reqs = workloads.request_stream(rate=60.0, duration=0.7, seed=5, n_lo=1e3, n_hi=4e4, nt_lo=20, nt_hi=300)
    assert len(reqs) >= 20
    # a budget that holds only a few requests at once, so admission has to wait for space
    srv = HeatServer(budget_bytes=2.5e6, tick_steps=64, T32=16,
                     init_fn=lambda req: torch.from_numpy(host_init(req)).cuda())
    try:
        st = srv.serve(reqs, drain=True, keep_results=True)
    finally:
        srv.close()
    s = st.summary()
    assert s["completed"] + s["rejected_too_large"] == len(reqs)
    assert st.max_inflight >= 2                              # requests overlapped on the device
    for d in st.done:
        req = reqs[d.index]
        u0 = host_init(req)
        if req.f32c:
            ref = oracle.run_f32c(u0.astype(np.float32), np.float32(req.r), req.nt, 16).astype(np.float64)
        else:
            ref = oracle.run(u0, req.r, req.nt)
        got = srv.results[d.index]
        assert np.array_equal(got.view(np.uint64), ref.view(np.uint64)), (d.index, req)
    assert s["p50_s"] is not None and s["p99_s"] >= s["p50_s"]


def test_oversized_requests_are_rejected_not_queued_forever():
    from paper_2307_01117_gb300.serve import HeatServer
    reqs = [Request(t_arrive=0.0, n=10**6, nt=10, r=0.3, f32c=False, seed=1),
            Request(t_arrive=0.0, n=1000, nt=10, r=0.3, f32c=False, seed=2)]
    srv = HeatServer(budget_bytes=1e6, tick_steps=16)
    try:
        st = srv.serve(reqs, drain=True)
    finally:
        srv.close()
    s = st.summary()
    assert s["rejected_too_large"] == 1 and s["completed"] == 1
