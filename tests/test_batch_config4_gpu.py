"""The 4096-ring batch at its real shape, through the library's default path,
against the oracle on a seeded sample of 64 rings.

The table: 4096 independent periodic rings, N log-uniform in [1e3, 1e6], np
uniform in {1, 2, 4, 8, 16}, nt uniform in [100, 5000], r uniform in
[0.05, 0.5], u0 ~ U[-1, 1) (seed 1) -- each ring one instance of Eq. 2 on a
loop (Section 2).  Every ring is admitted, the batch is tuned by
heat_batch_autotune and advanced by one heat_batch_run with the default
adaptive split between the FP64 unit and the integer pipes.  The sample holds
the largest ring and the ring with the most steps.  A sampled ring is compared
in full with the oracle's run when N*nt <= 5e8, else at its ends, at every
partition boundary and at 16 seeded random points through the oracle's light
cone (u^nt at a point from its (2nt+1)-wide cone, same operation order).
The oracle runs on host threads (its ctypes calls release the GIL)."""
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

import oracle
from paper_2307_01117_gb300 import heat as H
from paper_2307_01117_gb300 import workloads

pytestmark = pytest.mark.gpu

FULL_LIMIT = 5e8          # point-steps the oracle runs in full for one ring


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2307_01117_gb300 import build
    build.build()


def sample_indices(specs, count=64, seed=4):
    ns = np.array([s.n for s in specs])
    nts = np.array([s.nt for s in specs])
    must = {int(ns.argmax()), int(nts.argmax())}
    rng = np.random.Generator(np.random.PCG64(seed))
    rest = [int(i) for i in rng.permutation(len(specs)) if int(i) not in must]
    return sorted(must | set(rest[:count - len(must)]))


def cone_points(spec, seed):
    n, nx = spec.n, spec.nx
    pts = {0, n - 1}
    for p in range(1, spec.np_):
        pts |= {p * nx - 1, p * nx}
    rng = np.random.Generator(np.random.PCG64(seed))
    pts |= set(int(g) for g in rng.integers(0, n, 16))
    return np.array(sorted(pts), dtype=np.int64)


def check_ring(spec, got):
    u0 = workloads.ring_initial(spec)
    if spec.n * spec.nt <= FULL_LIMIT:
        ref = oracle.run(u0, spec.r, spec.nt)
        return "full", int(np.sum(got.view(np.uint64) != ref.view(np.uint64)))
    idx = cone_points(spec, spec.seed)
    ref = oracle.cone(u0, spec.r, spec.nt, idx)
    return "cone", int(np.sum(got[idx].view(np.uint64) != ref.view(np.uint64)))


def test_config4_sample_through_the_default_batch_path():
    specs = workloads.ring_table(4096, seed=1)
    sample = sample_indices(specs)
    assert len(sample) == 64
    b = H.heat_batch_create(sum(s.n + 64 for s in specs))
    try:
        ids = [H.heat_batch_add(b, s.nx, s.np_, s.r, 1.0, 1.0, s.nt, workloads.ring_initial(s)) for s in specs]
        T, seg = H.heat_batch_autotune(b)
        assert 1 <= T <= 64 and seg >= 512
        H.heat_batch_run(b, 0)
        H.heat_batch_sync(b)
        assert H.heat_batch_info(b)["last_point_steps"] == sum(s.n * s.nt for s in specs)
        got = {i: H.heat_batch_get(b, ids[i], specs[i].n) for i in sample}
        for i in sample:
            assert H.heat_batch_query(b, ids[i]) == (specs[i].nt, 0)
    finally:
        H.heat_batch_destroy(b)
    with ThreadPoolExecutor(max_workers=max(1, os.cpu_count() or 1)) as ex:
        results = list(ex.map(lambda i: (i, *check_ring(specs[i], got[i])), sample))
    kinds = {k for _, k, _ in results}
    assert kinds == {"full", "cone"}
    bad = [(i, specs[i].n, specs[i].nt, kind, nbad) for i, kind, nbad in results if nbad]
    assert not bad, (T, seg, bad)
