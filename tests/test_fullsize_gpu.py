"""Full-size parity: the 2^28-point ring (np = 256 x nx = 2^20, nt = 1000,
r = 0.25, u0 = U[0,1) + mode 3) in the launch configuration bench.py times (the
default form), checked point by point where the oracle can compute points one
by one (light cones: every partition-edge point plus seeded random points), by
conservation of sum(u), and against the other forms bitwise."""
import numpy as np
import pytest

import oracle
from paper_2307_01117_gb300 import heat as H
from paper_2307_01117_gb300 import workloads

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

NX, NP, NT, K = 1 << 20, 256, 1000, 0.25


@pytest.fixture(scope="module")
def full_run():
    import torch
    from paper_2307_01117_gb300 import build
    build.build()
    n = NX * NP
    u0 = workloads.uniform_plus_mode(n, seed=0, m=3)
    d0 = torch.from_numpy(u0).cuda()
    out = {}
    for form in ("auto", "plain"):
        with H.Heat(NX, NP, K, 1.0, 1.0, form=form) as h:
            H.heat_set_device(h.ctx, d0)
            s0 = h.sum()
            h.run(NT)
            s1 = h.sum()
            res = torch.empty_like(d0)
            H.heat_get_device(h.ctx, res)
            torch.cuda.synchronize()
            out[form] = (res.cpu().numpy(), s0, s1, H.heat_last_run(h.ctx))
    return u0, out


def test_light_cone_spot_checks(full_run):
    u0, out = full_run
    got = out["auto"][0]
    n = NX * NP
    edges = np.concatenate([np.arange(NP) * NX, np.arange(1, NP + 1) * NX - 1])
    rng = np.random.Generator(np.random.PCG64(123))
    idx = np.concatenate([edges, rng.integers(0, n, 512)])
    ref = oracle.cone(u0, oracle.coef(K, 1.0, 1.0), NT, idx)
    assert np.array_equal(got[idx].view(np.uint64), ref.view(np.uint64))


def test_forms_agree_bitwise_at_full_size(full_run):
    _, out = full_run
    assert out["auto"][3]["form"] == "tblock"
    assert np.array_equal(out["auto"][0].view(np.uint64), out["plain"][0].view(np.uint64))


def test_conservation_at_full_size(full_run):
    u0, out = full_run
    got, s0, s1, _ = out["auto"]
    n = NX * NP
    exact0 = float(np.sum(u0))          # pairwise sum: relative error ~ log2(n) eps
    assert abs(s0 - exact0) <= 1e-9 * abs(exact0)
    # each step perturbs the sum by at most a few roundings per point
    assert abs(s1 - s0) <= 4 * NT * n * 2.3e-16 * np.max(np.abs(u0))
    assert abs(float(np.sum(got)) - s1) <= 1e-9 * abs(s1)
