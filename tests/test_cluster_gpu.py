"""Cluster form (small rings in one thread-block cluster, ghost exchange through
distributed shared memory): bitwise the oracle, every size up to the form's
limit, both dtypes, T values that do and do not divide nt."""
import numpy as np
import pytest

import oracle
from paper_2307_01117_gb300 import heat as H
from paper_2307_01117_gb300 import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2307_01117_gb300 import build
    build.build()


def run(u0, np_, r, nt, T=0, dtype="f64"):
    n = len(u0)
    with H.Heat(n // np_, np_, r, 1.0, 1.0, dtype=dtype, form="cluster", T=T) as h:
        h.set(u0).run(nt)
        out = h.get()
        info = H.heat_last_run(h.ctx)
    return out, info


@pytest.mark.parametrize("n,np_", [(1, 1), (2, 1), (3, 1), (7, 1), (9, 1), (100, 4), (496, 1), (497, 1), (1000, 4),
                                   (4000, 4), (7936, 1), (7937, 1), (20000, 16), (31744, 1)])
@pytest.mark.parametrize("T", [0, 3, 8])
def test_cluster_f64_bitwise(n, np_, T):
    u0 = workloads.uniform(n, 300 + n, -1, 1)
    for nt, r in [(1, 0.5), (17, 0.3), (100, 0.25)]:
        got, info = run(u0, np_, r, nt, T)
        assert info["form"] == "cluster" and info["launches"] == 1
        ref = oracle.run(u0, r, nt)
        assert np.array_equal(got.view(np.uint64), ref.view(np.uint64)), (n, T, nt, info)


def test_paper_small_ring_in_one_launch():
    u0 = workloads.ramp(4000)
    got, info = run(u0, 4, 0.5, 100)
    assert info["segments"] >= 2                       # several CTAs exchanging halos
    assert np.array_equal(got.view(np.uint64), oracle.run(u0, 0.5, 100).view(np.uint64))


@pytest.mark.parametrize("r", [0.5, 0.25, -0.125])
def test_cluster_power_of_two_r_with_out_of_domain_windows(r):
    """r = +-2^k: windows whose values pass the screen multiply by moving the
    exponent; windows with zeros, -0 or subnormals take the plain FP64 steps.
    Both give the oracle's bits."""
    n = 20000
    u0 = workloads.uniform(n, 77, -1, 1)
    u0[100:180] = 0.0
    u0[3000] = -0.0
    u0[9000:9010] = 3e-310
    u0[15000:15020] = 1e-200
    for T in (0, 8):
        got, _ = run(u0, 4, r, 37, T)
        assert np.array_equal(got.view(np.uint64), oracle.run(u0, r, 37).view(np.uint64)), T


@pytest.mark.parametrize("n", [1, 5, 1000, 10000, 60000])
def test_cluster_f32c_bitwise(n):
    u0 = workloads.uniform(n, 11 + n, -1, 1)
    T, nt = 16, 53
    got, info = run(u0, 1, 0.3, nt, T, "f32c")
    ref = oracle.run_f32c(u0.astype(np.float32), np.float32(0.3), nt, T).astype(np.float64)
    assert np.array_equal(got, ref)


def test_cluster_rejects_rings_beyond_its_limit():
    with H.Heat(40000, 1, 0.3, 1.0, 1.0, form="cluster", T=8) as h:
        h.set(np.zeros(40000))
        with pytest.raises(H.HeatError) as e:
            h.run(5)
        assert e.value.code == H.HEAT_ENOTSUP


def test_auto_picks_cluster_for_small_rings():
    """Binary64: the cluster form up to 6144 points, temporal blocking above
    (depth 24 below 2^19 points); binary32: the cluster form while one cluster
    holds the ring."""
    with H.Heat(1000, 4, 0.5, 1.0, 1.0) as h:
        h.set(workloads.ramp(4000)).run(10)
        assert H.heat_last_run(h.ctx)["form"] == "cluster"
    with H.Heat(30000, 1, 0.5, 1.0, 1.0) as h:
        h.set(np.zeros(30000)).run(10)
        last = H.heat_last_run(h.ctx)
        assert last["form"] == "tblock" and last["T"] == 24
    with H.Heat(30000, 1, 0.5, 1.0, 1.0, dtype="f32c") as h:
        h.set(np.zeros(30000)).run(10)
        assert H.heat_last_run(h.ctx)["form"] == "cluster"
    with H.Heat(100000, 1, 0.5, 1.0, 1.0) as h:
        h.set(np.zeros(100000)).run(10)
        assert H.heat_last_run(h.ctx)["form"] == "tblock"
