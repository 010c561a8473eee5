"""Binary64 tiles computed on the integer pipes (heat_set_emulation) give
bitwise the oracle's result for every share, including data that leaves the
integer routines' domain (zeros, subnormals) and power-of-two and general r."""
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


def run(u0, r, nt, T, share, layout=1):
    with H.Heat(len(u0), 1, r, 1.0, 1.0, form="tblock", T=T) as h:
        H.heat_set_layout(h.ctx, layout)
        H.heat_set_emulation(h.ctx, share)
        h.set(u0).run(nt)
        return h.get()


def bits(a):
    return np.asarray(a).view(np.uint64)


@pytest.mark.parametrize("layout", [0, 1])
@pytest.mark.parametrize("share", [0, 1, 8, 16, 31, 32])
@pytest.mark.parametrize("r", [0.25, 0.5, 0.3, 0.123456789])
def test_every_share_is_bitwise_the_oracle(share, r, layout):
    n = 3 * 4096 + 17
    u0 = workloads.uniform(n, 90 + share, -1, 1)
    ref = oracle.run(u0, r, 21)
    assert np.array_equal(bits(run(u0, r, 21, 7, share, layout)), bits(ref))


@pytest.mark.parametrize("share", [16, 32])
def test_paper_ramp_with_zero_second_differences(share):
    u0 = workloads.ramp(4000)
    ref = oracle.run(u0, 0.5, 100)
    assert np.array_equal(bits(run(u0, 0.5, 100, 4, share)), bits(ref))


@pytest.mark.parametrize("layout", [0, 1])
@pytest.mark.parametrize("share", [32])
def test_out_of_domain_values_fall_back(share, layout):
    n = 8192
    u0 = workloads.uniform(n, 3, -1, 1)
    u0[100:140] = 0.0
    u0[500:520] = 5e-310           # subnormal
    u0[900] = -0.0
    u0[2000:2010] = 1e-300         # results go subnormal after a few steps
    ref = oracle.run(u0, 0.37, 12)
    assert np.array_equal(bits(run(u0, 0.37, 12, 4, share, layout)), bits(ref))


def test_constant_field_stays_constant():
    u0 = np.full(10000, 0.7)
    assert np.array_equal(run(u0, 0.25, 30, 8, 32), u0)


@pytest.mark.parametrize("split", [1, 2, 9, 17])
@pytest.mark.parametrize("r", [0.25, 0.3])
def test_split_levels_are_bitwise_the_oracle(split, r):
    n = 2 * 4096 + 333
    u0 = workloads.uniform(n, 7 + split, -1, 1)
    with H.Heat(n, 1, r, 1.0, 1.0, form="tblock", T=5) as h:
        H.heat_set_layout(h.ctx, 0)                 # the split applies to the strided layout
        H.heat_set_split(h.ctx, split)
        h.set(u0).run(23)
        got = h.get()
    assert np.array_equal(bits(got), bits(oracle.run(u0, r, 23)))


def test_split_with_out_of_domain_values():
    n = 8192
    u0 = workloads.uniform(n, 4, -1, 1)
    u0[10:30] = 0.0
    u0[300:310] = 4e-310
    with H.Heat(n, 1, 0.3, 1.0, 1.0, form="tblock", T=4) as h:
        H.heat_set_layout(h.ctx, 0)
        H.heat_set_split(h.ctx, 17)
        h.set(u0).run(10)
        got = h.get()
    assert np.array_equal(bits(got), bits(oracle.run(u0, 0.3, 10)))


def test_automatic_share_is_resolved_per_ring_and_exact():
    """The default (-1): large binary64 rings split their tiles adaptively
    between the integer pipes and the FP64 unit at depth 8; small rings keep
    every tile on the FP64 unit."""
    n = 5_000_000                                   # above the 2^18-point threshold
    u0 = workloads.uniform_plus_mode(n, seed=5, m=3)
    with H.Heat(n // 4, 4, 0.25, 1.0, 1.0, form="tblock") as h:
        assert H.heat_get_emulation(h.ctx) == -1        # adaptive: tiles claimed from both ends
        h.set(u0).run(20)
        assert H.heat_last_run(h.ctx)["T"] == 12          # at least 2^22 points
        got = h.get()
        H.heat_set_emulation(h.ctx, 0)
        assert H.heat_get_emulation(h.ctx) == 0
    assert np.array_equal(bits(got), bits(oracle.run(u0, 0.25, 20)))
    with H.Heat(40000, 1, 0.25, 1.0, 1.0, form="tblock") as h:
        assert H.heat_get_emulation(h.ctx) == 0
        h.set(workloads.uniform(40000, 6, -1, 1)).run(9)
        assert H.heat_last_run(h.ctx)["T"] == 24           # small ring: launch-bound
    with pytest.raises(H.HeatError):
        with H.Heat(100, 1, 0.25, 1.0, 1.0) as h:
            H.heat_set_emulation(h.ctx, -2)


@pytest.mark.parametrize("r", [0.5, 0.25, 0.125, -0.25])
@pytest.mark.parametrize("share", [0, 16])
def test_power_of_two_r_fp64_tiles(r, share):
    """r = +-2^k: screened FP64-unit tiles move the product's exponent on the
    integer pipes; tiles with zeros, -0, subnormals or tiny values take the
    plain FP64 steps.  Bitwise the oracle either way."""
    n = 3 * 4096 + 101
    u0 = workloads.uniform(n, 5, -1, 1)
    u0[10:50] = 0.0
    u0[2000] = -0.0
    u0[5000:5004] = 2e-310
    u0[7000:7010] = 1e-250
    assert np.array_equal(bits(run(u0, r, 29, 8, share)), bits(oracle.run(u0, r, 29)))


@pytest.mark.parametrize("k", [0.3, 0.25])
def test_two_engine_split_on_a_large_ring_is_bitwise_the_oracle(k):
    """The temporal-blocking form's default on 2^22 points (adaptive split
    between the FP64 unit and the integer pipes, depth 12, three blocks and a
    partial one), element by element against the oracle."""
    n = 1 << 22
    u0 = workloads.uniform_plus_mode(n, seed=11, m=5)
    with H.Heat(n // 8, 8, k, 1.0, 1.0, form="tblock") as h:
        got = h.set(u0).run(40).get()
        assert H.heat_get_emulation(h.ctx) == -1
        assert H.heat_last_run(h.ctx)["T"] == 12
    assert np.array_equal(bits(got), bits(oracle.run(u0, k, 40)))


@pytest.mark.parametrize("k", [0.25, 0.3])
def test_library_default_on_mid_size_rings_is_bitwise_the_oracle(k):
    """The library's default from 2^18 to 2^26 binary64 points: one
    dependency-driven launch (persistent temporal blocking, warp tiles split
    between the FP64 unit and the integer pipes), depth 16 below 2^19 points, 12
    from 2^19 to 2^21 and 16 above, element by element against the oracle with
    a partial last block."""
    for n, T in [(1 << 18, 16), (1 << 19, 12), (10**6, 12), (1 << 22, 16)]:
        u0 = workloads.uniform_plus_mode(n, seed=12, m=5)
        with H.Heat(n // 4, 4, k, 1.0, 1.0) as h:
            got = h.set(u0).run(3 * T + 5).get()
            last = H.heat_last_run(h.ctx)
        assert (last["form"], last["T"], last["launches"]) == ("persist_tb", T, 1), n
        assert np.array_equal(bits(got), bits(oracle.run(u0, k, 3 * T + 5))), n


@pytest.mark.parametrize("T", [0, 8])
@pytest.mark.parametrize("share", [-1, 0, 16, 32])
@pytest.mark.parametrize("r", [0.25, 0.3])
def test_persistent_temporal_blocking_takes_the_share(share, r, T):
    """heat_set_emulation reaches the persistent temporal-blocking form (one
    launch for the ring); every share gives the oracle's bits, at the default
    depth and at 8."""
    n = 5 * 4096 + 77
    u0 = workloads.uniform(n, 40 + share, -1, 1)
    u0[300:340] = 0.0
    with H.Heat(n, 1, r, 1.0, 1.0, form="persist_tb", T=T) as h:
        H.heat_set_emulation(h.ctx, share)
        got = h.set(u0).run(37).get()
        assert H.heat_last_run(h.ctx)["T"] == (T or 16)   # the default below 2^19 points
    assert np.array_equal(bits(got), bits(oracle.run(u0, r, 37)))
