"""Persistent forms: segmentation choices, and the bounded waits.

The fault is made on the host side: a test hook tells one segment's CTA to stop
publishing its edge values, so its neighbours' bounded waits run out, the run
reports HEAT_ETIMEOUT at the next sync, and every kernel returns normally.  No
GPU fault, trap or unbounded spin is involved.
"""
import time

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


def bits(a):
    return np.asarray(a).view(np.uint64)


@pytest.mark.parametrize("T", [0, 1, 6])
@pytest.mark.parametrize("segments", [0, -1, 1, 2, 3, 7, 64])
@pytest.mark.parametrize("nx,np_", [(1000, 4), (4099, 16), (65, 3), (1, 5), (1 << 14, 256)])
def test_segmentations_agree_bitwise(segments, nx, np_, T):
    """Depth 1: one value per queue message and one step per message; deeper
    (0: the library's depth): T values and T steps per message."""
    n = nx * np_
    u0 = workloads.uniform(n, 50 + segments, -1, 1)
    ref = oracle.run(u0, 0.3, 37)
    with H.Heat(nx, np_, 0.3, 1.0, 1.0, form="persist", T=T) as h:
        H.heat_set_segments(h.ctx, segments)
        h.set(u0).run(37)
        got = h.get()
    assert np.array_equal(bits(got), bits(ref))


@pytest.mark.parametrize("T", [1, 0])
def test_paper_partitions_one_cta_each(T):
    """np=256 partitions, one segment (CTA) per partition as in Section 2."""
    nx, np_ = 2048, 256
    u0 = workloads.uniform_plus_mode(nx * np_, seed=0, m=3)
    ref = oracle.run_segmented(u0, np_, 0.25, 20)
    with H.Heat(nx, np_, 0.25, 1.0, 1.0, form="persist", T=T) as h:
        H.heat_set_segments(h.ctx, -1)
        h.set(u0).run(20)
        got = h.get()
        assert H.heat_last_run(h.ctx)["segments"] == np_
    assert np.array_equal(bits(got), bits(ref))


@pytest.mark.parametrize("T", [1, 0])
@pytest.mark.parametrize("seg,step", [(0, 0), (3, 5), (6, 17)])
def test_stalled_producer_times_out_cleanly(seg, step, T):
    n = 7 * 4096
    u0 = workloads.uniform(n, 3, -1, 1)
    with H.Heat(4096, 7, 0.25, 1.0, 1.0, form="persist", T=T) as h:
        H.heat_set_segments(h.ctx, 7)
        H.heat_set_wait_limit(h.ctx, 50_000_000)       # 50 ms
        H.heat_inject_stall(h.ctx, seg, step)
        h.set(u0)
        t0 = time.time()
        h.run(40)                                     # launch succeeds
        with pytest.raises(H.HeatError) as e:
            h.sync()
        assert e.value.code == H.HEAT_ETIMEOUT
        assert time.time() - t0 < 10.0
        # the context refuses further runs until the state is reloaded ...
        with pytest.raises(H.HeatError) as e:
            h.run(1)
        assert e.value.code == H.HEAT_ESTATE
        with pytest.raises(H.HeatError):
            h.get()
        # ... and is fully usable again after heat_set with the hook cleared
        H.heat_inject_stall(h.ctx, -1, 0)
        h.set(u0).run(40)
        got = h.get()
    assert np.array_equal(bits(got), bits(oracle.run(u0, 0.25, 40)))


def test_device_stays_usable_after_timeout():
    import torch
    x = torch.arange(10, device="cuda", dtype=torch.float64)
    assert float(x.sum().item()) == 45.0


@pytest.mark.parametrize("tile,step", [(0, 0), (5, 16), (40, 33)])
def test_stalled_tile_times_out_cleanly_in_persistent_temporal_blocking(tile, step):
    """HEAT_FORM_PERSIST_TB: a tile that stops publishing its completion makes its
    neighbours' bounded waits run out; the run reports HEAT_ETIMEOUT, every
    warp returns, and the context works again after heat_set."""
    n = 1 << 16
    u0 = workloads.uniform(n, 4, -1, 1)
    with H.Heat(n, 1, 0.25, 1.0, 1.0, form="persist_tb", T=8) as h:
        H.heat_set_wait_limit(h.ctx, 50_000_000)       # 50 ms
        H.heat_inject_stall(h.ctx, tile, step)
        h.set(u0)
        t0 = time.time()
        h.run(64)
        with pytest.raises(H.HeatError) as e:
            h.sync()
        assert e.value.code == H.HEAT_ETIMEOUT
        assert time.time() - t0 < 10.0
        assert H.heat_last_run(h.ctx)["segments"] > tile
        with pytest.raises(H.HeatError) as e:
            h.run(1)
        assert e.value.code == H.HEAT_ESTATE
        H.heat_inject_stall(h.ctx, -1, 0)
        h.set(u0).run(64)
        got = h.get()
    assert np.array_equal(bits(got), bits(oracle.run(u0, 0.25, 64)))


@pytest.mark.parametrize("r", [0.25, 0.3])
def test_deep_queues_on_a_ragged_mid_size_ring(r):
    """The library's depth on a ring of 3 * 2^18 + 17 points (every co-resident
    CTA owns a segment; binary64 split between the FP64 unit and the integer
    pipes), a step count that leaves a partial last block."""
    n = 3 * (1 << 18) + 17
    u0 = workloads.uniform(n, 77, -1, 1)
    with H.Heat(n, 1, r, 1.0, 1.0, form="persist") as h:
        h.set(u0).run(45)
        got = h.get()
        last = H.heat_last_run(h.ctx)
    assert last["launches"] == 1 and last["T"] >= 2 and last["segments"] > 100
    assert np.array_equal(bits(got), bits(oracle.run(u0, r, 45)))


@pytest.mark.parametrize("T", [8, 32])
def test_deep_queues_binary32_compensated(T):
    n = 200_003
    u0 = workloads.uniform(n, 78, -1, 1)
    ref = oracle.run_f32c(u0.astype(np.float32), np.float32(0.25), 70, T).astype(np.float64)
    with H.Heat(n, 1, 0.25, 1.0, 1.0, dtype="f32c", form="persist", T=T) as h:
        h.set(u0).run(70)
        got = h.get()
    assert np.array_equal(got, ref)
