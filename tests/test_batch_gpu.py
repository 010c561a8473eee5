"""Batched rings (heat_batch_*): every ring's result equals the oracle's for that
ring alone, whatever the batch around it, the run splits, the tuning or the
arena placement; admission by arena space; checkpoint and restore."""
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


def small_table(count, seed, n_hi=20000, nt_hi=300):
    rng = np.random.Generator(np.random.PCG64(seed))
    specs = []
    for i in range(count):
        n_target = int(np.exp(rng.uniform(0, np.log(n_hi))))
        np_ = int(rng.choice([1, 2, 4, 8, 16]))
        nx = max(1, n_target // np_)
        nt = int(rng.integers(0, nt_hi + 1))
        k = float(rng.uniform(0.05, 0.5))
        specs.append((nx, np_, nt, k, workloads.uniform(nx * np_, 1000 + i, -1, 1)))
    return specs


def add_all(b, specs):
    return [H.heat_batch_add(b, nx, np_, k, 1.0, 1.0, nt, u0) for nx, np_, nt, k, u0 in specs]


@pytest.mark.parametrize("T,seg", [(4, 128), (1, 512), (7, 256), (16, 128), (32, 512), (12, 100000)])
def test_batch_matches_oracle_ring_by_ring(T, seg):
    specs = small_table(60, seed=T)
    specs += [(1, 1, 13, 0.3, np.array([0.7])), (2, 1, 9, 0.5, np.array([1.0, 3.0])),
              (3, 1, 20, 0.25, np.array([1.0, -2.0, 5.0])), (600, 1, 0, 0.3, workloads.uniform(600, 5, -1, 1))]
    cap = sum(nx * np_ + 64 for nx, np_, *_ in specs)
    b = H.heat_batch_create(cap)
    try:
        H.heat_batch_set_tuning(b, T, seg)
        ids = add_all(b, specs)
        H.heat_batch_run(b, 0)
        H.heat_batch_sync(b)
        for rid, (nx, np_, nt, k, u0) in zip(ids, specs):
            got = H.heat_batch_get(b, rid, nx * np_)
            assert np.array_equal(bits(got), bits(oracle.run(u0, k, nt))), (rid, nx * np_, nt)
            assert H.heat_batch_query(b, rid) == (nt, 0)
    finally:
        H.heat_batch_destroy(b)


def test_split_runs_equal_one_run():
    specs = small_table(30, seed=11, nt_hi=200)
    cap = sum(nx * np_ + 64 for nx, np_, *_ in specs)
    b = H.heat_batch_create(cap)
    try:
        ids = add_all(b, specs)
        for chunk in (7, 1, 50, 13, 0):
            H.heat_batch_run(b, chunk)
        for rid, (nx, np_, nt, k, u0) in zip(ids, specs):
            got = H.heat_batch_get(b, rid, nx * np_)
            assert np.array_equal(bits(got), bits(oracle.run(u0, k, nt)))
    finally:
        H.heat_batch_destroy(b)


def test_admission_by_arena_space_and_reuse():
    b = H.heat_batch_create(10000)
    try:
        u = workloads.uniform(4000, 1, -1, 1)
        a = H.heat_batch_add(b, 4000, 1, 0.25, 1.0, 1.0, 5, u)
        c = H.heat_batch_add(b, 4000, 1, 0.25, 1.0, 1.0, 5, u)
        with pytest.raises(H.HeatError) as e:
            H.heat_batch_add(b, 4000, 1, 0.25, 1.0, 1.0, 5, u)
        assert e.value.code == H.HEAT_ENOMEM
        H.heat_batch_remove(b, a)
        d = H.heat_batch_add(b, 2000, 2, 0.25, 1.0, 1.0, 5, u)   # reuses the freed space
        H.heat_batch_run(b, 0)
        ref = oracle.run(u, 0.25, 5)
        for rid in (c, d):
            assert np.array_equal(bits(H.heat_batch_get(b, rid, 4000)), bits(ref))
        H.heat_batch_remove(b, c)
        H.heat_batch_remove(b, d)
        assert H.heat_batch_info(b)["largest_free"] >= 10000       # freed blocks coalesce
        with pytest.raises(H.HeatError):
            H.heat_batch_get(b, c, 4000)
    finally:
        H.heat_batch_destroy(b)


def test_autotune_keeps_states_and_results(tmp_path, monkeypatch):
    monkeypatch.setenv("HEAT_TUNE_CACHE", str(tmp_path / "tune.txt"))
    specs = small_table(40, seed=21, n_hi=100000, nt_hi=120)
    cap = sum(nx * np_ + 64 for nx, np_, *_ in specs)
    b = H.heat_batch_create(cap)
    try:
        ids = add_all(b, specs)
        T, seg = H.heat_batch_autotune(b)
        assert 1 <= T <= 64 and seg in (128, 256, 512)
        assert (tmp_path / "tune.txt").read_text().count("|") == 1
        assert H.heat_batch_autotune(b) == (T, seg)             # served from the cache
        H.heat_batch_run(b, 0)
        for rid, (nx, np_, nt, k, u0) in zip(ids, specs):
            assert np.array_equal(bits(H.heat_batch_get(b, rid, nx * np_)), bits(oracle.run(u0, k, nt)))
    finally:
        H.heat_batch_destroy(b)


def test_save_and_restore():
    specs = small_table(20, seed=31)
    cap = sum(nx * np_ + 64 for nx, np_, *_ in specs)
    b = H.heat_batch_create(cap)
    try:
        ids = add_all(b, specs)
        H.heat_batch_run(b, 10)
        H.heat_batch_save(b)
        H.heat_batch_run(b, 0)
        first = [H.heat_batch_get(b, rid, nx * np_) for rid, (nx, np_, *_) in zip(ids, specs)]
        H.heat_batch_restore(b)
        H.heat_batch_run(b, 0)
        for rid, f, (nx, np_, nt, k, u0) in zip(ids, first, specs):
            again = H.heat_batch_get(b, rid, nx * np_)
            assert np.array_equal(bits(again), bits(f))
            assert np.array_equal(bits(again), bits(oracle.run(u0, k, nt)))
    finally:
        H.heat_batch_destroy(b)


def test_f32c_batch_matches_oracle_block_form():
    specs = small_table(25, seed=41, n_hi=30000, nt_hi=100)
    cap = sum(nx * np_ + 64 for nx, np_, *_ in specs)
    b = H.heat_batch_create(cap, H.HEAT_F32C)
    try:
        H.heat_batch_set_tuning(b, 8, 0)
        ids = add_all(b, specs)
        H.heat_batch_run(b, 0)
        for rid, (nx, np_, nt, k, u0) in zip(ids, specs):
            ref = oracle.run_f32c(u0.astype(np.float32), np.float32(k), nt, 8).astype(np.float64)
            assert np.array_equal(H.heat_batch_get(b, rid, nx * np_), ref), rid
    finally:
        H.heat_batch_destroy(b)


def test_batch_argument_errors():
    with pytest.raises(H.HeatError):
        H.heat_batch_create(0)
    b = H.heat_batch_create(1000)
    try:
        with pytest.raises(H.HeatError):
            H.heat_batch_add(b, 0, 1, 0.25, 1.0, 1.0, 5, np.zeros(0))
        with pytest.raises(H.HeatError):
            H.heat_batch_set_tuning(b, 65, 0)
        with pytest.raises(H.HeatError):
            H.heat_batch_set_tuning(b, 4, -1)
        H.heat_batch_set_tuning(b, 4, 100)                   # rounds up to the narrowest window
        with pytest.raises(H.HeatError):
            H.heat_batch_query(b, 3)
        with pytest.raises(H.HeatError):
            H.heat_batch_restore(b)                          # nothing saved yet
    finally:
        H.heat_batch_destroy(b)


def test_deep_blocks_widen_a_narrow_window():
    """T = 40 leaves a 128-point window 48 output points, fewer than 2T: the run
    widens the window and the rings still get the oracle's bits."""
    specs = small_table(10, seed=77, nt_hi=150)
    b = H.heat_batch_create(sum(nx * np_ + 64 for nx, np_, *_ in specs))
    try:
        H.heat_batch_set_tuning(b, 40, 128)
        ids = add_all(b, specs)
        H.heat_batch_run(b, 0)
        for rid, (nx, np_, nt, k, u0) in zip(ids, specs):
            assert np.array_equal(bits(H.heat_batch_get(b, rid, nx * np_)), bits(oracle.run(u0, k, nt)))
    finally:
        H.heat_batch_destroy(b)


def test_stalled_segment_times_out_and_batch_recovers():
    """Host-side fault injection: one tile of one ring stops publishing; the
    units that wait on it run out of their bounded waits, the run reports
    HEAT_ETIMEOUT, and after restore (with the hook cleared) the batch runs to
    the oracle's result."""
    specs = [(40000, 1, 60, 0.3, workloads.uniform(40000, 1, -1, 1)),
             (30000, 2, 45, 0.2, workloads.uniform(60000, 2, -1, 1))]
    b = H.heat_batch_create(sum(nx * np_ + 64 for nx, np_, *_ in specs))
    try:
        H.heat_batch_set_tuning(b, 4, 4096)
        ids = add_all(b, specs)
        H.heat_batch_save(b)
        H.heat_batch_set_wait_limit(b, 50_000_000)           # 50 ms
        H.heat_batch_inject_stall(b, ids[0], 3, 2)
        H.heat_batch_run(b, 0)
        with pytest.raises(H.HeatError) as e:
            H.heat_batch_sync(b)
        assert e.value.code == H.HEAT_ETIMEOUT
        with pytest.raises(H.HeatError) as e:
            H.heat_batch_run(b, 0)
        assert e.value.code == H.HEAT_ESTATE
        H.heat_batch_inject_stall(b, -1)
        H.heat_batch_restore(b)
        H.heat_batch_run(b, 0)
        for rid, (nx, np_, nt, k, u0) in zip(ids, specs):
            assert np.array_equal(bits(H.heat_batch_get(b, rid, nx * np_)), bits(oracle.run(u0, k, nt)))
    finally:
        H.heat_batch_destroy(b)


def test_graph_replay_of_a_fixed_batch():
    """Restore + run of the same batch replays the captured graph; results stay
    the oracle's, with graphs on and off."""
    specs = small_table(12, seed=51, nt_hi=150)
    b = H.heat_batch_create(sum(nx * np_ + 64 for nx, np_, *_ in specs))
    try:
        ids = add_all(b, specs)
        H.heat_batch_save(b)
        for graphs in (True, True, True, False):
            H.heat_batch_set_graphs(b, graphs)
            H.heat_batch_restore(b)
            H.heat_batch_run(b, 0)
            for rid, (nx, np_, nt, k, u0) in zip(ids, specs):
                assert np.array_equal(bits(H.heat_batch_get(b, rid, nx * np_)), bits(oracle.run(u0, k, nt)))
    finally:
        H.heat_batch_destroy(b)


@pytest.mark.parametrize("share", [0, 5, 16, 32])
def test_integer_pipe_tiles_keep_every_ring_bitwise(share):
    """Any share of a unit's tiles on the integer pipes gives each ring the
    oracle's result; power-of-two and general r, zeros and a subnormal ring
    (which fails the screen and stays on the FP64 unit)."""
    specs = small_table(30, seed=61 + share, n_hi=60000, nt_hi=60)
    specs += [(3000, 2, 17, 0.25, np.zeros(6000)),
              (2048, 1, 9, 0.5, np.full(2048, 5e-310)),
              (4096, 1, 23, 0.3, workloads.ramp(4096))]
    b = H.heat_batch_create(sum(nx * np_ + 64 for nx, np_, *_ in specs))
    try:
        H.heat_batch_set_emulation(b, share)
        ids = add_all(b, specs)
        H.heat_batch_run(b, 0)
        for rid, (nx, np_, nt, k, u0) in zip(ids, specs):
            assert np.array_equal(bits(H.heat_batch_get(b, rid, nx * np_)), bits(oracle.run(u0, k, nt))), rid
        with pytest.raises(H.HeatError):
            H.heat_batch_set_emulation(b, 33)
    finally:
        H.heat_batch_destroy(b)
