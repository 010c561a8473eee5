"""GPU parity of the Eq. 2 coefficient r = k*dt/dx^2 at dt, dx != 1.

Every other GPU test builds its rings with dt = dx = 1, where k*dt/dx^2, k*dt/dx
and k/(dx*dx) agree.  Here the library's coefficient is checked bitwise
against the oracle's ``coef`` (Eq. 2 under the h^2 reading of its printed
denominator), and every form, both dtypes and the batched runtime are run at
coefficients that only the h^2 reading, evaluated as (k*dt)/(dx*dx), gives.
"""
import numpy as np
import pytest

import oracle
from paper_2307_01117_gb300 import heat as H
from paper_2307_01117_gb300 import workloads

pytestmark = pytest.mark.gpu

# (k, dt, dx): two of the examples with exactly representable r (0.2, 0.3), one
# whose r is a power of two (0.25: the exponent-move multiply), and two drawn at
# random whose r differs in its last bits between (k*dt)/(dx*dx) and the other
# evaluation orders (checked on the CPU in test_oracle.py).
COEFS = [(0.1, 0.5, 0.5), (0.3, 0.25, 0.5), (0.5, 0.125, 0.5),
         (0.3286206332490522, 0.030200396783920985, 0.3),
         (0.44845565991743563, 0.6130994749175215, 1.3)]

FORMS = [("plain", 0), ("persist", 0), ("tblock", 0), ("tblock", 5), ("cluster", 0), ("persist_tb", 0),
         ("auto", 0)]


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2307_01117_gb300 import build
    build.build()


def same_bits(a, b):
    return np.array_equal(np.asarray(a).view(np.uint64), np.asarray(b).view(np.uint64))


@pytest.mark.parametrize("k,dt,dx", COEFS)
def test_info_reports_the_oracle_coefficient(k, dt, dx):
    for dtype in ("f64", "f32c"):
        with H.Heat(10, 3, k, dt, dx, dtype=dtype) as h:
            assert np.float64(h.r).view(np.uint64) == np.float64(oracle.coef(k, dt, dx)).view(np.uint64)


@pytest.mark.parametrize("form,T", FORMS)
@pytest.mark.parametrize("k,dt,dx", COEFS)
def test_every_form_bitwise_at_dt_dx_not_one(form, T, k, dt, dx):
    n, np_ = 4 * 4096 + 64, 4                  # within the cluster form's limit
    u0 = workloads.uniform(n, 31, -1, 1)
    r = oracle.coef(k, dt, dx)
    for nt in (1, 23):
        with H.Heat(n // np_, np_, k, dt, dx, form=form, T=T) as h:
            h.set(u0).run(nt)
            got = h.get()
        assert same_bits(got, oracle.run(u0, r, nt)), (form, T, k, dt, dx, nt)


@pytest.mark.parametrize("k,dt,dx", COEFS)
def test_large_ring_default_path_at_dt_dx_not_one(k, dt, dx):
    """2^18 + 192 points: the library's default (persistent temporal blocking)
    splits its warp tiles between the FP64 unit and the integer pipes, whose
    multiply takes r's bits; the temporal-blocking form does the same."""
    n, np_ = (1 << 18) + 192, 4
    u0 = workloads.uniform_plus_mode(n, seed=3, m=3)
    r = oracle.coef(k, dt, dx)
    ref = oracle.run(u0, r, 40)
    for form, want in (("auto", "persist_tb"), ("tblock", "tblock")):
        with H.Heat(n // np_, np_, k, dt, dx, form=form) as h:
            h.set(u0).run(40)
            got = h.get()
            info = H.heat_last_run(h.ctx)
        assert info["form"] == want
        assert same_bits(got, ref), (form, k, dt, dx)


@pytest.mark.parametrize("form,T", [("plain", 0), ("tblock", 8), ("auto", 0), ("persist_tb", 16)])
@pytest.mark.parametrize("k,dt,dx", COEFS[2:])
def test_f32c_at_dt_dx_not_one(form, T, k, dt, dx):
    n = 20000
    u0 = workloads.uniform(n, 17, -1, 1)
    rf = np.float32(oracle.coef(k, dt, dx))
    nt = 37
    with H.Heat(n, 1, k, dt, dx, dtype="f32c", form=form, T=T) as h:
        h.set(u0).run(nt)
        got = h.get()
        Tb = H.heat_last_run(h.ctx)["T"]
    ref = oracle.run_f32c(u0.astype(np.float32), rf, nt, Tb).astype(np.float64)
    assert np.array_equal(got, ref), (form, T, k, dt, dx)


def test_fused_reading_at_dt_dx_not_one():
    k, dt, dx = COEFS[3]
    n = 5003
    u0 = workloads.uniform(n, 8, -2, 2)
    r = oracle.coef(k, dt, dx)
    for form in ("plain", "tblock"):
        with H.Heat(n, 1, k, dt, dx, form=form, arith=H.HEAT_ARITH_FMA) as h:
            h.set(u0).run(30)
            assert same_bits(h.get(), oracle.run(u0, r, 30, fma=True)), form


def test_batch_rings_with_their_own_dt_dx():
    rng = np.random.Generator(np.random.PCG64(12))
    specs = []
    for i in range(40):
        k, dt, dx = COEFS[i % len(COEFS)]
        np_ = int(rng.choice([1, 2, 4, 8]))
        nx = int(rng.integers(1, 6000))
        nt = int(rng.integers(0, 120))
        specs.append((nx, np_, k, dt, dx, nt, workloads.uniform(nx * np_, 500 + i, -1, 1)))
    b = H.heat_batch_create(sum(nx * np_ + 64 for nx, np_, *_ in specs))
    try:
        ids = [H.heat_batch_add(b, nx, np_, k, dt, dx, nt, u0) for nx, np_, k, dt, dx, nt, u0 in specs]
        H.heat_batch_run(b, 0)
        H.heat_batch_sync(b)
        for rid, (nx, np_, k, dt, dx, nt, u0) in zip(ids, specs):
            got = H.heat_batch_get(b, rid, nx * np_)
            assert same_bits(got, oracle.run(u0, oracle.coef(k, dt, dx), nt)), (rid, k, dt, dx, nt)
    finally:
        H.heat_batch_destroy(b)

