"""Pins for the CPU oracle (CPU only).

The oracle is checked against things the paper and the mathematics fix, not
against itself:

* exact rational arithmetic (matrix form of Eq. 2 on tiny rings);
* IEEE round-to-nearest of each operation, emulated with exact fractions;
* conservation of sum(u) on the periodic ring;
* the closed-form decay factor 1 - 4 r sin^2(pi m / N) of every Fourier mode;
* the discrete maximum principle for r <= 1/2;
* hand-derived worked examples in tests/golden/;
* special cases (r = 0, constants, the alternating mode, N = 1 and N = 2);
* the segmented queue algorithm (Section 2) equal to the unsegmented ring.
"""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from exact_binary32 import compensated_exact, rn32
from paper_2307_01117_gb300 import workloads

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
EPS = np.finfo(np.float64).eps


# --- independent exact references -------------------------------------------------

def laplacian_matrix(n):
    """Periodic second-difference matrix built from its definition: -2 on the
    diagonal, +1 for each neighbour index (i-1) mod n and (i+1) mod n."""
    L = [[Fraction(0)] * n for _ in range(n)]
    for i in range(n):
        L[i][i] += -2
        L[i][(i - 1) % n] += 1
        L[i][(i + 1) % n] += 1
    return L


def exact_evolve(u0, r, nt):
    """u^nt = (I + r L)^nt u^0 in exact rationals."""
    n = len(u0)
    L = laplacian_matrix(n)
    A = [[(Fraction(1) if i == j else Fraction(0)) + r * L[i][j] for j in range(n)] for i in range(n)]
    u = [Fraction(x) for x in u0]
    for _ in range(nt):
        u = [sum((A[i][j] * u[j] for j in range(n)), Fraction(0)) for i in range(n)]
    return u


def rn(x: Fraction) -> float:
    """Round an exact rational to the nearest binary64, ties to even
    (CPython's int/int true division is correctly rounded)."""
    return x.numerator / x.denominator


# --- 1. exact rational brute force --------------------------------------------------

@pytest.mark.parametrize("r", [Fraction(1, 8), Fraction(1, 4), Fraction(1, 2)])
@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 8])
def test_exact_rationals(n, r):
    for seed in range(3):
        u0 = workloads.small_ints(n, seed)
        for nt in (0, 1, 2, 5, 12):
            exact = exact_evolve([int(x) for x in u0], r, nt)
            got = oracle.run(u0, float(r), nt)
            # every intermediate is a dyadic rational with < 53 significant bits,
            # so binary64 arithmetic is exact here and must equal the rationals
            assert [Fraction(x) for x in got] == exact, (n, r, nt, seed)


def test_exact_rationals_fma_form():
    for n in (3, 7):
        u0 = workloads.small_ints(n, 11)
        exact = exact_evolve([int(x) for x in u0], Fraction(1, 4), 9)
        got = oracle.run(u0, 0.25, 9, fma=True)
        assert [Fraction(x) for x in got] == exact


# --- 2. rounding of each operation ----------------------------------------------------

def test_each_operation_rounded_once_in_stated_order():
    rng = np.random.Generator(np.random.PCG64(5))
    n = 17
    for trial in range(20):
        u = rng.uniform(-3, 3, n) * 10.0 ** rng.integers(-3, 4, n)
        r = float(rng.uniform(0.01, 0.5))
        got = oracle.run(u, r, 1)
        fr = Fraction(r)
        for i in range(n):
            ul, uc, ur = (Fraction(float(u[(i - 1) % n])), Fraction(float(u[i])), Fraction(float(u[(i + 1) % n])))
            t1 = Fraction(rn(ul - 2 * uc))
            t2 = Fraction(rn(t1 + ur))
            t3 = Fraction(rn(fr * t2))
            v = rn(uc + t3)
            assert got[i] == v, (trial, i)
        got_f = oracle.run(u, r, 1, fma=True)
        for i in range(n):
            ul, uc, ur = (Fraction(float(u[(i - 1) % n])), Fraction(float(u[i])), Fraction(float(u[(i + 1) % n])))
            t1 = Fraction(rn(ul - 2 * uc))
            t2 = Fraction(rn(t1 + ur))
            v = rn(fr * t2 + uc)          # one rounding of the fused multiply-add
            assert got_f[i] == v, (trial, i)


# --- 3. conservation ------------------------------------------------------------------

@pytest.mark.parametrize("n,nt,r", [(4000, 100, 0.5), (997, 300, 0.25), (64, 1000, 0.37), (2, 50, 0.5)])
def test_conservation(n, nt, r):
    u0 = workloads.uniform(n, 3, -1, 1)
    u = oracle.run(u0, r, nt)
    drift = abs(math.fsum(u) - math.fsum(u0))
    # each step adds at most ~3 roundings of size eps*max|u| per point
    assert drift <= 4 * nt * n * EPS * np.max(np.abs(u0))


def test_conservation_paper_ic():
    # u(0, x_i) = x_i on N=4000: sum = N(N-1)/2 and it stays exactly that
    # (all values are integers or halves, so the arithmetic is exact).
    u = oracle.run(workloads.ramp(4000), 0.5, 100)
    assert math.fsum(u) == 7998000.0


# --- 4. Fourier modes --------------------------------------------------------------------

@pytest.mark.parametrize("n,m", [(16, 1), (16, 3), (16, 4), (16, 8), (64, 1), (64, 3), (64, 16), (64, 32),
                                 (4000, 1), (4000, 3), (4000, 1000), (4000, 2000)])
@pytest.mark.parametrize("r", [0.25, 0.5])
def test_fourier_mode_decay(n, m, r):
    nt = 200
    u0 = workloads.mode(n, m)
    lam = 1.0 - 4.0 * r * math.sin(math.pi * m / n) ** 2
    u = oracle.run(u0, r, nt)
    expect = (lam ** nt) * u0
    assert np.max(np.abs(u - expect)) <= 8 * nt * EPS


def test_fft_closed_form():
    """Every DFT coefficient c_m evolves as lambda_m^n c_m (numpy FFT as the
    independent transform)."""
    for n, nt, r in [(64, 50, 0.5), (1000, 40, 0.3), (4096, 20, 0.25)]:
        u0 = workloads.uniform(n, 7, -1, 1)
        u = oracle.run(u0, r, nt)
        m = np.arange(n)
        lam = 1.0 - 4.0 * r * np.sin(np.pi * m / n) ** 2
        pred = np.fft.fft(u0) * lam ** nt
        got = np.fft.fft(u)
        assert np.max(np.abs(got - pred)) <= 1e-11 * n


def test_wrong_operator_would_fail_mode_check():
    """Sanity of the pin itself: the decay check separates Eq. 2 from plausible
    mistakes (neighbours at distance 2, a missing factor 2, a flipped sign)."""
    n, m, r, nt = 64, 3, 0.25, 50
    u0 = workloads.mode(n, m)
    lam = 1.0 - 4.0 * r * math.sin(math.pi * m / n) ** 2
    wrong = [1.0 - 4.0 * r * math.sin(2 * math.pi * m / n) ** 2,   # distance-2 neighbours
             1.0 - 2.0 * r * math.sin(math.pi * m / n) ** 2,       # halved coefficient (2h reading)
             1.0 + 4.0 * r * math.sin(math.pi * m / n) ** 2]       # wrong sign
    u = oracle.run(u0, r, nt)
    assert np.max(np.abs(u - lam ** nt * u0)) <= 8 * nt * EPS
    for w in wrong:
        assert np.max(np.abs(u - w ** nt * u0)) > 1e-6


# --- 5. maximum principle ---------------------------------------------------------------------

def test_max_principle():
    rng = np.random.Generator(np.random.PCG64(9))
    for trial in range(200):
        n = int(rng.integers(1, 9))
        nt = int(rng.integers(0, 30))
        r = float(rng.uniform(0, 0.5))
        u0 = rng.uniform(-5, 5, n)
        u = oracle.run(u0, r, nt)
        slack = (nt + 1) * 4 * EPS * np.max(np.abs(u0))
        assert u.min() >= u0.min() - slack and u.max() <= u0.max() + slack


def test_max_principle_exact_on_dyadics():
    for n in range(1, 9):
        u0 = workloads.small_ints(n, 100 + n)
        u = oracle.run(u0, 0.125, 12)
        assert u.min() >= u0.min() and u.max() <= u0.max()


# --- 6. special cases ---------------------------------------------------------------------------

def test_r_zero_is_identity():
    u0 = workloads.uniform(1001, 4, -1e3, 1e3)
    assert np.array_equal(oracle.run(u0, 0.0, 17), u0)


def test_constant_stays_constant_bitwise():
    for c in (0.1, -3.7, 1e300, 5e-310):
        u0 = np.full(33, c)
        assert np.array_equal(oracle.run(u0, 0.37, 25), u0)


def test_alternating_mode_vanishes_in_one_step():
    u0 = np.array([(-1.0) ** g for g in range(10)]) * 3.5
    u = oracle.run(u0, 0.25, 1)
    assert np.all(u == 0.0)


def test_degenerate_rings():
    # N = 1: both neighbours are the point itself -> unchanged
    assert oracle.run([2.5], 0.5, 7)[0] == 2.5
    # N = 2: both neighbours are the other point: u0' = u0 + r*2*(u1 - u0)
    u = oracle.run([1.0, 3.0], 0.25, 1)
    assert list(u) == [2.0, 2.0]


def test_coefficient_h_squared_reading():
    assert oracle.coef(0.5, 1.0, 1.0) == 0.5
    assert oracle.coef(1.0, 0.5, 2.0) == 0.125          # k dt / dx^2, not k dt / (2 dx)
    assert oracle.coef(0.25, 1.0, 1.0) == 0.25


# (k, dt, dx) triples of the GPU coefficient tests whose r depends on the
# evaluation order in its last bits
ORDER_SENSITIVE = [(0.3286206332490522, 0.030200396783920985, 0.3),
                   (0.44845565991743563, 0.6130994749175215, 1.3)]


@pytest.mark.parametrize("k,dt,dx", ORDER_SENSITIVE)
def test_coefficient_rounding_of_the_stated_order(k, dt, dx):
    """r = (k*dt)/(dx*dx): the exact quotient of the two rounded products,
    rounded once.  Checked with exact fractions; the other evaluation orders
    (and the 2h and h readings) give other bits for these inputs, so the GPU
    coefficient tests at these triples tell the readings apart."""
    K, D, X = Fraction(k), Fraction(dt), Fraction(dx)
    want = rn(Fraction(rn(K * D)) / Fraction(rn(X * X)))
    assert oracle.coef(k, dt, dx) == want
    others = [rn(K * Fraction(rn(D / Fraction(rn(X * X))))),            # k*(dt/(dx*dx))
              rn(Fraction(rn(Fraction(rn(K * D)) / X)) / X),           # (k*dt/dx)/dx
              rn(Fraction(rn(K / Fraction(rn(X * X)))) * D),           # (k/(dx*dx))*dt
              rn(Fraction(rn(K * D)) / Fraction(rn(2 * X))),           # the printed 2h
              rn(Fraction(rn(K * D)) / X)]                             # a first power of h
    assert all(o != want for o in others)


# --- 7. worked examples (tests/golden) ---------------------------------------------------------

def _golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


@pytest.mark.parametrize("name", ["ramp4_r_half.json", "mode8_r_quarter.json"])
def test_golden_small(name):
    g = _golden(name)
    r = oracle.coef(g["k"], g["dt"], g["dx"])
    for nt, expect in g["expected"].items():
        assert list(oracle.run(g["u0"], r, int(nt))) == [float(x) for x in expect]


def test_golden_paper_ic_ring():
    g = _golden("ramp4000_r_half.json")
    r = oracle.coef(g["k"], g["dt"], g["dx"])
    u0 = workloads.ramp(g["N"], g["dx"])
    for nt, changed in g["changed"].items():
        u = oracle.run(u0, r, int(nt))
        expect = u0.copy()
        for k, v in changed.items():
            expect[int(k)] = v
        assert np.array_equal(u, expect)
        assert math.fsum(u) == g["sum"]


# --- 8. the segmented algorithm (Section 2) and the light cone ----------------------------------

@pytest.mark.parametrize("np_,nx", [(1, 1), (1, 9), (2, 1), (3, 5), (4, 1000), (7, 3), (16, 4)])
def test_segmented_equals_unsegmented(np_, nx):
    u0 = workloads.uniform(np_ * nx, 21, -1, 1)
    for nt in (0, 1, 13):
        a = oracle.run(u0, 0.31, nt)
        b = oracle.run_segmented(u0, np_, 0.31, nt)
        assert np.array_equal(a, b)


@pytest.mark.parametrize("np_,nx", [(1, 1), (1, 9), (2, 1), (3, 5), (4, 1000), (7, 3), (16, 4), (32, 257)])
def test_threaded_baseline_equals_unsegmented(np_, nx):
    """The threaded CPU baseline (one host thread per segment, mutex/condition-
    variable queues) computes the oracle's result bitwise, whatever the
    thread interleaving."""
    u0 = workloads.uniform(np_ * nx, 23, -1, 1)
    for nt in (0, 1, 40):
        assert np.array_equal(oracle.run_threaded(u0, np_, 0.27, nt), oracle.run(u0, 0.27, nt))


@pytest.mark.parametrize("n,nt", [(1, 3), (5, 4), (64, 10), (300, 40)])
@pytest.mark.parametrize("fma", [False, True])
def test_cone_equals_full_run(n, nt, fma):
    u0 = workloads.uniform(n, 8, -1, 1)
    full = oracle.run(u0, 0.4, nt, fma=fma)
    idx = np.arange(n)
    assert np.array_equal(oracle.cone(u0, 0.4, nt, idx, fma=fma), full)


# --- 9. FP32 storage with the compensated update ------------------------------------------------

def test_f32c_exact_on_dyadics():
    """Small integers with r = 1/4: every binary32 operation is exact, so the
    compensated form equals exact rational evolution for any block length T."""
    for n in (1, 2, 5, 8):
        u0 = workloads.small_ints(n, 40 + n)
        exact = exact_evolve([int(x) for x in u0], Fraction(1, 4), 8)
        for T in (1, 3, 8, 100):
            got = oracle.run_f32c(u0.astype(np.float32), 0.25, 8, T)
            assert [Fraction(float(x)) for x in got] == exact


def test_f32c_block_of_one_is_plain_binary32():
    """With T = 1 the correction term starts at zero every step and TwoSum's
    pair rounds back to its sum, so each step is plain binary32 Eq. 2 with each
    operation rounded once (checked with exact fractions rounded to binary32)."""
    rng = np.random.Generator(np.random.PCG64(12))
    n = 13
    u = rng.uniform(-2, 2, n).astype(np.float32)
    rf = np.float32(0.3)
    got = oracle.run_f32c(u, rf, 1, 1)
    F = lambda x: Fraction(float(x))
    for i in range(n):
        ul, uc, ur = F(u[(i - 1) % n]), F(u[i]), F(u[(i + 1) % n])
        t1 = F(rn32(ul - 2 * uc))
        t2 = F(rn32(t1 + ur))
        t3 = F(rn32(F(rf) * t2))
        assert got[i] == rn32(uc + t3), i


@pytest.mark.parametrize("T", [2, 3, 5])
def test_f32c_blocks_longer_than_one_by_value(T):
    """T > 1 on non-dyadic binary32 data: the carried low part, the TwoSum
    error term and the end-of-block rounding are each checked by value against
    the compensated form written out with every binary32 operation rounded
    once (exact fractions), including a shorter last block."""
    rng = np.random.Generator(np.random.PCG64(20 + T))
    n = 11
    u = rng.uniform(-2, 2, n).astype(np.float32)
    rf = np.float32(0.3)
    nt = 2 * T + 1
    want = compensated_exact(u, rf, nt, T)
    got = oracle.run_f32c(u, rf, nt, T)
    assert [float(x) for x in got] == [float(x) for x in want]
    # the low part matters here: plain binary32 steps (T = 1) give other bits
    assert [float(x) for x in oracle.run_f32c(u, rf, nt, 1)] != [float(x) for x in want]


def test_f32c_error_bound_and_benefit():
    """Against the FP64 oracle the compensated form loses at most about one
    binary32 rounding per block; longer blocks are more accurate."""
    n, nt, r = 256, 400, 0.25
    u0 = workloads.modes(n, [1, 7, 64])
    ref = oracle.run(u0, r, nt)
    u32 = u0.astype(np.float32)
    ulp = np.spacing(np.float32(np.max(np.abs(u0))))
    errs = {}
    for T in (1, 8, 32):
        got = oracle.run_f32c(u32, np.float32(r), nt, T).astype(np.float64)
        errs[T] = np.max(np.abs(got - ref))
        bound = (nt / T + 2) * float(ulp)
        assert errs[T] <= bound, (T, errs[T], bound)
    assert errs[32] < errs[1]


def test_total_matches_exact_sum_within_bound():
    u = workloads.uniform(100000, 30, -1, 1)
    s = oracle.total(u)
    assert abs(s - math.fsum(u)) <= u.size * EPS * np.sum(np.abs(u))
