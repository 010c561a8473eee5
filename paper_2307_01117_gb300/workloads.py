"""Seeded synthetic inputs for the periodic heat ring.

This module only draws and lays out input data (initial states, ring tables,
request streams).  It holds none of the stencil's arithmetic, so both the GPU
tests and the CPU oracle tests may use it.

Workload shapes follow the paper's model problem (Section 2: u(0, x_i) = x_i on a
periodic ring; Section 6: 1,000,000 nodes and 1000 time steps) and the library's
benchmark set:

* ``ramp``          -- u[g] = g*dx, the paper's initial condition (Section 2).
* ``uniform_plus_mode`` -- U[0,1) from a PCG64 seed plus one Fourier mode.
* ``modes``         -- a sum of discrete Fourier modes sin(2 pi m g / N).
* ``ring_table``    -- many independent rings of uneven size (batched runs).
* ``request_stream``-- Poisson arrivals of heat solves (serving).

Phases m*g are reduced modulo N in exact integer arithmetic before scaling, so
sin(2 pi m g / N) stays accurate at N = 2^28.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


def ramp(n: int, dx: float = 1.0) -> np.ndarray:
    """u[g] = g*dx for g = 0..n-1 (the paper's u(0, x_i) = x_i)."""
    return np.arange(n, dtype=np.float64) * float(dx)


def mode(n: int, m: int, amplitude: float = 1.0) -> np.ndarray:
    """amplitude * sin(2 pi m g / n), phase reduced as (m*g) mod n in int64."""
    g = np.arange(n, dtype=np.int64)
    ph = (np.int64(m) * g) % np.int64(n)
    return amplitude * np.sin((2.0 * np.pi / n) * ph.astype(np.float64))


def modes(n: int, ms, amplitude: float = 1.0) -> np.ndarray:
    out = np.zeros(n, dtype=np.float64)
    for m in ms:
        out += mode(n, int(m), amplitude)
    return out


def uniform(n: int, seed: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.uniform(lo, hi, size=n)


def uniform_plus_mode(n: int, seed: int = 0, m: int = 3, amplitude: float = 1.0) -> np.ndarray:
    """U[0,1) from PCG64(seed) plus amplitude*sin(2 pi m g / n)."""
    u = uniform(n, seed)
    u += mode(n, m, amplitude)
    return u


def small_ints(n: int, seed: int, lo: int = -8, hi: int = 8) -> np.ndarray:
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.integers(lo, hi + 1, size=n).astype(np.float64)


@dataclass(frozen=True)
class RingSpec:
    """One independent ring: np_ partitions of nx points, nt steps, coefficient r."""
    nx: int
    np_: int
    nt: int
    r: float
    seed: int

    @property
    def n(self) -> int:
        return self.nx * self.np_


def ring_table(count: int, seed: int = 1, n_lo: float = 1e3, n_hi: float = 1e6,
               nt_lo: int = 100, nt_hi: int = 5000, r_lo: float = 0.05, r_hi: float = 0.5,
               nps=(1, 2, 4, 8, 16)) -> list[RingSpec]:
    """Rings with N log-uniform in [n_lo, n_hi], np uniform over nps,
    nx = round(N/np) (>= 1), nt uniform in [nt_lo, nt_hi], r uniform in [r_lo, r_hi]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for i in range(count):
        n_target = float(np.exp(rng.uniform(np.log(n_lo), np.log(n_hi))))
        np_ = int(rng.choice(np.asarray(nps)))
        nx = max(1, int(round(n_target / np_)))
        nt = int(rng.integers(nt_lo, nt_hi + 1))
        r = float(rng.uniform(r_lo, r_hi))
        out.append(RingSpec(nx=nx, np_=np_, nt=nt, r=r, seed=int(rng.integers(0, 2**31 - 1))))
    return out


def ring_initial(spec: RingSpec) -> np.ndarray:
    """u ~ U[-1, 1) for one ring of a table, from the ring's own seed."""
    return uniform(spec.n, spec.seed, -1.0, 1.0)


@dataclass(frozen=True)
class Request:
    t_arrive: float
    n: int
    nt: int
    r: float
    f32c: bool
    seed: int


def request_stream(rate: float, duration: float, seed: int = 2, n_lo: float = 1e4, n_hi: float = 1e7,
                   nt_lo: int = 100, nt_hi: int = 2000, r_lo: float = 0.05, r_hi: float = 0.5,
                   f32c_share: float = 0.5) -> list[Request]:
    """Poisson arrivals at `rate` per second over `duration` seconds."""
    rng = np.random.Generator(np.random.PCG64(seed))
    t = 0.0
    out = []
    while True:
        t += float(rng.exponential(1.0 / rate))
        if t >= duration:
            break
        n = max(1, int(round(float(np.exp(rng.uniform(np.log(n_lo), np.log(n_hi)))))))
        nt = int(rng.integers(nt_lo, nt_hi + 1))
        r = float(rng.uniform(r_lo, r_hi))
        f32c = bool(rng.uniform() < f32c_share)
        out.append(Request(t_arrive=t, n=n, nt=nt, r=r, f32c=f32c, seed=int(rng.integers(0, 2**31 - 1))))
    return out
