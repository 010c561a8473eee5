"""The oracle's pins catch planted mistakes (CPU only).

Each mutant is a copy of oracle/heat_oracle.c with one plausible mistake
planted in it (a wrong neighbour index, a flipped sign, a dropped or reordered
term, a halved coefficient, a transposed operand, a dropped correction of the
binary32 compensated form, a wrong light-cone index, swapped ghost queues).
The copy is compiled with the oracle's own flags and run through the same kinds
of checks that pin the oracle (exact rational evolution, rounding of each
operation, Fourier-mode decay, conservation, the coefficient's reading, the
compensated form's error bound, light cone and segmented algorithm against the
plain ring).  The unmodified source passes every check; every mutant fails at
least one.  Two more mutants of the threaded CPU baseline (oracle/heat_threaded.c:
edge values sent the wrong way, ghosts taken from the wrong side) must differ
from the plain ring; they run in a child process with a time limit."""
import ctypes
import math
import os
import shutil
import subprocess
import sys
from fractions import Fraction

import numpy as np
import pytest

import oracle
from exact_binary32 import compensated_exact
from paper_2307_01117_gb300 import workloads

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "heat_oracle.c")
EPS = np.finfo(np.float64).eps


class Lib:
    """ctypes view of one compiled copy of heat_oracle.c."""

    def __init__(self, path):
        d, i64, i32, ip, vp = ctypes.c_double, ctypes.c_int64, ctypes.c_int32, ctypes.c_int, ctypes.c_void_p
        self.lib = lib = ctypes.CDLL(path)
        lib.heat_oracle_r.restype = d
        lib.heat_oracle_r.argtypes = [d, d, d]
        lib.heat_oracle_run.restype = ip
        lib.heat_oracle_run.argtypes = [vp, vp, i64, d, i64, ip]
        lib.heat_oracle_run_segmented.restype = ip
        lib.heat_oracle_run_segmented.argtypes = [vp, i64, i32, d, i64]
        lib.heat_oracle_cone.restype = ip
        lib.heat_oracle_cone.argtypes = [vp, i64, d, i64, vp, i64, vp, ip]
        lib.heat_oracle_run_f32c.restype = ip
        lib.heat_oracle_run_f32c.argtypes = [vp, i64, ctypes.c_float, i64, i64]

    def coef(self, k, dt, dx):
        return self.lib.heat_oracle_r(k, dt, dx)

    def run(self, u0, r, nt, fma=False):
        u = np.array(u0, dtype=np.float64)
        w = np.empty_like(u)
        assert self.lib.heat_oracle_run(u.ctypes.data, w.ctypes.data, u.size, r, nt, int(fma)) == 0
        return u

    def segmented(self, u0, np_, r, nt):
        u = np.array(u0, dtype=np.float64)
        assert self.lib.heat_oracle_run_segmented(u.ctypes.data, u.size // np_, np_, r, nt) == 0
        return u

    def cone(self, u0, r, nt, idx):
        u = np.ascontiguousarray(u0, dtype=np.float64)
        ix = np.ascontiguousarray(idx, dtype=np.int64)
        out = np.empty(ix.size)
        assert self.lib.heat_oracle_cone(u.ctypes.data, u.size, r, nt, ix.ctypes.data, ix.size,
                                         out.ctypes.data, 0) == 0
        return out

    def f32c(self, u0, rf, nt, T):
        u = np.array(u0, dtype=np.float32)
        assert self.lib.heat_oracle_run_f32c(u.ctypes.data, u.size, ctypes.c_float(rf), nt, T) == 0
        return u


def rn(q: Fraction) -> float:
    return float(q)   # Fraction -> float rounds to nearest-even


# --- the checks: each returns True when the copy behaves as Eq. 2 says ------------------

def exact_rationals(L):
    rng = np.random.Generator(np.random.PCG64(1))
    for n in (1, 2, 3, 5, 8):
        for r in (Fraction(1, 8), Fraction(1, 4), Fraction(1, 2)):
            u0 = [int(x) for x in rng.integers(-8, 9, n)]
            q = [Fraction(x) for x in u0]
            for nt in range(1, 9):
                q = [q[i] + r * (q[i - 1] - 2 * q[i] + q[(i + 1) % n]) for i in range(n)]
                if [Fraction(float(x)) for x in L.run(np.array(u0, float), float(r), nt)] != q:
                    return False
    return True


def rounding_order(L):
    rng = np.random.Generator(np.random.PCG64(5))
    n = 17
    for _ in range(10):
        u = rng.uniform(-3, 3, n) * 10.0 ** rng.integers(-3, 4, n)
        r = float(rng.uniform(0.01, 0.5))
        got = L.run(u, r, 1)
        for i in range(n):
            ul, uc, ur = Fraction(u[(i - 1) % n]), Fraction(u[i]), Fraction(u[(i + 1) % n])
            t2 = Fraction(rn(Fraction(rn(ul - 2 * uc)) + ur))
            if got[i] != rn(uc + Fraction(rn(Fraction(r) * t2))):
                return False
    return True


def fourier_decay(L):
    n, m, r, nt = 64, 3, 0.25, 50
    u0 = workloads.mode(n, m)
    lam = 1.0 - 4.0 * r * math.sin(math.pi * m / n) ** 2
    return float(np.max(np.abs(L.run(u0, r, nt) - lam ** nt * u0))) <= 8 * nt * EPS


def conservation(L):
    u0 = workloads.uniform(997, 3, -1, 1)
    u = L.run(u0, 0.3, 200)
    return abs(math.fsum(u) - math.fsum(u0)) <= 4 * 200 * 997 * EPS


def coefficient_reading(L):
    # r = k dt / dx^2 (second-order differences: h^2 in Eq. 2's denominator)
    return L.coef(0.5, 1.0, 1.0) == 0.5 and L.coef(1.0, 0.5, 0.5) == 2.0


def fused_reading_close(L):
    u0 = workloads.uniform(500, 4, -1, 1)
    return float(np.max(np.abs(L.run(u0, 0.3, 100, fma=True) - L.run(u0, 0.3, 100)))) <= 1e-12


def compensated_bound(L):
    # about one binary32 rounding per block against binary64, and longer
    # blocks more accurate than plain binary32 (blocks of one step)
    n, nt, r = 256, 400, 0.25
    u0 = workloads.modes(n, [1, 7, 64])
    ref = L.run(u0, r, nt)
    if not np.all(np.isfinite(ref)):
        return False
    ulp = float(np.spacing(np.float32(np.max(np.abs(u0)))))
    err = {T: float(np.max(np.abs(L.f32c(u0, np.float32(r), nt, T).astype(np.float64) - ref))) for T in (1, 32)}
    return err[32] <= (nt / 32 + 2) * ulp and err[32] < err[1]


def compensated_block_of_one(L):
    # with T = 1 the compensated form is plain binary32 Eq. 2 (every
    # intermediate of these small dyadic values is exact)
    u0 = np.array([1.0, -2.0, 0.5, 3.0, -1.25, 0.75, 2.0], np.float32)
    q = [Fraction(float(x)) for x in u0]
    r = Fraction(1, 4)
    for _ in range(3):
        q = [q[i] + r * (q[i - 1] - 2 * q[i] + q[(i + 1) % len(q)]) for i in range(len(q))]
    return [Fraction(float(x)) for x in L.f32c(u0, np.float32(0.25), 3, 1)] == q


def compensated_by_value(L):
    # blocks of 2 and 3 steps on non-dyadic binary32 data against the
    # compensated form with every binary32 operation rounded once
    rng = np.random.Generator(np.random.PCG64(21))
    u = rng.uniform(-2, 2, 9).astype(np.float32)
    for T in (2, 3):
        want = [float(x) for x in compensated_exact(u, np.float32(0.3), 2 * T + 1, T)]
        if [float(x) for x in L.f32c(u, np.float32(0.3), 2 * T + 1, T)] != want:
            return False
    return True


def light_cone(L):
    u0 = workloads.uniform(300, 8, -1, 1)
    idx = [0, 1, 17, 150, 298, 299]
    return np.array_equal(L.cone(u0, 0.3, 40, idx), L.run(u0, 0.3, 40)[idx])


def segmented(L):
    u0 = workloads.uniform(7 * 13, 9, -1, 1)
    return np.array_equal(L.segmented(u0, 7, 0.3, 25), L.run(u0, 0.3, 25))


CHECKS = [exact_rationals, rounding_order, fourier_decay, conservation, coefficient_reading,
          fused_reading_close, compensated_bound, compensated_block_of_one, compensated_by_value, light_cone,
          segmented]

# (name, text in heat_oracle.c, planted replacement)
MUTANTS = [
    ("right neighbour at distance 2", "    double ur = u[(i + 1) % N];\n    v[i] = u[i] + r",
     "    double ur = u[(i + 2) % N];\n    v[i] = u[i] + r"),
    ("flipped sign of 2u", "v[i] = u[i] + r * ((ul - 2.0 * u[i]) + ur);", "v[i] = u[i] + r * ((ul + 2.0 * u[i]) + ur);"),
    ("dropped right neighbour", "v[i] = u[i] + r * ((ul - 2.0 * u[i]) + ur);", "v[i] = u[i] + r * (ul - 2.0 * u[i]);"),
    ("reordered sum", "v[i] = u[i] + r * ((ul - 2.0 * u[i]) + ur);", "v[i] = u[i] + r * (ul + (ur - 2.0 * u[i]));"),
    ("transposed operand", "v[i] = u[i] + r * ((ul - 2.0 * u[i]) + ur);", "v[i] = ul + r * ((ul - 2.0 * u[i]) + ur);"),
    ("halved coefficient (2h reading)", "return (k * dt) / (dx * dx);", "return (k * dt) / (2.0 * dx * dx);"),
    ("fused form without the factor 2", "v[i] = fma(r, fma(-2.0, u[i], ul) + ur, u[i]);",
     "v[i] = fma(r, fma(-1.0, u[i], ul) + ur, u[i]);"),
    ("compensation term dropped", "l2[i] = l[i] + err;", "l2[i] = l[i];"),
    ("low parts left out of the difference", "float d = dh + dl;", "float d = dh;"),
    ("low part not accumulated", "l2[i] = l[i] + err;", "l2[i] = err;"),
    ("TwoSum error without its second term", "float ee = (a - (ss - bb)) + (b - bb);",
     "float ee = (a - (ss - bb));"),
    ("sign of the low parts' 2l flipped", "float dl = (l[im] - 2.0f * l[i]) + l[ip];",
     "float dl = (l[im] + 2.0f * l[i]) + l[ip];"),
    ("low part dropped at the block's end", "u[i] = h[i] + l[i];", "u[i] = h[i];"),
    ("light cone read one place off", "out[q] = w[nt];", "out[q] = w[nt + 1 < W ? nt + 1 : nt];"),
    ("ghost queues swapped", "c[0] = fifo_pop(&from_left[p]);\n      c[nx + 1] = fifo_pop(&from_right[p]);",
     "c[0] = fifo_pop(&from_right[p]);\n      c[nx + 1] = fifo_pop(&from_left[p]);"),
]


def compile_copy(text, tmp_path, name):
    src = tmp_path / f"{name}.c"
    src.write_text(text)
    so = tmp_path / f"{name}.so"
    subprocess.check_call(["gcc", *oracle.CFLAGS, "-o", str(so), str(src), "-lm"])
    return Lib(str(so))


pytestmark = pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")


def test_unmodified_oracle_passes_every_check(tmp_path):
    L = compile_copy(open(SRC).read(), tmp_path, "original")
    failed = [c.__name__ for c in CHECKS if not c(L)]
    assert failed == []


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_is_caught(name, old, new, tmp_path):
    text = open(SRC).read()
    assert text.count(old) == 1, name
    L = compile_copy(text.replace(old, new), tmp_path, "mutant")
    caught = [c.__name__ for c in CHECKS if not c(L)]
    assert caught, f"no check catches: {name}"


# --- the threaded CPU baseline (oracle/heat_threaded.c) -----------------------------------

THREADED_SRC = os.path.join(ROOT, "oracle", "heat_threaded.c")

# (name, text in heat_threaded.c, planted replacement); each mutant still pushes
# and pops one value per queue and step, so none of them can block
THREADED_MUTANTS = [
    ("edge values sent the wrong way", "q_push(g->to_left, c[1]);\n    q_push(g->to_right, c[nx]);",
     "q_push(g->to_left, c[nx]);\n    q_push(g->to_right, c[1]);"),
    ("ghosts taken from the wrong side", "c[0] = q_pop(g->from_left);\n    c[nx + 1] = q_pop(g->from_right);",
     "c[0] = q_pop(g->from_right);\n    c[nx + 1] = q_pop(g->from_left);"),
]

_THREADED_PROBE = r"""
import ctypes, sys
import numpy as np
lib = ctypes.CDLL(sys.argv[1])
d, i64, i32, ip, vp = ctypes.c_double, ctypes.c_int64, ctypes.c_int32, ctypes.c_int, ctypes.c_void_p
lib.heat_threaded_run.restype = ip
lib.heat_threaded_run.argtypes = [vp, i64, i32, d, i64]
lib.heat_oracle_run.restype = ip
lib.heat_oracle_run.argtypes = [vp, vp, i64, d, i64, ip]
rng = np.random.Generator(np.random.PCG64(3))
u0 = rng.uniform(-1, 1, 5 * 7)
a = u0.copy(); w = np.empty_like(a)
assert lib.heat_oracle_run(a.ctypes.data, w.ctypes.data, a.size, 0.3, 20, 0) == 0
b = u0.copy()
assert lib.heat_threaded_run(b.ctypes.data, 7, 5, 0.3, 20) == 0
print("equal" if np.array_equal(a, b) else "differ")
"""


def threaded_equals_plain(threaded_text, tmp_path, name):
    src = tmp_path / f"{name}_threaded.c"
    src.write_text(threaded_text)
    so = tmp_path / f"{name}.so"
    subprocess.check_call(["gcc", *oracle.CFLAGS, "-o", str(so), SRC, str(src), "-lm"])
    p = subprocess.run([sys.executable, "-c", _THREADED_PROBE, str(so)], capture_output=True, text=True, timeout=60)
    assert p.returncode == 0, p.stderr
    return p.stdout.strip() == "equal"


def test_unmodified_threaded_baseline_equals_the_plain_ring(tmp_path):
    assert threaded_equals_plain(open(THREADED_SRC).read(), tmp_path, "original")


@pytest.mark.parametrize("name,old,new", THREADED_MUTANTS, ids=[m[0] for m in THREADED_MUTANTS])
def test_planted_mistake_in_the_threaded_baseline_is_caught(name, old, new, tmp_path):
    text = open(THREADED_SRC).read()
    assert text.count(old) == 1, name
    assert not threaded_equals_plain(text.replace(old, new), tmp_path, "mutant")
