"""CPU oracle for the periodic 1D heat stencil (paper Section 2, Eq. 2).

TEST INFRASTRUCTURE ONLY.  Only the test suite, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package.  The GPU library
(``paper_2307_01117_gb300``) never imports it and shares no code with it.

The arithmetic lives in ``heat_oracle.c`` (plain C, binary64, built with
``-O2 -ffp-contract=off -fno-fast-math``).  This module compiles it with gcc
on first use and exposes numpy-level wrappers:

* ``coef(k, dt, dx)``        -- r = k*dt/dx^2 (Eq. 2, h^2 reading of the denominator)
* ``run(u0, r, nt, fma)``    -- nt steps of Eq. 2 on the periodic ring (unsegmented)
* ``run_segmented(u0, np_, r, nt)`` -- the segmented algorithm with SPSC ghost queues
  (Section 2, parallel algorithm), single-threaded
* ``run_threaded(u0, np_, r, nt)`` -- the same with one host thread per segment
  (``heat_threaded.c``; the threaded CPU baseline)
* ``cone(u0, r, nt, idx, fma)`` -- u^nt at selected points from their light cone
* ``run_f32c(u0, rf, nt, T)`` -- FP32 storage with the compensated update
* ``total(u)``               -- left-to-right FP64 sum (conservation diagnostic)
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "heat_oracle.c")
_SRC_THREADED = os.path.join(_HERE, "heat_threaded.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

CFLAGS = ["-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-std=gnu99", "-pthread"]


def build(force: bool = False) -> str:
    """Compile heat_oracle.c into oracle/_build/liboracle.so (idempotent)."""
    os.makedirs(_BUILD, exist_ok=True)
    srcs = [_SRC, _SRC_THREADED]
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(os.path.getmtime(p) for p in srcs):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", *CFLAGS, "-o", tmp, *srcs, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        d, i64, i32, ip = ctypes.c_double, ctypes.c_int64, ctypes.c_int32, ctypes.c_int
        vp = ctypes.c_void_p
        lib.heat_oracle_r.restype = d
        lib.heat_oracle_r.argtypes = [d, d, d]
        lib.heat_oracle_run.restype = ip
        lib.heat_oracle_run.argtypes = [vp, vp, i64, d, i64, ip]
        lib.heat_oracle_run_segmented.restype = ip
        lib.heat_oracle_run_segmented.argtypes = [vp, i64, i32, d, i64]
        lib.heat_threaded_run.restype = ip
        lib.heat_threaded_run.argtypes = [vp, i64, i32, d, i64]
        lib.heat_oracle_cone.restype = ip
        lib.heat_oracle_cone.argtypes = [vp, i64, d, i64, vp, i64, vp, ip]
        lib.heat_oracle_run_f32c.restype = ip
        lib.heat_oracle_run_f32c.argtypes = [vp, i64, ctypes.c_float, i64, i64]
        lib.heat_oracle_sum.restype = d
        lib.heat_oracle_sum.argtypes = [vp, i64]
        _lib = lib
        return lib


def _f64(u) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(u, dtype=np.float64)).copy()


def coef(k: float, dt: float, dx: float) -> float:
    """r = (k*dt)/(dx*dx), the Eq. 2 coefficient under the h^2 reading."""
    return _load().heat_oracle_r(float(k), float(dt), float(dx))


def run(u0, r: float, nt: int, fma: bool = False) -> np.ndarray:
    """u^nt from u^0 by nt forward-Euler steps of Eq. 2 on the periodic ring."""
    u = _f64(u0)
    work = np.empty_like(u)
    rc = _load().heat_oracle_run(u.ctypes.data, work.ctypes.data, u.size, float(r), int(nt), int(bool(fma)))
    if rc != 0:
        raise ValueError(f"heat_oracle_run failed ({rc})")
    return u


def run_segmented(u0, np_: int, r: float, nt: int) -> np.ndarray:
    """The paper's segmented algorithm: np_ segments exchanging ghosts through queues."""
    u = _f64(u0)
    if u.size % np_ != 0:
        raise ValueError("ring length must be np_ * nx")
    rc = _load().heat_oracle_run_segmented(u.ctypes.data, u.size // np_, int(np_), float(r), int(nt))
    if rc != 0:
        raise ValueError(f"heat_oracle_run_segmented failed ({rc})")
    return u


def run_threaded(u0, np_: int, r: float, nt: int) -> np.ndarray:
    """The segmented algorithm with one host thread per segment and mutex/condition-
    variable SPSC ghost queues (heat_threaded.c: the threaded CPU baseline)."""
    u = _f64(u0)
    if u.size % np_ != 0:
        raise ValueError("ring length must be np_ * nx")
    rc = _load().heat_threaded_run(u.ctypes.data, u.size // np_, int(np_), float(r), int(nt))
    if rc != 0:
        raise ValueError(f"heat_threaded_run failed ({rc})")
    return u


def cone(u0, r: float, nt: int, idx, fma: bool = False) -> np.ndarray:
    """u^nt[idx] recomputed from each point's (2nt+1)-wide light cone."""
    u = np.ascontiguousarray(np.asarray(u0, dtype=np.float64))
    ix = np.ascontiguousarray(np.asarray(idx, dtype=np.int64))
    out = np.empty(ix.size, dtype=np.float64)
    rc = _load().heat_oracle_cone(u.ctypes.data, u.size, float(r), int(nt), ix.ctypes.data, ix.size,
                                  out.ctypes.data, int(bool(fma)))
    if rc != 0:
        raise ValueError(f"heat_oracle_cone failed ({rc})")
    return out


def run_f32c(u0, rf: float, nt: int, T: int = 1) -> np.ndarray:
    """FP32-stored state advanced with the TwoSum-compensated update, blocks of T steps."""
    u = np.ascontiguousarray(np.asarray(u0, dtype=np.float32)).copy()
    rc = _load().heat_oracle_run_f32c(u.ctypes.data, u.size, ctypes.c_float(np.float32(rf)), int(nt), int(T))
    if rc != 0:
        raise ValueError(f"heat_oracle_run_f32c failed ({rc})")
    return u


def total(u) -> float:
    """Left-to-right FP64 sum of u."""
    a = np.ascontiguousarray(np.asarray(u, dtype=np.float64))
    return _load().heat_oracle_sum(a.ctypes.data, a.size)
