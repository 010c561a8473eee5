"""ctypes binding of libheat.so (include/heat.h), argument marshalling only.

Every function keeps the C name and raises ``HeatError`` on a non-zero status.
Arrays are numpy binary64 on the host, or torch CUDA tensors / raw device
pointers for the ``*_device`` calls.  There is no CPU fallback: if libheat.so
is missing or cannot load, every call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libheat.so")

HEAT_F64, HEAT_F32C = 0, 1
HEAT_OK, HEAT_EINVAL, HEAT_ENOMEM, HEAT_ECUDA, HEAT_ETIMEOUT, HEAT_ESTATE, HEAT_ENOTSUP = 0, -1, -2, -3, -4, -5, -6
HEAT_FORM_PLAIN, HEAT_FORM_PERSIST, HEAT_FORM_TBLOCK, HEAT_FORM_AUTO, HEAT_FORM_CLUSTER = 0, 1, 2, 3, 4
HEAT_FORM_PERSIST_TB = 5
HEAT_ARITH_EXACT, HEAT_ARITH_FMA = 0, 1

FORMS = {"plain": HEAT_FORM_PLAIN, "persist": HEAT_FORM_PERSIST, "tblock": HEAT_FORM_TBLOCK, "auto": HEAT_FORM_AUTO,
         "cluster": HEAT_FORM_CLUSTER, "persist_tb": HEAT_FORM_PERSIST_TB}
DTYPES = {"f64": HEAT_F64, "f32c": HEAT_F32C}


class HeatError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {heat_strerror(code)} ({code})")


_lock = threading.Lock()
_lib = None

# C prototypes: name -> (restype, argtypes)
_vp, _i64, _i32, _int, _d = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int, ctypes.c_double
_PROTOS = {
    "heat_create": (_int, [ctypes.POINTER(_vp), _i64, _i32, _d, _d, _d, _int]),
    "heat_destroy": (None, [_vp]),
    "heat_set": (_int, [_vp, _vp, _i64]),
    "heat_get": (_int, [_vp, _vp, _i64]),
    "heat_set_device": (_int, [_vp, _vp, _i64]),
    "heat_get_device": (_int, [_vp, _vp, _i64]),
    "heat_run": (_int, [_vp, _i64]),
    "heat_sync": (_int, [_vp]),
    "heat_set_stream": (_int, [_vp, _vp]),
    "heat_set_form": (_int, [_vp, _int, _int]),
    "heat_set_arith": (_int, [_vp, _int]),
    "heat_set_segments": (_int, [_vp, _int]),
    "heat_set_emulation": (_int, [_vp, _int]),
    "heat_get_emulation": (_int, [_vp, ctypes.POINTER(ctypes.c_int)]),
    "heat_set_split": (_int, [_vp, _int]),
    "heat_set_layout": (_int, [_vp, _int]),
    "heat_set_graphs": (_int, [_vp, _int]),
    "heat_sum": (_int, [_vp, ctypes.POINTER(_d)]),
    "heat_steps": (_int, [_vp, ctypes.POINTER(_i64)]),
    "heat_last_run": (_int, [_vp, ctypes.POINTER(_int), ctypes.POINTER(_int), ctypes.POINTER(_i64),
                             ctypes.POINTER(_int)]),
    "heat_info": (_int, [_vp, ctypes.POINTER(_i64), ctypes.POINTER(_i32), ctypes.POINTER(_d), ctypes.POINTER(_int)]),
    "heat_state_ptr": (_int, [_vp, ctypes.POINTER(_vp)]),
    "heat_set_wait_limit": (_int, [_vp, _i64]),
    "heat_inject_stall": (_int, [_vp, _i32, _i64]),
    "heat_batch_create": (_int, [ctypes.POINTER(_vp), _i64, _int]),
    "heat_batch_destroy": (None, [_vp]),
    "heat_batch_add": (_int, [_vp, _i64, _i32, _d, _d, _d, _i64, _vp, ctypes.POINTER(_i32)]),
    "heat_batch_add_device": (_int, [_vp, _i64, _i32, _d, _d, _d, _i64, _vp, ctypes.POINTER(_i32)]),
    "heat_batch_get_device": (_int, [_vp, _i32, _vp, _i64]),
    "heat_batch_run": (_int, [_vp, _i64]),
    "heat_batch_sync": (_int, [_vp]),
    "heat_batch_query": (_int, [_vp, _i32, ctypes.POINTER(_i64), ctypes.POINTER(_i64)]),
    "heat_batch_get": (_int, [_vp, _i32, _vp, _i64]),
    "heat_batch_remove": (_int, [_vp, _i32]),
    "heat_batch_set_tuning": (_int, [_vp, _int, _i64]),
    "heat_batch_autotune": (_int, [_vp, ctypes.POINTER(_int), ctypes.POINTER(_i64)]),
    "heat_batch_set_stream": (_int, [_vp, _vp]),
    "heat_batch_set_ctas_per_sm": (_int, [_vp, _int]),
    "heat_batch_set_wait_limit": (_int, [_vp, _i64]),
    "heat_batch_set_graphs": (_int, [_vp, _int]),
    "heat_batch_set_emulation": (_int, [_vp, _int]),
    "heat_batch_inject_stall": (_int, [_vp, _i32, _i64, _i64]),
    "heat_batch_save": (_int, [_vp]),
    "heat_batch_restore": (_int, [_vp]),
    "heat_batch_info": (_int, [_vp, ctypes.POINTER(_i32), ctypes.POINTER(_i64), ctypes.POINTER(_i64)]),
    "heat_run_noalloc": (_int, [_vp, _vp, _i64, _d, _d, _d, _i64, _int, _vp]),
    "heat_server_create": (_int, [ctypes.POINTER(_vp), _i64, _int, _i32, _int, _int]),
    "heat_server_destroy": (None, [_vp]),
    "heat_server_submit": (_int, [_vp, _i64, _d, _d, _d, _i64, _vp, ctypes.POINTER(_i32)]),
    "heat_server_poll": (_int, [_vp, ctypes.POINTER(_i32), _i32, ctypes.POINTER(_i32)]),
    "heat_server_get_device": (_int, [_vp, _i32, _vp, _i64, _vp]),
    "heat_server_release": (_int, [_vp, _i32]),
    "heat_server_info": (_int, [_vp, ctypes.POINTER(_i64), ctypes.POINTER(_i32), ctypes.POINTER(_int),
                                ctypes.POINTER(_i64)]),
    "heat_server_set_limits": (_int, [_vp, _i64, _i64]),
    "heat_probe_pipes": (_int, [_vp, ctypes.POINTER(_d), ctypes.POINTER(_d), ctypes.POINTER(_d)]),
    "heat_strerror": (ctypes.c_char_p, [_int]),
}


def lib() -> ctypes.CDLL:
    """Load libheat.so (raises if it was not built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2307_01117_gb300.build.build()")
            l = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in _PROTOS.items():
                fn = getattr(l, name)
                fn.restype = res
                fn.argtypes = args
            _lib = l
        return _lib


def _check(code: int, where: str) -> None:
    if code != HEAT_OK:
        raise HeatError(code, where)


def _dev_ptr(x) -> int:
    """Device address of a torch CUDA tensor, or an int address."""
    if isinstance(x, int):
        return x
    ptr = getattr(x, "data_ptr", None)
    if ptr is None:
        raise TypeError("expected a torch CUDA tensor or an int device address")
    if not x.is_cuda or not x.is_contiguous():
        raise ValueError("device tensor must be a contiguous CUDA tensor")
    return int(ptr())


def heat_strerror(code: int) -> str:
    return lib().heat_strerror(int(code)).decode()


def heat_create(nx: int, np_: int, k: float, dt: float, dx: float, dtype: int = HEAT_F64) -> int:
    h = _vp()
    _check(lib().heat_create(ctypes.byref(h), int(nx), int(np_), float(k), float(dt), float(dx), int(dtype)),
           "heat_create")
    return h.value


def heat_destroy(ctx: int) -> None:
    lib().heat_destroy(ctx)


def heat_set(ctx: int, u) -> None:
    a = np.ascontiguousarray(np.asarray(u, dtype=np.float64))
    _check(lib().heat_set(ctx, a.ctypes.data, a.size), "heat_set")


def heat_get(ctx: int, out: np.ndarray | None = None) -> np.ndarray:
    if out is None:
        nx, np_, _, _ = heat_info(ctx)
        out = np.empty(nx * np_, dtype=np.float64)
    if out.dtype != np.float64 or not out.flags.c_contiguous:
        raise ValueError("out must be a contiguous float64 array")
    _check(lib().heat_get(ctx, out.ctypes.data, out.size), "heat_get")
    return out


def heat_set_device(ctx: int, dev_u, n: int | None = None) -> None:
    n = int(dev_u.numel()) if n is None else int(n)
    _check(lib().heat_set_device(ctx, _dev_ptr(dev_u), n), "heat_set_device")


def heat_get_device(ctx: int, dev_u, n: int | None = None) -> None:
    n = int(dev_u.numel()) if n is None else int(n)
    _check(lib().heat_get_device(ctx, _dev_ptr(dev_u), n), "heat_get_device")


def heat_run(ctx: int, nt: int) -> None:
    _check(lib().heat_run(ctx, int(nt)), "heat_run")


def heat_sync(ctx: int) -> None:
    _check(lib().heat_sync(ctx), "heat_sync")


def heat_set_stream(ctx: int, stream) -> None:
    """stream: a torch.cuda.Stream, a raw cudaStream_t int, or None."""
    handle = None if stream is None else int(getattr(stream, "cuda_stream", stream))
    _check(lib().heat_set_stream(ctx, handle), "heat_set_stream")


def heat_set_form(ctx: int, form, T: int = 0) -> None:
    f = FORMS[form] if isinstance(form, str) else int(form)
    _check(lib().heat_set_form(ctx, f, int(T)), "heat_set_form")


def heat_set_segments(ctx: int, segments: int) -> None:
    _check(lib().heat_set_segments(ctx, int(segments)), "heat_set_segments")


def heat_set_emulation(ctx: int, share: int) -> None:
    _check(lib().heat_set_emulation(ctx, int(share)), "heat_set_emulation")


def heat_get_emulation(ctx: int) -> int:
    share = ctypes.c_int(0)
    _check(lib().heat_get_emulation(ctx, ctypes.byref(share)), "heat_get_emulation")
    return share.value


def heat_set_graphs(ctx: int, enable: bool) -> None:
    _check(lib().heat_set_graphs(ctx, int(bool(enable))), "heat_set_graphs")


def heat_set_layout(ctx: int, layout: int) -> None:
    _check(lib().heat_set_layout(ctx, int(layout)), "heat_set_layout")


def heat_set_split(ctx: int, level: int) -> None:
    _check(lib().heat_set_split(ctx, int(level)), "heat_set_split")


def heat_set_arith(ctx: int, arith: int) -> None:
    _check(lib().heat_set_arith(ctx, int(arith)), "heat_set_arith")


def heat_sum(ctx: int) -> float:
    out = _d()
    _check(lib().heat_sum(ctx, ctypes.byref(out)), "heat_sum")
    return out.value


def heat_steps(ctx: int) -> int:
    out = _i64()
    _check(lib().heat_steps(ctx, ctypes.byref(out)), "heat_steps")
    return out.value


def heat_last_run(ctx: int) -> dict:
    """Form, block depth T, stencil launches and segments of the last heat_run."""
    f, T, n, sg = _int(), _int(), _i64(), _int()
    _check(lib().heat_last_run(ctx, ctypes.byref(f), ctypes.byref(T), ctypes.byref(n), ctypes.byref(sg)),
           "heat_last_run")
    names = {v: k for k, v in FORMS.items()}
    return {"form": names.get(f.value, str(f.value)), "T": T.value, "launches": n.value, "segments": sg.value}


def heat_info(ctx: int) -> tuple[int, int, float, int]:
    nx, np_, r, dt = _i64(), _i32(), _d(), _int()
    _check(lib().heat_info(ctx, ctypes.byref(nx), ctypes.byref(np_), ctypes.byref(r), ctypes.byref(dt)), "heat_info")
    return nx.value, np_.value, r.value, dt.value


def heat_state_ptr(ctx: int) -> int:
    out = _vp()
    _check(lib().heat_state_ptr(ctx, ctypes.byref(out)), "heat_state_ptr")
    return out.value


def heat_set_wait_limit(ctx: int, ns: int) -> None:
    _check(lib().heat_set_wait_limit(ctx, int(ns)), "heat_set_wait_limit")


def heat_inject_stall(ctx: int, segment: int, from_step: int = 0) -> None:
    _check(lib().heat_inject_stall(ctx, int(segment), int(from_step)), "heat_inject_stall")


def heat_run_noalloc(dev_u0, dev_u, n: int, k: float, dt: float, dx: float, nt: int,
                     arith: int = HEAT_ARITH_EXACT, stream=None) -> None:
    """Allocation-free run: u^nt of dev_u0 into dev_u (device tensors or addresses)."""
    handle = None if stream is None else int(getattr(stream, "cuda_stream", stream))
    _check(lib().heat_run_noalloc(_dev_ptr(dev_u0), _dev_ptr(dev_u), int(n), float(k), float(dt), float(dx),
                                  int(nt), int(arith), handle), "heat_run_noalloc")


def heat_probe_pipes(stream=None) -> dict:
    """Measured lane operations per second: binary64 FMA, binary64 add, integer ALU."""
    handle = None if stream is None else int(getattr(stream, "cuda_stream", stream))
    f, a, i = _d(), _d(), _d()
    _check(lib().heat_probe_pipes(handle, ctypes.byref(f), ctypes.byref(a), ctypes.byref(i)), "heat_probe_pipes")
    return {"dfma_lane_ops_per_s": f.value, "dadd_lane_ops_per_s": a.value, "alu_lane_ops_per_s": i.value}


def heat_server_create(capacity_points: int, dtype: int = HEAT_F64, max_requests: int = 4096, T: int = 0,
                       ctas_per_sm: int = 0) -> int:
    h = _vp()
    _check(lib().heat_server_create(ctypes.byref(h), int(capacity_points), int(dtype), int(max_requests), int(T),
                                    int(ctas_per_sm)), "heat_server_create")
    return h.value


def heat_server_destroy(s: int) -> None:
    lib().heat_server_destroy(s)


def heat_server_submit(s: int, n: int, k: float, dt: float, dx: float, nt: int, dev_u) -> int:
    rid = _i32()
    _check(lib().heat_server_submit(s, int(n), float(k), float(dt), float(dx), int(nt), _dev_ptr(dev_u),
                                    ctypes.byref(rid)), "heat_server_submit")
    return rid.value


_poll_buf = (_i32 * 65536)()
_poll_lock = threading.Lock()


def heat_server_poll(s: int, max_ids: int = 65536) -> list:
    """Ids of the requests completed since the last poll (no waiting)."""
    l, cnt = lib(), _i32()
    with _poll_lock:
        _check(l.heat_server_poll(s, _poll_buf, min(int(max_ids), 65536), ctypes.byref(cnt)), "heat_server_poll")
        return [_poll_buf[i] for i in range(cnt.value)]


def heat_server_get_device(s: int, req: int, dev_u, n: int, event=None) -> None:
    """Queue the completed request's state into dev_u; `event` (a torch.cuda.Event
    or a raw cudaEvent_t) is recorded behind the copy."""
    ev = None if event is None else int(getattr(event, "cuda_event", event))
    _check(lib().heat_server_get_device(s, int(req), _dev_ptr(dev_u), int(n), ev), "heat_server_get_device")


def heat_server_release(s: int, req: int) -> None:
    _check(lib().heat_server_release(s, int(req)), "heat_server_release")


def heat_server_info(s: int) -> dict:
    ps, fl, run, nl = _i64(), _i32(), _int(), _i64()
    _check(lib().heat_server_info(s, ctypes.byref(ps), ctypes.byref(fl), ctypes.byref(run), ctypes.byref(nl)),
           "heat_server_info")
    return {"point_steps": ps.value, "in_flight": fl.value, "running": bool(run.value), "launches": nl.value}


def heat_server_set_limits(s: int, wait_ns: int = 0, idle_ns: int = 0) -> None:
    _check(lib().heat_server_set_limits(s, int(wait_ns), int(idle_ns)), "heat_server_set_limits")


def heat_batch_create(capacity_points: int, dtype: int = HEAT_F64) -> int:
    h = _vp()
    _check(lib().heat_batch_create(ctypes.byref(h), int(capacity_points), int(dtype)), "heat_batch_create")
    return h.value


def heat_batch_destroy(b: int) -> None:
    lib().heat_batch_destroy(b)


def heat_batch_add(b: int, nx: int, np_: int, k: float, dt: float, dx: float, nt: int, u) -> int:
    a = np.ascontiguousarray(np.asarray(u, dtype=np.float64))
    if a.size != int(nx) * int(np_):
        raise ValueError("initial state must have nx*np values")
    rid = _i32()
    _check(lib().heat_batch_add(b, int(nx), int(np_), float(k), float(dt), float(dx), int(nt), a.ctypes.data,
                                ctypes.byref(rid)), "heat_batch_add")
    return rid.value


def heat_batch_add_device(b: int, nx: int, np_: int, k: float, dt: float, dx: float, nt: int, dev_u) -> int:
    rid = _i32()
    _check(lib().heat_batch_add_device(b, int(nx), int(np_), float(k), float(dt), float(dx), int(nt),
                                       _dev_ptr(dev_u), ctypes.byref(rid)), "heat_batch_add_device")
    return rid.value


def heat_batch_get_device(b: int, ring: int, dev_u, n: int) -> None:
    _check(lib().heat_batch_get_device(b, int(ring), _dev_ptr(dev_u), int(n)), "heat_batch_get_device")


def heat_batch_run(b: int, max_steps: int = 0) -> None:
    _check(lib().heat_batch_run(b, int(max_steps)), "heat_batch_run")


def heat_batch_sync(b: int) -> None:
    _check(lib().heat_batch_sync(b), "heat_batch_sync")


def heat_batch_query(b: int, ring: int) -> tuple[int, int]:
    d, l = _i64(), _i64()
    _check(lib().heat_batch_query(b, int(ring), ctypes.byref(d), ctypes.byref(l)), "heat_batch_query")
    return d.value, l.value


def heat_batch_get(b: int, ring: int, n: int, out: np.ndarray | None = None) -> np.ndarray:
    if out is None:
        out = np.empty(int(n), dtype=np.float64)
    _check(lib().heat_batch_get(b, int(ring), out.ctypes.data, int(n)), "heat_batch_get")
    return out


def heat_batch_remove(b: int, ring: int) -> None:
    _check(lib().heat_batch_remove(b, int(ring)), "heat_batch_remove")


def heat_batch_set_tuning(b: int, T: int = 0, window_points: int = 0) -> None:
    _check(lib().heat_batch_set_tuning(b, int(T), int(window_points)), "heat_batch_set_tuning")


def heat_batch_autotune(b: int) -> tuple[int, int]:
    T, sg = _int(), _i64()
    _check(lib().heat_batch_autotune(b, ctypes.byref(T), ctypes.byref(sg)), "heat_batch_autotune")
    return T.value, sg.value


def heat_batch_set_stream(b: int, stream) -> None:
    handle = None if stream is None else int(getattr(stream, "cuda_stream", stream))
    _check(lib().heat_batch_set_stream(b, handle), "heat_batch_set_stream")


def heat_batch_set_ctas_per_sm(b: int, ctas: int) -> None:
    _check(lib().heat_batch_set_ctas_per_sm(b, int(ctas)), "heat_batch_set_ctas_per_sm")


def heat_batch_set_graphs(b: int, enable: bool) -> None:
    _check(lib().heat_batch_set_graphs(b, int(bool(enable))), "heat_batch_set_graphs")


def heat_batch_set_emulation(b: int, share: int) -> None:
    _check(lib().heat_batch_set_emulation(b, int(share)), "heat_batch_set_emulation")


def heat_batch_set_wait_limit(b: int, ns: int) -> None:
    _check(lib().heat_batch_set_wait_limit(b, int(ns)), "heat_batch_set_wait_limit")


def heat_batch_inject_stall(b: int, ring: int, segment: int = 0, from_level: int = 0) -> None:
    _check(lib().heat_batch_inject_stall(b, int(ring), int(segment), int(from_level)), "heat_batch_inject_stall")


def heat_batch_save(b: int) -> None:
    _check(lib().heat_batch_save(b), "heat_batch_save")


def heat_batch_restore(b: int) -> None:
    _check(lib().heat_batch_restore(b), "heat_batch_restore")


def heat_batch_info(b: int) -> dict:
    live, free, ps = _i32(), _i64(), _i64()
    _check(lib().heat_batch_info(b, ctypes.byref(live), ctypes.byref(free), ctypes.byref(ps)), "heat_batch_info")
    return {"live": live.value, "largest_free": free.value, "last_point_steps": ps.value}


class Heat:
    """Owning wrapper: a ring of np_ x nx points advanced by Eq. 2 on the GPU."""

    def __init__(self, nx: int, np_: int, k: float, dt: float, dx: float, dtype="f64", form="auto", T: int = 0,
                 arith: int = HEAT_ARITH_EXACT, stream=None):
        self.ctx = heat_create(nx, np_, k, dt, dx, DTYPES[dtype] if isinstance(dtype, str) else int(dtype))
        try:
            heat_set_form(self.ctx, form, T)
            heat_set_arith(self.ctx, arith)
            if stream is not None:
                heat_set_stream(self.ctx, stream)
        except Exception:
            self.close()
            raise
        self.nx, self.np_ = int(nx), int(np_)
        self.n = self.nx * self.np_

    def set(self, u) -> "Heat":
        heat_set(self.ctx, u)
        return self

    def get(self) -> np.ndarray:
        return heat_get(self.ctx)

    def run(self, nt: int) -> "Heat":
        heat_run(self.ctx, nt)
        return self

    def sync(self) -> None:
        heat_sync(self.ctx)

    def sum(self) -> float:
        return heat_sum(self.ctx)

    @property
    def r(self) -> float:
        return heat_info(self.ctx)[2]

    @property
    def steps(self) -> int:
        return heat_steps(self.ctx)

    def close(self) -> None:
        if getattr(self, "ctx", None):
            heat_destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
