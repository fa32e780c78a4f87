"""Binding of include/fbp_serve.h (served form); argument marshalling only.

The server's scheduling, admission and every kernel run inside libfbp.so (a
native worker thread); this module converts arguments and keeps the host
result buffers of pending requests alive.
"""
from __future__ import annotations

import ctypes as C
import threading

import numpy as np

from . import fbp as F

FBP_REQ_QUEUED, FBP_REQ_RUNNING, FBP_REQ_DONE, FBP_REQ_FAILED = range(4)


class fbp_server_config(C.Structure):
    _fields_ = [("hbm_budget_bytes", C.c_int64), ("max_inflight", C.c_int32), ("iters_per_tick", C.c_int32)]


class fbp_request_info(C.Structure):
    _fields_ = [("state", C.c_int32), ("status", C.c_int32), ("iters", C.c_int32), ("session", C.c_int32),
                ("residual", C.c_double), ("queue_ms", C.c_double), ("latency_ms", C.c_double),
                ("device_ms", C.c_double)]


class fbp_server_stats(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("completed", C.c_int64), ("failed", C.c_int64),
                ("ticks", C.c_int64), ("kernel_launches", C.c_int64), ("resident_bytes", C.c_int64),
                ("peak_resident_bytes", C.c_int64), ("sessions_resident", C.c_int32),
                ("sessions_waiting", C.c_int32), ("sessions_warming", C.c_int32), ("peak_inflight", C.c_int32)]


def bind(L) -> None:
    if not hasattr(L, "fbp_server_create"):
        return
    vp, i32, i64 = C.c_void_p, C.c_int32, C.c_int64
    L.fbp_server_create.argtypes = [C.POINTER(fbp_server_config), C.POINTER(vp)]
    L.fbp_server_session_open.argtypes = [vp, vp, C.POINTER(i32)]
    L.fbp_server_session_close.argtypes = [vp, i32]
    L.fbp_server_submit.argtypes = [vp, i32, i32, C.c_int8, vp, C.c_int, C.POINTER(i64)]
    L.fbp_server_poll.argtypes = [vp, i64, C.POINTER(fbp_request_info)]
    L.fbp_server_wait.argtypes = [vp, i64, C.POINTER(fbp_request_info)]
    L.fbp_server_drain.argtypes = [vp]
    L.fbp_server_get_stats.argtypes = [vp, C.POINTER(fbp_server_stats)]
    L.fbp_server_destroy.argtypes = [vp]
    L.fbp_server_destroy.restype = None
    for n in ("fbp_server_create", "fbp_server_session_open", "fbp_server_session_close", "fbp_server_submit",
              "fbp_server_poll", "fbp_server_wait", "fbp_server_drain", "fbp_server_get_stats"):
        getattr(L, n).restype = C.c_int


def _info(i: fbp_request_info) -> dict:
    return {k: getattr(i, k) for k, _ in fbp_request_info._fields_}


def fbp_server_create(hbm_budget_bytes: int = 0, max_inflight: int = 0, iters_per_tick: int = 0):
    cfg = fbp_server_config(int(hbm_budget_bytes), int(max_inflight), int(iters_per_tick))
    h = C.c_void_p()
    F._check(F.load().fbp_server_create(C.byref(cfg), C.byref(h)))
    return h


def fbp_server_session_open(srv, graph, strategy: str = "PARALL", max_iters: int = 500, tol: float = 1e-6,
                            edge_rank=None, factor_rank=None) -> int:
    from .fbp_batch import fbp_graph_desc
    fp, fv, ft, fpar, pr, ev = F._graph_arrays(graph)
    spec, keep = F._spec(strategy, edge_rank, factor_rank)
    d = fbp_graph_desc(int(graph.n_vars), int(fp.shape[0] - 1), fp.ctypes.data, fv.ctypes.data, ft.ctypes.data,
                       fpar.ctypes.data, pr.ctypes.data, ev.ctypes.data, spec, int(max_iters), float(tol))
    sid = C.c_int32()
    F._check(F.load().fbp_server_session_open(srv, C.byref(d), C.byref(sid)))
    del keep
    return sid.value


def fbp_server_session_close(srv, session: int) -> int:
    return F._check(F.load().fbp_server_session_close(srv, int(session)))


def fbp_server_submit(srv, session: int, var: int, value: int, result=None) -> int:
    """result: None, a float32 numpy array (host) or a CUDA float32 tensor of n_vars."""
    ptr, dev = None, 0
    if result is not None:
        if hasattr(result, "data_ptr"):
            ptr, dev = result.data_ptr(), 1
        else:
            assert result.dtype == np.float32 and result.flags["C_CONTIGUOUS"]
            ptr = result.ctypes.data
    t = C.c_int64()
    F._check(F.load().fbp_server_submit(srv, int(session), int(var), int(value), ptr, dev, C.byref(t)))
    return t.value


def fbp_server_poll(srv, ticket: int) -> dict:
    i = fbp_request_info()
    F._check(F.load().fbp_server_poll(srv, int(ticket), C.byref(i)))
    return _info(i)


def fbp_server_wait(srv, ticket: int) -> dict:
    i = fbp_request_info()
    F._check(F.load().fbp_server_wait(srv, int(ticket), C.byref(i)))
    return _info(i)


def fbp_server_drain(srv) -> int:
    return F._check(F.load().fbp_server_drain(srv))


def fbp_server_get_stats(srv) -> dict:
    s = fbp_server_stats()
    F._check(F.load().fbp_server_get_stats(srv, C.byref(s)))
    return {k: getattr(s, k) for k, _ in fbp_server_stats._fields_}


def fbp_server_destroy(srv) -> None:
    if srv:
        F.load().fbp_server_destroy(srv)


class Server:
    """Owner of one server handle; keeps each pending request's result buffer alive."""

    def __init__(self, hbm_budget_bytes: int = 0, max_inflight: int = 0, iters_per_tick: int = 0):
        self.h = fbp_server_create(hbm_budget_bytes, max_inflight, iters_per_tick)
        self._results: dict[int, object] = {}
        self._lock = threading.Lock()
        self.n_vars: dict[int, int] = {}

    def open(self, graph, strategy="PARALL", max_iters=500, tol=1e-6, **ranks) -> int:
        sid = fbp_server_session_open(self.h, graph, strategy, max_iters, tol, **ranks)
        self.n_vars[sid] = int(graph.n_vars)
        return sid

    def close_session(self, sid: int) -> None:
        fbp_server_session_close(self.h, sid)

    def submit(self, sid: int, var: int, value: int, result=True) -> int:
        """result=True allocates a host float32 array for the marginals."""
        buf = np.empty(max(self.n_vars.get(sid, 0), 1), np.float32) if result is True else result
        t = fbp_server_submit(self.h, sid, var, value, buf)
        if buf is not None:
            with self._lock:
                self._results[t] = buf
        return t

    def poll(self, ticket: int) -> dict:
        return fbp_server_poll(self.h, ticket)

    def wait(self, ticket: int):
        """(info, marginals or None) once the request is done."""
        info = fbp_server_wait(self.h, ticket)
        with self._lock:
            buf = self._results.pop(ticket, None)
        return info, buf

    def drain(self) -> None:
        fbp_server_drain(self.h)

    def stats(self) -> dict:
        return fbp_server_get_stats(self.h)

    def close(self) -> None:
        if getattr(self, "h", None):
            fbp_server_destroy(self.h)
            self.h = None
            self._results.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass
