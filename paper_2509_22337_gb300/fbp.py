"""Thin Python binding of the C ABI in include/fbp.h (argument marshalling only).

Every function here has the name of the C entry point it calls and does no
arithmetic of its own: all belief-propagation work runs in libfbp.so's CUDA
kernels.  PyTorch provides device memory (its caching allocator is handed to
the library as the device allocator) and the CUDA stream.

Loading fails loudly (RuntimeError) when libfbp.so has not been built: there is
no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import build as _build

FBP_OK, FBP_NOT_CONVERGED = 0, 1
FBP_ERR_INVALID_ARG, FBP_ERR_OOM, FBP_ERR_CUDA, FBP_ERR_SCHEDULE, FBP_ERR_TIMEOUT = -1, -2, -3, -4, -5
FBP_AND, FBP_OR, FBP_NOT, FBP_EQ, FBP_NOISY_IMPLY, FBP_NOISY_AND, FBP_PRIOR, FBP_TERMS = range(8)
FBP_PARALL, FBP_SEQFIX, FBP_TOPO, FBP_TOPO_FB, FBP_RESIDUAL, FBP_CUSTOM_RANK = range(6)
STRATEGY = dict(PARALL=0, SEQFIX=1, TOPO=2, TOPO_FB=3, RESIDUAL=4, CUSTOM=5, CUSTOM_RANK=5)


class FbpError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"fbp error {code}: {msg}")
        self.code = code


class _Allocator(C.Structure):
    _fields_ = [("alloc", C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)),
                ("free", C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)),
                ("ctx", C.c_void_p)]


class _Spec(C.Structure):
    _fields_ = [("strategy", C.c_int32), ("edge_rank", C.c_void_p), ("factor_rank", C.c_void_p),
                ("residual_buckets", C.c_int32)]


class fbp_stats(C.Structure):
    _fields_ = [("updates", C.c_int64), ("guards", C.c_int64), ("iters", C.c_int32),
                ("levels", C.c_int32), ("residual", C.c_double), ("run_ms", C.c_double),
                ("kernel_launches", C.c_int64)]


_lib = None
_lock = threading.Lock()
_keep = []  # ctypes callbacks that must outlive every graph


def lib_path() -> str:
    return _build.LIB


def load(path: str | None = None):
    """Load libfbp.so (build it first with paper_2509_22337_gb300.build.build())."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = path or lib_path()
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA library not built: {path} is missing "
                               "(run __graft_entry__.build()); there is no CPU fallback")
        L = C.CDLL(path)
        vp, i32, i64, f64 = C.c_void_p, C.c_int32, C.c_int64, C.c_double
        L.fbp_graph_create.argtypes = [i32, i32, vp, vp, vp, vp, vp, vp, vp, vp, C.POINTER(vp)]
        L.fbp_schedule_set.argtypes = [vp, C.POINTER(_Spec)]
        L.fbp_run.argtypes = [vp, i32, f64, C.POINTER(i32), C.POINTER(f64)]
        L.fbp_marginals.argtypes = [vp, vp, C.c_int]
        L.fbp_schedule_levels.argtypes = [vp, C.POINTER(i32), vp, vp]
        L.fbp_schedule_build_host.argtypes = [i32, i32, vp, vp, C.POINTER(_Spec), i32, C.POINTER(i32), vp, vp]
        L.fbp_set_evidence.argtypes = [vp, i32, C.c_int8]
        L.fbp_messages_export.argtypes = [vp, vp]
        L.fbp_messages_import.argtypes = [vp, vp]
        L.fbp_get_stats.argtypes = [vp, C.POINTER(fbp_stats)]
        L.fbp_messages_reset.argtypes = [vp]
        L.fbp_set_option.argtypes = [vp, i32, i64]
        L.fbp_run_fixed_scratch.argtypes = [vp, i32, f64, C.POINTER(i32), C.POINTER(f64)]
        L.fbp_set_factor_terms.argtypes = [vp, vp, vp, vp]
        L.fbp_graph_destroy.argtypes = [vp]
        L.fbp_graph_destroy.restype = None
        L.fbp_last_error.restype = C.c_char_p
        for name in ("fbp_graph_create", "fbp_schedule_set", "fbp_run", "fbp_marginals",
                     "fbp_schedule_levels", "fbp_schedule_build_host", "fbp_set_evidence",
                     "fbp_messages_export", "fbp_messages_import", "fbp_get_stats", "fbp_messages_reset",
                     "fbp_set_option", "fbp_run_fixed_scratch", "fbp_set_factor_terms"):
            getattr(L, name).restype = C.c_int
        _bind_extras(L)
        _lib = L
        return L


def _bind_extras(L) -> None:
    """Batched and serving entry points (declared in include/fbp_batch.h)."""
    from . import fbp_batch as B
    B.bind(L)


def _check(rc: int) -> int:
    if rc < 0:
        raise FbpError(rc, fbp_last_error())
    return rc


def fbp_last_error() -> str:
    return (load().fbp_last_error() or b"").decode()


def _ptr(a):
    return None if a is None else a.ctypes.data


def torch_allocator():
    """fbp_allocator backed by PyTorch's CUDA caching allocator on the current stream."""
    import torch

    def _alloc(n, ctx):
        try:
            return torch.cuda.caching_allocator_alloc(int(n), stream=torch.cuda.current_stream())
        except Exception:  # noqa: BLE001 - reported as NULL -> FBP_ERR_OOM
            return None

    def _free(p, ctx):
        if p:
            torch.cuda.caching_allocator_delete(int(p))

    a = _Allocator(_Allocator._fields_[0][1](_alloc), _Allocator._fields_[1][1](_free), None)
    _keep.append(a)
    return a


_default_alloc = None


def _graph_arrays(g):
    return (np.ascontiguousarray(g.factor_ptr, np.int64), np.ascontiguousarray(g.factor_vars, np.int32),
            np.ascontiguousarray(g.factor_type, np.uint8), np.ascontiguousarray(g.factor_param, np.float32),
            np.ascontiguousarray(g.prior_p1, np.float32), np.ascontiguousarray(g.evidence, np.int8))


def fbp_graph_create(n_vars, n_factors, factor_ptr, factor_vars, factor_type, factor_param,
                     prior_p1=None, evidence=None, alloc="torch", stream=None):
    """Returns an opaque handle (int).  alloc: "torch" (PyTorch caching
    allocator), None (cudaMalloc) or an _Allocator.  stream: a torch.cuda.Stream,
    a raw cudaStream_t int, or None for the current torch stream."""
    global _default_alloc
    L = load()
    fp = np.ascontiguousarray(factor_ptr, np.int64)
    fv = np.ascontiguousarray(factor_vars, np.int32)
    ft = np.ascontiguousarray(factor_type, np.uint8)
    fpar = np.ascontiguousarray(factor_param, np.float32)
    pr = None if prior_p1 is None else np.ascontiguousarray(prior_p1, np.float32)
    ev = None if evidence is None else np.ascontiguousarray(evidence, np.int8)
    if alloc == "torch":
        if _default_alloc is None:
            _default_alloc = torch_allocator()
        alloc = _default_alloc
    s = _stream_ptr(stream)
    out = C.c_void_p()
    _check(L.fbp_graph_create(int(n_vars), int(n_factors), _ptr(fp), _ptr(fv), _ptr(ft), _ptr(fpar),
                              _ptr(pr), _ptr(ev), None if alloc is None else C.addressof(alloc),
                              s, C.byref(out)))
    return out.value


def _stream_ptr(stream):
    if stream is None:
        try:
            import torch
            return torch.cuda.current_stream().cuda_stream or None
        except Exception:  # noqa: BLE001
            return None
    if isinstance(stream, int):
        return stream or None
    return stream.cuda_stream or None


def _spec(strategy, edge_rank=None, factor_rank=None, buckets=0):
    s = STRATEGY[strategy] if isinstance(strategy, str) else int(strategy)
    er = None if edge_rank is None else np.ascontiguousarray(edge_rank, np.int64)
    fr = None if factor_rank is None else np.ascontiguousarray(factor_rank, np.int32)
    return _Spec(s, _ptr(er), _ptr(fr), int(buckets)), (er, fr)


def fbp_schedule_set(g, strategy, edge_rank=None, factor_rank=None, residual_buckets=0):
    spec, keep = _spec(strategy, edge_rank, factor_rank, residual_buckets)
    return _check(load().fbp_schedule_set(g, C.byref(spec)))


def fbp_run(g, max_iters: int, tol: float):
    """Returns (status, iters, residual); status FBP_OK or FBP_NOT_CONVERGED."""
    it, res = C.c_int32(), C.c_double()
    rc = _check(load().fbp_run(g, int(max_iters), float(tol), C.byref(it), C.byref(res)))
    return rc, it.value, res.value


# include/fbp_fixed.h
FBP_FIXED_SCRATCH_MAX_ITERS = 16384


def fbp_run_fixed_scratch(g, max_iters: int, tol: float):
    """fbp_run for a static strategy with no device allocation (per-run scratch
    in the library's static device array; one call at a time per device).
    Returns (status, iters, residual) like fbp_run."""
    it, res = C.c_int32(), C.c_double()
    rc = _check(load().fbp_run_fixed_scratch(g, int(max_iters), float(tol), C.byref(it), C.byref(res)))
    return rc, it.value, res.value


def fbp_marginals(g, n_vars: int, out=None):
    """Host numpy float32 [n_vars] (default) or into a CUDA torch tensor `out`."""
    if out is not None and hasattr(out, "data_ptr"):
        _check(load().fbp_marginals(g, out.data_ptr(), 1))
        return out
    p = np.empty(max(int(n_vars), 1), np.float32)
    _check(load().fbp_marginals(g, p.ctypes.data, 0))
    return p[:n_vars]


def fbp_schedule_levels(g):
    k = C.c_int32()
    _check(load().fbp_schedule_levels(g, C.byref(k), None, None))
    lp = np.zeros(k.value + 1, np.int64)
    _check(load().fbp_schedule_levels(g, C.byref(k), lp.ctypes.data, None))
    le = np.zeros(max(int(lp[-1]), 1), np.int32)
    _check(load().fbp_schedule_levels(g, C.byref(k), lp.ctypes.data, le.ctypes.data))
    return lp, le[: int(lp[-1])]


def fbp_schedule_build_host(n_vars, n_factors, factor_ptr, factor_vars, strategy, edge_rank=None,
                            factor_rank=None, backward=False):
    """Host-only Algorithm 2: (level_ptr, level_edges) as fbp_schedule_set builds them."""
    L = load()
    fp = np.ascontiguousarray(factor_ptr, np.int64)
    fv = np.ascontiguousarray(factor_vars, np.int32)
    spec, keep = _spec(strategy, edge_rank, factor_rank)
    k = C.c_int32()
    _check(L.fbp_schedule_build_host(int(n_vars), int(n_factors), _ptr(fp), _ptr(fv), C.byref(spec),
                                     int(backward), C.byref(k), None, None))
    lp = np.zeros(k.value + 1, np.int64)
    le = np.zeros(max(int(fp[-1]), 1), np.int32)
    _check(L.fbp_schedule_build_host(int(n_vars), int(n_factors), _ptr(fp), _ptr(fv), C.byref(spec),
                                     int(backward), C.byref(k), lp.ctypes.data, le.ctypes.data))
    return lp, le[: int(fp[-1])]


def fbp_set_factor_terms(g, term_ptr, term_ind, term_w) -> int:
    """Term lists of the generic (FBP_TERMS) factors (layout: include/fbp.h)."""
    tp = np.ascontiguousarray(term_ptr, np.int64)
    ti = np.ascontiguousarray(term_ind, np.int8)
    tw = np.ascontiguousarray(term_w, np.float32)
    return _check(load().fbp_set_factor_terms(g, tp.ctypes.data, ti.ctypes.data if ti.size else None,
                                              tw.ctypes.data if tw.size else None))


def fbp_set_evidence(g, var: int, value: int):
    return _check(load().fbp_set_evidence(g, int(var), int(value)))


def fbp_messages_export(g, n_edges: int) -> np.ndarray:
    out = np.empty(2 * max(int(n_edges), 1), np.float32)
    _check(load().fbp_messages_export(g, out.ctypes.data))
    return out[: 2 * n_edges].reshape(-1, 2)


def fbp_messages_import(g, a2v) -> int:
    a = np.ascontiguousarray(a2v, np.float32).reshape(-1)
    return _check(load().fbp_messages_import(g, a.ctypes.data if a.size else None))


FBP_OPT_SPIN_LIMIT, FBP_OPT_ENGINE_GRID, FBP_OPT_ENGINE, FBP_OPT_ENGINE_CLUSTER = 1, 2, 3, 4
FBP_OPT_FLOOD_HUB_MIN, FBP_OPT_FLOOD_CHUNK, FBP_OPT_RESIDUAL_DEVICE = 5, 6, 7
FBP_OPT_ENGINE_FUSE_LANES, FBP_OPT_ENGINE_SOLO_LANES = 8, 9


def fbp_set_option(g, option: int, value: int) -> int:
    return _check(load().fbp_set_option(g, int(option), int(value)))


def fbp_messages_reset(g) -> int:
    return _check(load().fbp_messages_reset(g))


def fbp_get_stats(g) -> dict:
    s = fbp_stats()
    _check(load().fbp_get_stats(g, C.byref(s)))
    return {k: getattr(s, k) for k, _ in fbp_stats._fields_}


def fbp_graph_destroy(g) -> None:
    if g:
        load().fbp_graph_destroy(g)


class Graph:
    """Convenience owner of one graph handle built from a FactorGraph."""

    def __init__(self, fg, strategy="PARALL", alloc="torch", stream=None, **spec):
        fp, fv, ft, fpar, pr, ev = _graph_arrays(fg)
        self.n_vars, self.n_edges = int(fg.n_vars), int(fp[-1])
        self.h = fbp_graph_create(fg.n_vars, fp.shape[0] - 1, fp, fv, ft, fpar, pr, ev,
                                  alloc=alloc, stream=stream)
        if getattr(fg, "terms", None) is not None:
            fbp_set_factor_terms(self.h, *fg.terms)
        if strategy != "PARALL" or spec:
            fbp_schedule_set(self.h, strategy, **spec)

    def run(self, max_iters: int, tol: float = 0.0):
        return fbp_run(self.h, max_iters, tol)

    def run_fixed_scratch(self, max_iters: int, tol: float = 0.0):
        return fbp_run_fixed_scratch(self.h, max_iters, tol)

    def marginals(self, out=None):
        return fbp_marginals(self.h, self.n_vars, out)

    def levels(self):
        return fbp_schedule_levels(self.h)

    def messages(self):
        return fbp_messages_export(self.h, self.n_edges)

    def set_messages(self, a2v):
        return fbp_messages_import(self.h, a2v)

    def set_option(self, option, value):
        return fbp_set_option(self.h, option, value)

    def reset(self):
        return fbp_messages_reset(self.h)

    def set_evidence(self, var, value):
        return fbp_set_evidence(self.h, var, value)

    def stats(self):
        return fbp_get_stats(self.h)

    def close(self):
        if getattr(self, "h", None):
            fbp_graph_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass
