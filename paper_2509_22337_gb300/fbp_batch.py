"""Binding of include/fbp_batch.h (batched form); argument marshalling only."""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import fbp as F


class fbp_graph_desc(C.Structure):
    _fields_ = [("n_vars", C.c_int32), ("n_factors", C.c_int32), ("factor_ptr", C.c_void_p),
                ("factor_vars", C.c_void_p), ("factor_type", C.c_void_p), ("factor_param", C.c_void_p),
                ("prior_p1", C.c_void_p), ("evidence", C.c_void_p), ("schedule", F._Spec),
                ("max_iters", C.c_int32), ("tol", C.c_double)]


class fbp_batch_config(C.Structure):
    _fields_ = [("one_launch", C.c_int32), ("static_queue", C.c_int32)]


class fbp_batch_tuning(C.Structure):
    _fields_ = [("engine_grid", C.c_int32), ("engine_cluster", C.c_int32), ("flood_hub_min", C.c_int32),
                ("flood_chunk", C.c_int32), ("engine_fuse_lanes", C.c_int32), ("engine_solo_lanes", C.c_int32),
                ("queue_clusters", C.c_int32)]


def bind(L) -> None:
    vp, i32 = C.c_void_p, C.c_int32
    if not hasattr(L, "fbp_batch_create"):
        return
    L.fbp_batch_create.argtypes = [i32, vp, vp, vp, C.POINTER(vp)]
    L.fbp_batch_create_ex.argtypes = [i32, vp, vp, vp, vp, C.POINTER(vp)]
    L.fbp_batch_create_ex.restype = C.c_int
    L.fbp_batch_one_launch.argtypes = [vp]
    L.fbp_batch_one_launch.restype = C.c_int
    L.fbp_batch_run.argtypes = [vp, vp, vp, vp]
    L.fbp_batch_marginals.argtypes = [vp, i32, vp, C.c_int]
    L.fbp_batch_messages_export.argtypes = [vp, i32, vp]
    L.fbp_batch_reset.argtypes = [vp]
    L.fbp_batch_set_tuning.argtypes = [vp, vp]
    L.fbp_batch_get_stats.argtypes = [vp, C.POINTER(F.fbp_stats)]
    L.fbp_batch_destroy.argtypes = [vp]
    L.fbp_batch_destroy.restype = None
    for n in ("fbp_batch_create", "fbp_batch_run", "fbp_batch_marginals", "fbp_batch_messages_export",
              "fbp_batch_reset", "fbp_batch_set_tuning", "fbp_batch_get_stats"):
        getattr(L, n).restype = C.c_int
    from . import fbp_serve as S
    S.bind(L)


def fbp_batch_create(graphs, schedules, max_iters, tols, alloc="torch", stream=None, one_launch=None,
                     static_queue=None):
    """graphs: list of FactorGraph; schedules: list of strategy names; max_iters,
    tols: per-graph lists; one_launch / static_queue: the form of the batch
    (include/fbp_batch.h; None for both = the library's default).  Returns the
    handle."""
    L = F.load()
    n = len(graphs)
    descs = (fbp_graph_desc * max(n, 1))()
    keep = []
    for i, g in enumerate(graphs):
        arrs = F._graph_arrays(g)
        keep.append(arrs)
        fp, fv, ft, fpar, pr, ev = arrs
        spec, k2 = F._spec(schedules[i])
        keep.append(k2)
        descs[i] = fbp_graph_desc(int(g.n_vars), int(fp.shape[0] - 1), fp.ctypes.data, fv.ctypes.data,
                                  ft.ctypes.data, fpar.ctypes.data, pr.ctypes.data, ev.ctypes.data, spec,
                                  int(max_iters[i]), float(tols[i]))
    if alloc == "torch":
        if F._default_alloc is None:
            F._default_alloc = F.torch_allocator()
        alloc = F._default_alloc
    out = C.c_void_p()
    cfg = None
    if one_launch is not None or static_queue is not None:
        cfg = fbp_batch_config(1 if one_launch else 0, 0 if static_queue is False else 1)
    F._check(L.fbp_batch_create_ex(n, C.addressof(descs), None if alloc is None else C.addressof(alloc),
                                   F._stream_ptr(stream), None if cfg is None else C.addressof(cfg), C.byref(out)))
    return out.value


def fbp_batch_run(b, n):
    it = np.zeros(max(n, 1), np.int32)
    res = np.zeros(max(n, 1), np.float64)
    st = np.zeros(max(n, 1), np.int32)
    rc = F._check(F.load().fbp_batch_run(b, it.ctypes.data, res.ctypes.data, st.ctypes.data))
    return rc, it[:n], res[:n], st[:n]


def fbp_batch_marginals(b, graph, n_vars, out=None):
    if out is not None and hasattr(out, "data_ptr"):
        F._check(F.load().fbp_batch_marginals(b, int(graph), out.data_ptr(), 1))
        return out
    p = np.empty(max(int(n_vars), 1), np.float32)
    F._check(F.load().fbp_batch_marginals(b, int(graph), p.ctypes.data, 0))
    return p[:n_vars]


def fbp_batch_messages_export(b, graph, n_edges):
    out = np.empty(2 * max(int(n_edges), 1), np.float32)
    F._check(F.load().fbp_batch_messages_export(b, int(graph), out.ctypes.data))
    return out[: 2 * n_edges].reshape(-1, 2)


def fbp_batch_reset(b):
    return F._check(F.load().fbp_batch_reset(b))


def fbp_batch_set_tuning(b, engine_grid=0, engine_cluster=0, flood_hub_min=0, flood_chunk=0, engine_fuse_lanes=-1,
                         engine_solo_lanes=-1, queue_clusters=0):
    t = fbp_batch_tuning(int(engine_grid), int(engine_cluster), int(flood_hub_min), int(flood_chunk),
                         int(engine_fuse_lanes), int(engine_solo_lanes), int(queue_clusters))
    return F._check(F.load().fbp_batch_set_tuning(b, C.addressof(t)))


def fbp_batch_get_stats(b):
    s = F.fbp_stats()
    F._check(F.load().fbp_batch_get_stats(b, C.byref(s)))
    return {k: getattr(s, k) for k, _ in F.fbp_stats._fields_}


def fbp_batch_destroy(b):
    if b:
        F.load().fbp_batch_destroy(b)


class Batch:
    """Owner of one batch handle."""

    def __init__(self, graphs, schedules, max_iters, tols, stream=None, one_launch=None, static_queue=None):
        self.graphs = graphs
        self.n = len(graphs)
        self.h = fbp_batch_create(graphs, schedules, max_iters, tols, stream=stream, one_launch=one_launch,
                                  static_queue=static_queue)
        self.one_launch = bool(F.load().fbp_batch_one_launch(self.h))
        # the form's name for the tuner: static members in the member queue
        # unless asked otherwise (the library falls back to the level engine
        # where the queue cannot launch; the queue's knobs are then no-ops)
        self.form = "one" if self.one_launch else ("engine" if static_queue is False else "queue")

    def run(self):
        return fbp_batch_run(self.h, self.n)

    def marginals(self, i, out=None):
        return fbp_batch_marginals(self.h, i, self.graphs[i].n_vars, out)

    def messages(self, i):
        return fbp_batch_messages_export(self.h, i, self.graphs[i].n_edges)

    def reset(self):
        return fbp_batch_reset(self.h)

    def tune(self, engine_grid=0, engine_cluster=0, flood_hub_min=0, flood_chunk=0, engine_fuse_lanes=-1,
             engine_solo_lanes=-1, queue_clusters=0):
        return fbp_batch_set_tuning(self.h, engine_grid, engine_cluster, flood_hub_min, flood_chunk,
                                    engine_fuse_lanes, engine_solo_lanes, queue_clusters)

    def stats(self):
        return fbp_batch_get_stats(self.h)

    def close(self):
        if getattr(self, "h", None):
            fbp_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass
