"""ctypes wrapper around the FP64 sequential oracle (oracle/fbp_oracle.c).

TEST INFRASTRUCTURE: the checker for the CUDA path.  Only the tests, the
package smoke check and the benchmark's CPU-baseline leg may import this
module.  It imports nothing from the CUDA package; the two meet only through
the seeded input generators' FactorGraph arrays.

Every function mirrors one C entry point; see the C file for the paper
passages each follows.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fbp_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liborc.so")
_lock = threading.Lock()
_lib = None

PARALL, SEQFIX, TOPO, TOPO_FB, RESIDUAL, CUSTOM = range(6)
STRATEGY = dict(PARALL=PARALL, SEQFIX=SEQFIX, TOPO=TOPO, TOPO_FB=TOPO_FB, RESIDUAL=RESIDUAL,
                CUSTOM=CUSTOM)

_p = np.ctypeslib.ndpointer
_i64 = _p(dtype=np.int64, flags="C_CONTIGUOUS")
_i32 = _p(dtype=np.int32, flags="C_CONTIGUOUS")
_u8 = _p(dtype=np.uint8, flags="C_CONTIGUOUS")
_i8 = _p(dtype=np.int8, flags="C_CONTIGUOUS")
_f32 = _p(dtype=np.float32, flags="C_CONTIGUOUS")
_f64 = _p(dtype=np.float64, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (strict IEEE double arithmetic: no fast-math,
    no FMA contraction) into oracle/_build/liborc.so."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    base = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math", "-Wall",
            "-Wno-unused-function", "-o", tmp, _SRC, "-lm"]
    # OpenMP only spreads a level's independent updates over host threads
    # (orc_set_threads); without it the oracle runs on one thread
    if subprocess.run(base + ["-fopenmp"], capture_output=True).returncode != 0:
        subprocess.check_call(base)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            L.orc_terms.argtypes = [C.c_int, C.c_int, C.c_double, _i8, _f64, C.c_int]
            L.orc_terms.restype = C.c_int
            L.orc_alg1.argtypes = [C.c_int, C.c_int, C.c_int, _i8, _f64, _f64, C.c_int, C.c_int]
            L.orc_alg1.restype = C.c_double
            L.orc_graph_new.argtypes = [C.c_int32, C.c_int32, _i64, _i32, _u8, _f32, _f32, _i8]
            L.orc_graph_new.restype = C.c_void_p
            L.orc_graph_free.argtypes = [C.c_void_p]
            L.orc_graph_free.restype = None
            L.orc_set_evidence.argtypes = [C.c_void_p, C.c_int32, C.c_int8, C.c_float]
            L.orc_set_evidence.restype = C.c_int
            L.orc_set_terms.argtypes = [C.c_void_p, _i64, _i8, _f64]
            L.orc_set_terms.restype = C.c_int
            L.orc_ranks.argtypes = [C.c_void_p, C.c_int, C.c_void_p, C.c_int, _i64]
            L.orc_ranks.restype = C.c_int
            for fn in (L.orc_levels_literal, L.orc_levels_nbr):
                fn.argtypes = [C.c_void_p, _i64, C.c_void_p, C.c_int64, _i64, _i32]
                fn.restype = C.c_int64
            L.orc_in_ne.argtypes = [C.c_void_p, C.c_int64, C.c_int64]
            L.orc_in_ne.restype = C.c_int
            L.orc_run.argtypes = [C.c_void_p, C.c_int, C.c_void_p, C.c_int, C.c_double, C.c_int,
                                  C.c_int, _f64, C.POINTER(C.c_int32), C.POINTER(C.c_double),
                                  C.c_void_p, C.POINTER(C.c_int64), C.POINTER(C.c_int64),
                                  C.POINTER(C.c_double)]
            L.orc_run.restype = C.c_int
            L.orc_marginals.argtypes = [C.c_void_p, _f64, _f64]
            L.orc_marginals.restype = C.c_int64
            L.orc_v2a_row.argtypes = [C.c_void_p, _f64, C.c_int32, _f64, C.c_int]
            L.orc_v2a_row.restype = C.c_int
            L.orc_update_edges.argtypes = [C.c_void_p, _f64, C.c_int64, _i64, _f64]
            L.orc_update_edges.restype = C.c_int
            L.orc_residual_classes.argtypes = [C.c_void_p, _f64, C.c_double, _i64, _i64]
            L.orc_residual_classes.restype = C.c_int64
            L.orc_set_threads.argtypes = [C.c_int]
            L.orc_set_threads.restype = C.c_int
            _lib = L
    return _lib


def terms(ftype: int, b: int, p: float, lmax: int | None = None):
    """Term list of a factor (Eq. 4): (indicator[b, l], weights[l])."""
    lmax = lmax or (b + 2)
    ind = np.zeros(b * lmax, dtype=np.int8)
    w = np.zeros(lmax, dtype=np.float64)
    l = lib().orc_terms(int(ftype), int(b), float(p), ind, w, int(lmax))
    if l < 0:
        raise ValueError("invalid factor type/arity")
    return ind.reshape(b, lmax)[:, :l].copy(), w[:l].copy()


def alg1(ind: np.ndarray, w: np.ndarray, mu: np.ndarray, v: int, xv: int) -> float:
    """Algorithm 1 for target variable v and value xv; mu is [b, 2]."""
    b, l = ind.shape
    flat = np.ascontiguousarray(ind, dtype=np.int8).reshape(-1)
    return lib().orc_alg1(b, l, l, flat, np.ascontiguousarray(w, np.float64),
                          np.ascontiguousarray(mu, np.float64).reshape(-1), v, xv)


def message(ftype: int, p: float, mu: np.ndarray, v: int) -> np.ndarray:
    """Normalised mu_{a->v} (unnormalised pair returned as well if needed)."""
    ind, w = terms(ftype, mu.shape[0], p)
    return np.array([alg1(ind, w, mu, v, 0), alg1(ind, w, mu, v, 1)])


class Oracle:
    """One factor graph held by the oracle."""

    def __init__(self, g):
        self.g = g
        self.n_vars = int(g.n_vars)
        self.n_edges = int(g.factor_ptr[-1])
        self._h = lib().orc_graph_new(
            int(g.n_vars), int(g.factor_ptr.shape[0] - 1),
            np.ascontiguousarray(g.factor_ptr, np.int64), np.ascontiguousarray(g.factor_vars, np.int32),
            np.ascontiguousarray(g.factor_type, np.uint8), np.ascontiguousarray(g.factor_param, np.float32),
            np.ascontiguousarray(g.prior_p1, np.float32), np.ascontiguousarray(g.evidence, np.int8))
        if not self._h:
            raise ValueError("oracle rejected the graph")
        if getattr(g, "terms", None) is not None:
            tp, ti, tw = g.terms
            if lib().orc_set_terms(self._h, np.ascontiguousarray(tp, np.int64), np.ascontiguousarray(ti, np.int8),
                                   np.ascontiguousarray(tw, np.float64)) != 0:
                raise ValueError("oracle rejected the term lists")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and _lib is not None:
            _lib.orc_graph_free(h)
            self._h = None

    def set_evidence(self, var: int, value: int, prior: float = float("nan")) -> None:
        if lib().orc_set_evidence(self._h, int(var), int(value), float(prior)) != 0:
            raise ValueError("bad variable")

    def ranks(self, strategy, custom: np.ndarray | None = None, backward: bool = False) -> np.ndarray:
        s = STRATEGY[strategy] if isinstance(strategy, str) else int(strategy)
        r = np.zeros(self.n_edges + 1, dtype=np.int64)
        cbuf = None if custom is None else np.ascontiguousarray(custom, np.int64)
        rc = lib().orc_ranks(self._h, s, None if cbuf is None else cbuf.ctypes.data, int(backward), r)
        if rc != 0:
            raise ValueError(f"rank construction failed ({rc})")
        return r[: self.n_edges]

    def levels(self, rank: np.ndarray, edges: np.ndarray | None = None, literal: bool = False):
        """Algorithm 2: returns (level_ptr[k+1], level_edges[n])."""
        rank = np.ascontiguousarray(rank, np.int64)
        n = self.n_edges if edges is None else int(edges.shape[0])
        eb = None if edges is None else np.ascontiguousarray(edges, np.int64)
        lp = np.zeros(n + 2, dtype=np.int64)
        le = np.zeros(max(n, 1), dtype=np.int32)
        fn = lib().orc_levels_literal if literal else lib().orc_levels_nbr
        k = fn(self._h, rank, None if eb is None else eb.ctypes.data, n, lp, le)
        return lp[: k + 1].copy(), le[:n].copy()

    def in_ne(self, e: int, f: int) -> bool:
        """Definition 1: is edge e in N_E(f)?"""
        return bool(lib().orc_in_ne(self._h, int(e), int(f)))

    def run(self, strategy="PARALL", max_iters: int = 50, tol: float = 0.0,
            custom: np.ndarray | None = None, def2: bool = False, a2v: np.ndarray | None = None,
            history: bool = False, threads: int = 1) -> dict:
        """threads > 1 runs each level's independent updates on that many host
        threads (same results; out["threads"] is the count actually used)."""
        used = lib().orc_set_threads(int(threads))
        try:
            out = self._run(strategy, max_iters, tol, custom, def2, a2v, history)
        finally:
            lib().orc_set_threads(1)
        out["threads"] = used
        return out

    def _run(self, strategy, max_iters, tol, custom, def2, a2v, history) -> dict:
        s = STRATEGY[strategy] if isinstance(strategy, str) else int(strategy)
        init = a2v is not None
        msgs = (np.ascontiguousarray(a2v, np.float64).reshape(-1).copy() if init
                else np.zeros(2 * self.n_edges + 2, dtype=np.float64))
        if msgs.shape[0] < 2 * self.n_edges + 2:
            msgs = np.concatenate([msgs, np.zeros(2 * self.n_edges + 2 - msgs.shape[0])])
        it, res, gd, up, mp = C.c_int32(), C.c_double(), C.c_int64(), C.c_int64(), C.c_double()
        hist = np.zeros(max(max_iters, 1), dtype=np.float64) if history else None
        cbuf = None if custom is None else np.ascontiguousarray(custom, np.int64)
        rc = lib().orc_run(self._h, s, None if cbuf is None else cbuf.ctypes.data, int(max_iters),
                           float(tol), int(def2), int(init), msgs, C.byref(it), C.byref(res),
                           None if hist is None else hist.ctypes.data, C.byref(gd), C.byref(up),
                           C.byref(mp))
        if rc < 0:
            raise ValueError(f"oracle run failed ({rc})")
        out = dict(converged=rc == 0, iters=int(it.value), residual=float(res.value),
                   guards=int(gd.value), updates=int(up.value), min_pos=float(mp.value),
                   a2v=msgs[: 2 * self.n_edges].reshape(-1, 2).copy())
        if hist is not None:
            out["res_hist"] = hist[: out["iters"]].copy()
        return out

    def marginals(self, a2v: np.ndarray) -> np.ndarray:
        p1 = np.zeros(self.n_vars + 1, dtype=np.float64)
        m = np.ascontiguousarray(a2v, np.float64).reshape(-1)
        if m.shape[0] < 2:
            m = np.zeros(2, np.float64)
        lib().orc_marginals(self._h, m, p1)
        return p1[: self.n_vars]

    def v2a_row(self, a2v: np.ndarray, v: int, literal: bool) -> np.ndarray:
        out = np.zeros(2 * self.n_edges + 2, dtype=np.float64)
        lib().orc_v2a_row(self._h, np.ascontiguousarray(a2v, np.float64).reshape(-1), int(v), out,
                          int(literal))
        return out[: 2 * self.n_edges].reshape(-1, 2)

    def update_edges(self, a2v: np.ndarray, edges: np.ndarray) -> np.ndarray:
        """One synchronous update of the listed edges from the given state."""
        edges = np.ascontiguousarray(edges, np.int64)
        out = np.zeros(2 * edges.shape[0] + 2, dtype=np.float64)
        lib().orc_update_edges(self._h, np.ascontiguousarray(a2v, np.float64).reshape(-1),
                               int(edges.shape[0]), edges, out)
        return out[: 2 * edges.shape[0]].reshape(-1, 2)

    def residual_classes(self, dres: np.ndarray, tol: float):
        """The residual strategy's classes from previous-iteration per-edge
        |delta m1| values: (rank per edge, -1 = skipped; active edges)."""
        rank = np.zeros(self.n_edges + 1, dtype=np.int64)
        edges = np.zeros(self.n_edges + 1, dtype=np.int64)
        n = lib().orc_residual_classes(self._h, np.ascontiguousarray(dres, np.float64), float(tol), rank, edges)
        return rank[: self.n_edges].copy(), edges[:n].copy()
