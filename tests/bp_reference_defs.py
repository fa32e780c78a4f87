"""Plain definitions used to pin the oracle, written independently of it.

- `factor_table`: the factor function f_a of each logical type as a dense
  table over all assignments, from the type's logical meaning (the readings of
  the noisy types are stated with each); `terms_table`: the table of a generic
  factor given as an explicit term list (each term a sub-factor that is w_t on
  the assignments it matches and 0 elsewhere, Eq. 4).
- `brute_force_marginals`: exact marginals by enumerating every assignment of
  a small graph (the quantity BP reproduces exactly on trees, Sec. 3.2).
- `sync_bp` / `seq_bp`: textbook synchronous and round-robin sequential BP on
  dense tables (Eq. 1-3), the two update strategies the paper contrasts in
  Sec. 2.1, used to pin the oracle's level-mode and Definition-2 executions.

None of this imports or mirrors the oracle's code: it works on dense tables
rather than term lists and on Python dictionaries rather than CSR arrays.
"""
from __future__ import annotations

import itertools

import numpy as np

AND, OR, NOT, EQ, NOISY_IMPLY, NOISY_AND, PRIOR, TERMS = range(8)


def factor_value(ftype: int, p: float, x: tuple) -> float:
    """f_a at assignment x (premises first, output last)."""
    *prem, y = x
    allx = all(v == 1 for v in prem)
    anyx = any(v == 1 for v in prem)
    if ftype == AND:
        return 1.0 if y == int(allx) else 0.0
    if ftype == OR:
        return 1.0 if y == int(anyx) else 0.0
    if ftype == NOT:
        return 1.0 if y == 1 - prem[0] else 0.0
    if ftype == EQ:
        return 1.0 if len(set(x)) == 1 else 0.0
    if ftype == NOISY_AND:  # y only through the rule: fires with p when all premises hold
        if allx:
            return p if y == 1 else 1.0 - p
        return 1.0 if y == 0 else 0.0
    if ftype == NOISY_IMPLY:  # p: x1 & ... & xn -> y; y free when a premise fails
        if allx:
            return p if y == 1 else 1.0 - p
        return 1.0
    if ftype == PRIOR:
        return p if y == 1 else 1.0 - p
    raise ValueError(ftype)


def factor_table(ftype: int, p: float, b: int) -> np.ndarray:
    t = np.zeros((2,) * b)
    for x in itertools.product((0, 1), repeat=b):
        t[x] = factor_value(ftype, p, x)
    return t


def terms_table(ind: np.ndarray, w: np.ndarray) -> np.ndarray:
    """f(x) = sum over terms t of w_t [x matches t], where term t fixes
    variable j to ind[t, j] in {0, 1} or leaves it free (-1)."""
    l, b = ind.shape
    t = np.zeros((2,) * b)
    for x in itertools.product((0, 1), repeat=b):
        t[x] = sum(w[k] for k in range(l) if all(ind[k, j] < 0 or ind[k, j] == x[j] for j in range(b)))
    return t


def table_of(g, a: int) -> np.ndarray:
    """Dense table of factor a of graph g (typed, or generic with its terms)."""
    b = int(g.factor_ptr[a + 1] - g.factor_ptr[a])
    if int(g.factor_type[a]) == TERMS:
        tp, ti, tw = g.terms
        off = int(sum((tp[k + 1] - tp[k]) * (g.factor_ptr[k + 1] - g.factor_ptr[k]) for k in range(a)))
        l = int(tp[a + 1] - tp[a])
        return terms_table(np.asarray(ti[off:off + l * b]).reshape(l, b), np.asarray(tw[tp[a]:tp[a + 1]]))
    return factor_table(int(g.factor_type[a]), float(g.factor_param[a]), b)


def dense_message(table: np.ndarray, mu: np.ndarray, v: int) -> np.ndarray:
    """Eq. (2): sum over all assignments with x_v fixed of f times the incoming
    messages of the other variables."""
    b = table.ndim
    out = np.zeros(2)
    for x in itertools.product((0, 1), repeat=b):
        w = table[x]
        for j in range(b):
            if j != v:
                w *= mu[j][x[j]]
        out[x[v]] += w
    return out


def phi_of(g, v: int) -> np.ndarray:
    ev = int(g.evidence[v])
    if ev == 0:
        return np.array([1.0, 0.0])
    if ev == 1:
        return np.array([0.0, 1.0])
    p = float(g.prior_p1[v])
    if not np.isnan(p):
        return np.array([1.0 - p, p])
    return np.array([1.0, 1.0])


def brute_force_marginals(g) -> tuple[np.ndarray, float]:
    """Exact P(x_v = 1) by enumeration; returns (p1, Z)."""
    n = g.n_vars
    assert n <= 20
    X = ((np.arange(1 << n)[:, None] >> np.arange(n)[None, :]) & 1).astype(np.int64)
    w = np.ones(1 << n)
    for v in range(n):
        ph = phi_of(g, v)
        w *= ph[X[:, v]]
    for a in range(g.n_factors):
        row = g.factor_vars[g.factor_ptr[a]:g.factor_ptr[a + 1]]
        tab = table_of(g, a)
        w *= tab[tuple(X[:, int(v)] for v in row)]
    Z = w.sum()
    return (w[:, None] * X).sum(0) / Z if Z > 0 else np.full(n, np.nan), Z


def _structures(g):
    rows = [g.factor_vars[g.factor_ptr[a]:g.factor_ptr[a + 1]].tolist() for a in range(g.n_factors)]
    tabs = [table_of(g, a) for a in range(g.n_factors)]
    nbrs = {v: [] for v in range(g.n_vars)}
    for a, r in enumerate(rows):
        for v in r:
            nbrs[v].append(a)
    return rows, tabs, nbrs


def _norm(m):
    s = m.sum()
    return m / s if s > 0 and np.isfinite(s) else np.array([0.5, 0.5])


def _v2a(g, msgs, nbrs, v, a):
    m = phi_of(g, v).copy()
    for b in nbrs[v]:
        if b != a:
            m = m * msgs[(b, v)]
    return _norm(m)


def sync_bp(g, iters: int):
    """Synchronous BP: every message of iteration t from iteration t-1's."""
    rows, tabs, nbrs = _structures(g)
    msgs = {(a, v): np.array([0.5, 0.5]) for a, r in enumerate(rows) for v in r}
    for _ in range(iters):
        new = {}
        for a, r in enumerate(rows):
            mu = [_v2a(g, msgs, nbrs, u, a) for u in r]
            for i, v in enumerate(r):
                new[(a, v)] = _norm(dense_message(tabs[a], mu, i))
        msgs = new
    return msgs


def seq_bp(g, iters: int, order: list[tuple[int, int]]):
    """Round-robin asynchronous BP (Sec. 2.1): the factor-to-variable messages
    are recomputed one at a time in `order`, each from the most recent values."""
    rows, tabs, nbrs = _structures(g)
    msgs = {(a, v): np.array([0.5, 0.5]) for a, r in enumerate(rows) for v in r}
    for _ in range(iters):
        for (a, v) in order:
            r = rows[a]
            mu = [_v2a(g, msgs, nbrs, u, a) for u in r]
            msgs[(a, v)] = _norm(dense_message(tabs[a], mu, r.index(v)))
    return msgs


def marginals_from(g, msgs):
    _, _, nbrs = _structures(g)
    out = np.zeros(g.n_vars)
    for v in range(g.n_vars):
        m = phi_of(g, v).copy()
        for a in nbrs[v]:
            m = m * msgs[(a, v)]
        out[v] = _norm(m)[1]
    return out


def msgs_to_edges(g, msgs) -> np.ndarray:
    """Dictionary of messages -> [E, 2] in factor-major edge order."""
    out = np.zeros((g.n_edges, 2))
    for a in range(g.n_factors):
        for e in range(int(g.factor_ptr[a]), int(g.factor_ptr[a + 1])):
            out[e] = msgs[(a, int(g.factor_vars[e]))]
    return out
