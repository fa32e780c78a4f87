"""Seeded synthetic factor-graph generators.

These stand in for the program-analysis graphs that FastLBP is evaluated on
(SmartFL fault-localisation graphs and BINGO derivation graphs, Sec. 6.1.1),
which are not available here.  Every generator is a pure function of its seed
and size arguments and returns a :class:`FactorGraph` in the input format of
the library's graph-creation call: a factor-major CSR with the output variable
of each logical factor stored last.

This module holds no belief-propagation arithmetic: it only draws structure,
factor types, parameters, priors and evidence.  It is shared by the CUDA path's
tests and benchmark and by the oracle's tests, and imports neither of them.

Factor type codes (the input format; each side of the library/oracle boundary
declares its own copy of these numbers):

    AND=0  OR=1  NOT=2  EQ=3  NOISY_IMPLY=4  NOISY_AND=5  PRIOR=6
    TERMS=7  (generic: the factor's local structure is an explicit term list)
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

AND, OR, NOT, EQ, NOISY_IMPLY, NOISY_AND, PRIOR, TERMS = range(8)
TYPE_NAMES = ("AND", "OR", "NOT", "EQ", "NOISY_IMPLY", "NOISY_AND", "PRIOR", "TERMS")


@dataclass
class FactorGraph:
    """A binary factor graph in factor-major CSR form.

    factor_ptr   int64  [A+1]  row offsets into factor_vars
    factor_vars  int32  [E]    variable ids; premises first, output last
    factor_type  uint8  [A]    type code
    factor_param float32[A]    p for NOISY_IMPLY / NOISY_AND / PRIOR, else 0
    prior_p1     float32[V]    prior P(x=1) or NaN for no prior
    evidence     int8   [V]    -1 none, 0 or 1 clamped value
    terms        optional (term_ptr int64 [A+1], term_ind int8, term_w float64):
                 the term lists of the TERMS factors (others have none); factor
                 a's indicators are a (terms x variables) block, term after
                 term, values 0 / 1 / -1 (free), blocks in factor order
    """

    n_vars: int
    factor_ptr: np.ndarray
    factor_vars: np.ndarray
    factor_type: np.ndarray
    factor_param: np.ndarray
    prior_p1: np.ndarray
    evidence: np.ndarray
    name: str = "graph"
    meta: dict = field(default_factory=dict)
    terms: tuple | None = None

    @property
    def n_factors(self) -> int:
        return int(self.factor_ptr.shape[0] - 1)

    @property
    def n_edges(self) -> int:
        return int(self.factor_ptr[-1])

    def fan(self) -> np.ndarray:
        return np.diff(self.factor_ptr)

    def nbytes(self) -> int:
        return int(sum(a.nbytes for a in (self.factor_ptr, self.factor_vars, self.factor_type,
                                          self.factor_param, self.prior_p1, self.evidence)))


def _csr(rows: list[np.ndarray]) -> tuple[np.ndarray, np.ndarray]:
    lens = np.fromiter((len(r) for r in rows), dtype=np.int64, count=len(rows))
    ptr = np.zeros(len(rows) + 1, dtype=np.int64)
    np.cumsum(lens, out=ptr[1:])
    vars_ = np.concatenate(rows).astype(np.int32) if rows else np.zeros(0, np.int32)
    return ptr, vars_


def _distinct_rows(rng: np.random.Generator, draw, k: np.ndarray, forbid: np.ndarray,
                   kmax: int) -> np.ndarray:
    """Draw a [n, kmax] matrix of ids where the first k[i] entries of row i are
    pairwise distinct and differ from forbid[i].  ``draw(idx, col)`` returns
    fresh candidates for rows ``idx`` in column ``col``; collisions are redrawn."""
    n = k.shape[0]
    out = np.full((n, kmax), -1, dtype=np.int64)
    for col in range(kmax):
        idx = np.nonzero(k > col)[0]
        for _ in range(10000):
            if idx.size == 0:
                break
            cand = draw(idx, col)
            out[idx, col] = cand
            bad = cand == forbid[idx]
            for prev in range(col):
                bad |= cand == out[idx, prev]
            idx = idx[bad]
        else:  # pragma: no cover - only on degenerate size arguments
            raise RuntimeError("could not draw distinct ids")
    return out


def _powerlaw_in(rng: np.random.Generator, lo: np.ndarray, hi: np.ndarray, alpha: float) -> np.ndarray:
    """Integer v in [lo, hi) drawn with weight (v+1)^(-1/(alpha-1)) by inverse CDF of
    the continuous density on [lo, hi)."""
    b = 1.0 / (alpha - 1.0)
    a = 1.0 - b
    u = rng.random(lo.shape[0])
    A = (lo + 1.0) ** a
    B = (hi + 1.0) ** a
    x = (A + u * (B - A)) ** (1.0 / a) - 1.0
    return np.clip(np.floor(x).astype(np.int64), lo, hi - 1)


def _derivation_graph(rng: np.random.Generator, n_tuples: int, rule_concl: np.ndarray,
                      rule_prem: np.ndarray, rule_k: np.ndarray, p_fire: np.ndarray,
                      prior_frac: float, name: str, meta: dict) -> FactorGraph:
    """BINGO's clause/tuple encoding: each rule instance r gets a derivation
    variable d_r = NOISY_AND(premises -> d_r); each derived tuple c gets
    OR({d_r : r concludes c} -> c).  Rules are grouped by conclusion, and each
    conclusion's OR factor follows its rules."""
    n_rules = rule_concl.shape[0]
    order = np.argsort(rule_concl, kind="stable")
    rule_concl = rule_concl[order]
    rule_prem = rule_prem[order]
    rule_k = rule_k[order]
    p_fire = p_fire[order]
    d_ids = n_tuples + np.arange(n_rules, dtype=np.int64)
    n_vars = n_tuples + n_rules

    concl_vals, first, counts = np.unique(rule_concl, return_index=True, return_counts=True)
    n_or = concl_vals.shape[0]
    n_fac = n_rules + n_or
    # factor order: for each conclusion, its rules then its OR factor
    fan = np.empty(n_fac, dtype=np.int64)
    ftype = np.empty(n_fac, dtype=np.uint8)
    fparam = np.zeros(n_fac, dtype=np.float32)
    # position of rule r in factor order = r + (number of ORs of earlier conclusions)
    grp = np.repeat(np.arange(n_or), counts)          # group index per (sorted) rule
    rule_pos = np.arange(n_rules) + grp
    or_pos = first + counts - 1 + np.arange(n_or) + 1  # after the group's last rule
    fan[rule_pos] = rule_k + 1
    ftype[rule_pos] = NOISY_AND
    fparam[rule_pos] = p_fire.astype(np.float32)
    fan[or_pos] = counts + 1
    ftype[or_pos] = OR
    ptr = np.zeros(n_fac + 1, dtype=np.int64)
    np.cumsum(fan, out=ptr[1:])
    fvars = np.empty(int(ptr[-1]), dtype=np.int32)
    # rule rows: premises then d_r
    kmax = rule_prem.shape[1]
    for j in range(kmax):
        sel = rule_k > j
        fvars[ptr[rule_pos[sel]] + j] = rule_prem[sel, j]
    fvars[ptr[rule_pos] + rule_k] = d_ids
    # OR rows: d_r of the group's rules, then the conclusion
    within = np.arange(n_rules) - np.repeat(first, counts)
    fvars[ptr[or_pos[grp]] + within] = d_ids
    fvars[ptr[or_pos] + counts] = concl_vals

    prior = np.full(n_vars, np.nan, dtype=np.float32)
    n_prior = int(round(prior_frac * n_tuples))
    pv = rng.choice(n_tuples, size=n_prior, replace=False)
    prior[pv] = rng.uniform(0.05, 0.95, size=n_prior).astype(np.float32)
    evidence = np.full(n_vars, -1, dtype=np.int8)
    meta = dict(meta, n_tuples=n_tuples, n_rules=n_rules, n_or=n_or)
    return FactorGraph(n_vars, ptr, fvars, ftype, fparam, prior, evidence, name, meta)


def tiny(seed: int = 1) -> FactorGraph:
    """Tiny derivation DAG: 2,000 tuples (roots 0-199), 3,000 NOISY_AND(0.9)
    rules with 2-4 distinct premises drawn uniformly below the conclusion, a
    derivation variable per rule, an OR per derived tuple, priors U(0.05,0.95)
    on 10% of tuples."""
    rng = np.random.default_rng(seed)
    n_t, n_roots, n_r = 2000, 200, 3000
    concl = rng.integers(n_roots, n_t, size=n_r)
    k = rng.integers(2, 5, size=n_r)
    prem = _distinct_rows(rng, lambda idx, col: rng.integers(0, concl[idx]), k,
                          np.full(n_r, -1), 4)
    p = np.full(n_r, 0.9)
    return _derivation_graph(rng, n_t, concl, prem, k, p, 0.10, "tiny",
                             dict(seed=seed, schedule="PARALL", iters=50))


def bingo(n_tuples: int = 1_000_000, seed: int = 3, rules_per_tuple: float = 2.0,
          alpha: float = 2.1, back_frac: float = 0.05, n_rule_types: int = 200,
          p_fire: float = 0.99, min_concl: int = 16, name: str | None = None) -> FactorGraph:
    """BINGO-shaped cyclic derivation graph: rules_per_tuple*N NOISY_AND rule
    instances with 1-3 distinct premises; premise v drawn with weight
    (v+1)^(-1/(alpha-1)) from below the conclusion, or (probability back_frac)
    from above it, which closes a cycle; rule type uniform over n_rule_types, all
    with firing probability p_fire; no evidence; priors on 10% of tuples."""
    rng = np.random.default_rng(seed)
    n_r = int(round(rules_per_tuple * n_tuples))
    lo_c = min(min_concl, max(n_tuples - 1, 0))
    concl = rng.integers(lo_c, n_tuples, size=n_r)
    k = rng.integers(1, 4, size=n_r)
    back = rng.random(n_r) < back_frac
    back &= concl + 4 <= n_tuples  # room for 3 distinct ids above c
    fwd_ok = concl >= 3
    back |= ~fwd_ok
    rule_type = rng.integers(0, n_rule_types, size=n_r)

    def draw(idx, col):
        b = back[idx]
        lo = np.where(b, concl[idx] + 1, 0)
        hi = np.where(b, n_tuples, concl[idx])
        return _powerlaw_in(rng, lo, hi, alpha)

    prem = _distinct_rows(rng, draw, k, concl, 3)
    p = np.full(n_r, p_fire)
    g = _derivation_graph(rng, n_tuples, concl, prem, k, p, 0.10,
                          name or f"bingo{n_tuples}",
                          dict(seed=seed, alpha=alpha, back_frac=back_frac,
                               n_rule_types=n_rule_types))
    g.meta["rule_type_counts_max"] = int(np.bincount(rule_type, minlength=n_rule_types).max())
    return g


def smartfl(n_layers: int = 200, width: int = 1000, extra_per_var: float = 101000 / 199000,
            evidence_frac: float = 0.05, seed: int = 2, planted: bool = False,
            name: str | None = None) -> FactorGraph:
    """SmartFL-shaped layered DAG.  Layer 0 holds the roots; every variable of
    layers 1..L-1 gets one defining factor over distinct inputs from the layer
    below (AND .3 / OR .3 / NOT .1 / EQ .1 / NOISY_IMPLY .2, fan-in
    min(Geometric(0.4), 8), NOT and EQ one input, NOISY_IMPLY p~U(0.9,0.99)).
    extra_per_var extra NOISY_IMPLY factors per non-root variable have a
    uniformly chosen non-root output and inputs from the layer below it.
    evidence_frac of the variables are observed, value Bernoulli(0.5); with
    planted=True the observed values come from one forward sample of the model
    instead, so that the evidence is consistent."""
    rng = np.random.default_rng(seed)
    n_vars = n_layers * width
    n_def = (n_layers - 1) * width
    out_def = np.arange(width, n_vars, dtype=np.int64)
    tcode = np.array([AND, OR, NOT, EQ, NOISY_IMPLY], dtype=np.uint8)
    t_def = tcode[rng.choice(5, size=n_def, p=[0.3, 0.3, 0.1, 0.1, 0.2])]
    k_def = np.minimum(rng.geometric(0.4, size=n_def), min(8, width))
    k_def[(t_def == NOT) | (t_def == EQ)] = 1
    n_extra = int(round(extra_per_var * n_def))
    out_x = rng.integers(width, n_vars, size=n_extra)
    k_x = np.minimum(rng.geometric(0.4, size=n_extra), min(8, width))
    t_x = np.full(n_extra, NOISY_IMPLY, dtype=np.uint8)
    outs = np.concatenate([out_def, out_x])
    ks = np.concatenate([k_def, k_x])
    ts = np.concatenate([t_def, t_x])
    layer_lo = (outs // width - 1) * width

    prem = _distinct_rows(rng, lambda idx, col: layer_lo[idx] + rng.integers(0, width, size=idx.size),
                          ks, np.full(outs.shape[0], -1), 8)
    n_fac = outs.shape[0]
    fan = ks + 1
    ptr = np.zeros(n_fac + 1, dtype=np.int64)
    np.cumsum(fan, out=ptr[1:])
    fvars = np.empty(int(ptr[-1]), dtype=np.int32)
    for j in range(8):
        sel = ks > j
        fvars[ptr[:-1][sel] + j] = prem[sel, j]
    fvars[ptr[1:] - 1] = outs
    fparam = np.zeros(n_fac, dtype=np.float32)
    ni = ts == NOISY_IMPLY
    fparam[ni] = rng.uniform(0.9, 0.99, size=int(ni.sum())).astype(np.float32)

    prior = np.full(n_vars, np.nan, dtype=np.float32)
    evidence = np.full(n_vars, -1, dtype=np.int8)
    n_ev = int(round(evidence_frac * n_vars))
    ev_vars = rng.choice(n_vars, size=n_ev, replace=False)
    if planted:
        x = _forward_sample(rng, n_vars, width, ptr, fvars, ts, fparam)
        evidence[ev_vars] = x[ev_vars]
    else:
        evidence[ev_vars] = rng.integers(0, 2, size=n_ev).astype(np.int8)
    return FactorGraph(n_vars, ptr, fvars, ts, fparam, prior, evidence,
                       name or f"smartfl{n_vars}",
                       dict(seed=seed, n_layers=n_layers, width=width, n_extra=n_extra,
                            planted=planted, schedule="TOPO_FB"))


def _forward_sample(rng, n_vars, width, ptr, fvars, ts, fparam) -> np.ndarray:
    """One joint sample of the layered model's defining factors (roots fair
    coins); used only to plant consistent evidence.  Extra NOISY_IMPLY factors
    are ignored, so the planted evidence can still conflict with them softly but
    never with a deterministic factor."""
    x = np.zeros(n_vars, dtype=np.int8)
    x[:width] = rng.integers(0, 2, size=width)
    n_def = n_vars - width
    for layer in range(1, n_vars // width):
        f = np.arange((layer - 1) * width, layer * width)
        for fi in f:
            row = fvars[ptr[fi]:ptr[fi + 1]]
            ins = x[row[:-1]]
            t = ts[fi]
            if t == AND:
                v = int(ins.all())
            elif t == OR:
                v = int(ins.any())
            elif t == NOT:
                v = 1 - int(ins[0])
            elif t == EQ:
                v = int(ins[0])
            else:
                v = int(rng.random() < fparam[fi]) if ins.all() else int(rng.integers(0, 2))
            x[row[-1]] = v
    assert n_def >= 0
    return x


def tree_subgraph(g: FactorGraph, n_target: int = 12, max_seeds: int = 1000) -> FactorGraph:
    """Grow a tree-shaped factor subgraph of exactly n_target variables from g:
    starting at a seed factor, accept (in id order, repeatedly) every factor that
    shares exactly one variable with the current tree while the variable count
    stays <= n_target; if growth stalls below n_target, start again from the
    next seed factor.  Priors and evidence of the kept variables are carried over
    and variables are renumbered in first-appearance order."""
    ptr, fv = g.factor_ptr, g.factor_vars
    A = g.n_factors
    rows = [fv[ptr[a]:ptr[a + 1]] for a in range(A)]
    for seed in range(min(A, max_seeds)):
        if len(set(rows[seed].tolist())) != len(rows[seed]) or len(rows[seed]) > n_target:
            continue
        vars_in = set(rows[seed].tolist())
        chosen = [seed]
        grown = True
        while grown and len(vars_in) < n_target:
            grown = False
            for a in range(A):
                if a in chosen:
                    continue
                r = rows[a].tolist()
                shared = sum(1 for v in r if v in vars_in)
                if shared == 1 and len(vars_in) + len(r) - 1 <= n_target:
                    chosen.append(a)
                    vars_in.update(r)
                    grown = True
                    if len(vars_in) == n_target:
                        break
        if len(vars_in) != n_target:
            continue
        remap: dict[int, int] = {}
        new_rows = []
        for a in chosen:
            nr = []
            for v in rows[a].tolist():
                if v not in remap:
                    remap[v] = len(remap)
                nr.append(remap[v])
            new_rows.append(np.array(nr, dtype=np.int32))
        nptr, nfv = _csr(new_rows)
        old = np.array(sorted(remap, key=remap.get), dtype=np.int64)
        return FactorGraph(n_target, nptr, nfv, g.factor_type[chosen].copy(),
                           g.factor_param[chosen].copy(), g.prior_p1[old].copy(),
                           g.evidence[old].copy(), f"{g.name}_tree{n_target}",
                           dict(source=g.name, factors=chosen))
    raise RuntimeError("no tree-shaped subgraph of the requested size")


def random_tree(n_vars: int, seed: int, max_fan: int = 4, types=(AND, OR, NOT, EQ, NOISY_IMPLY,
                                                                    NOISY_AND, PRIOR),
                evidence_frac: float = 0.1, prior_frac: float = 0.3) -> FactorGraph:
    """Random tree-shaped factor graph: every new factor joins exactly one existing
    variable and adds fresh ones, so the factor graph is a tree.  Used for
    brute-force exactness checks on up to ~20 variables."""
    rng = np.random.default_rng(seed)
    rows: list[np.ndarray] = []
    types_out, params = [], []
    nv = 1
    while nv < n_vars:
        t = int(rng.choice(types))
        if t == PRIOR:
            rows.append(np.array([int(rng.integers(0, nv))], dtype=np.int32))
            types_out.append(t)
            params.append(float(rng.uniform(0.05, 0.95)))
            continue
        if t == NOT:
            fan = 2
        else:
            fan = int(rng.integers(2, max_fan + 1))
        fan = min(fan, n_vars - nv + 1)
        if fan < 2:
            fan = 2
        join = int(rng.integers(0, nv))
        fresh = list(range(nv, nv + fan - 1))
        nv += fan - 1
        row = fresh + [join]
        rng.shuffle(row)
        rows.append(np.array(row, dtype=np.int32))
        types_out.append(t)
        params.append(float(rng.uniform(0.6, 0.99)) if t in (NOISY_IMPLY, NOISY_AND) else 0.0)
    ptr, fv = _csr(rows)
    prior = np.full(nv, np.nan, dtype=np.float32)
    m = rng.random(nv) < prior_frac
    prior[m] = rng.uniform(0.05, 0.95, size=int(m.sum())).astype(np.float32)
    ev = np.full(nv, -1, dtype=np.int8)
    m = rng.random(nv) < evidence_frac
    ev[m] = rng.integers(0, 2, size=int(m.sum())).astype(np.int8)
    return FactorGraph(nv, ptr, fv, np.array(types_out, np.uint8), np.array(params, np.float32),
                       prior, ev, f"tree{nv}_s{seed}")


def random_loopy(n_vars: int, n_factors: int, seed: int, max_fan: int = 5,
                 evidence_frac: float = 0.05, prior_frac: float = 0.2,
                 types=(AND, OR, NOT, EQ, NOISY_IMPLY, NOISY_AND, PRIOR)) -> FactorGraph:
    """Small random loopy factor graph with every factor type (parity and
    schedule tests)."""
    rng = np.random.default_rng(seed)
    rows, ts, ps = [], [], []
    for _ in range(n_factors):
        t = int(rng.choice(types))
        fan = 1 if t == PRIOR else 2 if t == NOT else int(rng.integers(2, max_fan + 1))
        fan = min(fan, n_vars)
        rows.append(rng.choice(n_vars, size=fan, replace=False).astype(np.int32))
        ts.append(t)
        ps.append(float(rng.uniform(0.6, 0.99)) if t in (NOISY_IMPLY, NOISY_AND, PRIOR) else 0.0)
    ptr, fv = _csr(rows)
    prior = np.full(n_vars, np.nan, dtype=np.float32)
    m = rng.random(n_vars) < prior_frac
    prior[m] = rng.uniform(0.05, 0.95, size=int(m.sum())).astype(np.float32)
    ev = np.full(n_vars, -1, dtype=np.int8)
    m = rng.random(n_vars) < evidence_frac
    ev[m] = rng.integers(0, 2, size=int(m.sum())).astype(np.int8)
    return FactorGraph(n_vars, ptr, fv, np.array(ts, np.uint8), np.array(ps, np.float32),
                       prior, ev, f"loopy{n_vars}x{n_factors}_s{seed}")


def hub_and_wide(n_hub: int = 3000, n_medium: int = 200, n_pool: int = 500, seed: int = 71) -> FactorGraph:
    """Rows and factors at the size boundaries of the kernels' work split: one
    hub variable in n_hub NOISY_AND(0.9) factors [hub, x, y] (its row spans
    several 1,024-entry chunks and a ragged tail), one variable in n_medium OR
    factors [medium, u, z] (a row between 9 and 256 entries), pool variables u
    of degree ~1-3, and four factors wider than a warp over pool variables: EQ
    over 40 variables, OR with 34 premises, AND with 33 premises, NOISY_IMPLY(0.95)
    with 40 premises.  x, y, z and the wide factors' outputs are fresh variables,
    so no loop runs through the hub and the premise -> output relation is
    acyclic (every factor has depth 1).  A factor whose output carries no
    information sends exactly uniform messages to its premises, which would
    leave the hub's long products untested; the outputs y, z carry priors in
    U(0.45, 0.55) instead, so every factor sends a mildly informative message
    and the hub's belief stays away from 0 and 1.  x and pool variables carry
    priors in U(0.2, 0.8); 2% of the pool is clamped."""
    rng = np.random.default_rng(seed)
    hub, medium = 0, 1
    pool = np.arange(2, 2 + n_pool, dtype=np.int32)
    nxt = 2 + n_pool
    rows, ts, ps = [], [], []
    weak, strong = [], []  # fresh variables with near-1/2 priors / with U(0.2, 0.8) priors

    def fresh(kind: list) -> int:
        nonlocal nxt
        nxt += 1
        kind.append(nxt - 1)
        return nxt - 1

    for _ in range(n_hub):
        rows.append(np.array([hub, fresh(strong), fresh(weak)], np.int32))
        ts.append(NOISY_AND)
        ps.append(0.9)
    for _ in range(n_medium):
        rows.append(np.array([medium, rng.choice(pool), fresh(weak)], np.int32))
        ts.append(OR)
        ps.append(0.0)
    for t, n_prem, p in ((EQ, 39, 0.0), (OR, 34, 0.0), (AND, 33, 0.0), (NOISY_IMPLY, 40, 0.95)):
        prem = rng.choice(pool, size=n_prem, replace=False).astype(np.int32)
        rows.append(np.concatenate([prem, np.array([fresh(weak)], np.int32)]))
        ts.append(t)
        ps.append(p)
    ptr, fv = _csr(rows)
    n_vars = nxt
    prior = np.full(n_vars, np.nan, dtype=np.float32)
    prior[pool] = rng.uniform(0.2, 0.8, size=n_pool).astype(np.float32)
    st, wk = np.array(strong, np.int64), np.array(weak, np.int64)
    prior[st] = rng.uniform(0.2, 0.8, size=st.size).astype(np.float32)
    prior[wk] = rng.uniform(0.45, 0.55, size=wk.size).astype(np.float32)
    ev = np.full(n_vars, -1, dtype=np.int8)
    clamp = rng.choice(pool, size=max(1, n_pool // 50), replace=False)
    ev[clamp] = rng.integers(0, 2, size=clamp.size).astype(np.int8)
    return FactorGraph(n_vars, ptr, fv, np.array(ts, np.uint8), np.array(ps, np.float32), prior, ev,
                       f"hub{n_hub}_wide_s{seed}")


def planted_alarms(g: FactorGraph, n_alarms: int, seed: int, fire: float = 0.6,
                   base_true: float = 0.9) -> tuple[np.ndarray, np.ndarray]:
    """Planted ground truth for an alarm-ranking run on a derivation graph
    (tiny/bingo layout: tuples 0..n_tuples-1, NOISY_AND rule rows
    [premises, d_r], OR rows [d_r..., conclusion]).  Base tuples (no OR
    factor concludes them) are true with their prior, or with probability
    base_true where they have none.  Each rule instance truly fires with
    probability `fire` (the model assumes its own, higher p).  A derived tuple
    is true iff some truly firing rule with all premises true derives it: the
    least fixed point, reached by iterating from all derived tuples false, so
    that a cycle supports nothing by itself.  Returns n_alarms distinct derived
    tuples and their truth (int8)."""
    rng = np.random.default_rng(seed)
    n_t = int(g.meta["n_tuples"])
    fp = np.asarray(g.factor_ptr, np.int64)
    fv = np.asarray(g.factor_vars, np.int64)
    ft = np.asarray(g.factor_type)
    rules = np.flatnonzero(ft == NOISY_AND)
    ors = np.flatnonzero(ft == OR)
    out_of = lambda a: fv[fp[a + 1] - 1]                      # noqa: E731  output variable of factors a
    concl = out_of(ors)
    derived = np.zeros(n_t, bool)
    derived[concl] = True
    pr = np.asarray(g.prior_p1[:n_t], np.float64)
    u = rng.random(n_t)
    base_truth = ~derived & np.where(np.isnan(pr), u < base_true, u < np.nan_to_num(pr))
    fires = rng.random(rules.size) < fire
    # premise edges of every rule, and the rule each belongs to
    r_len = fp[rules + 1] - fp[rules] - 1
    r_prem = np.concatenate([fv[fp[a]:fp[a + 1] - 1] for a in rules]) if rules.size else np.zeros(0, np.int64)
    r_of = np.repeat(np.arange(rules.size), r_len)
    d_of_rule = out_of(rules)
    # the OR factor (index into ors) that each derivation variable feeds
    or_of_d = np.full(g.n_vars, -1, np.int64)
    for k, a in enumerate(ors):
        or_of_d[fv[fp[a]:fp[a + 1] - 1]] = k
    truth = np.zeros(g.n_vars, bool)
    truth[:n_t] = base_truth
    while True:
        bad = np.zeros(rules.size, np.int64)  # premises of each rule that are false
        np.add.at(bad, r_of, ~truth[r_prem])
        d_true = fires & (bad == 0)
        c_true = np.zeros(ors.size, bool)
        c_true[or_of_d[d_of_rule[d_true]]] = True
        new = base_truth.copy()
        new[concl[c_true]] = True
        if np.array_equal(new, truth[:n_t]):
            truth[d_of_rule] = d_true
            break
        truth[:n_t] = new
    cand = np.flatnonzero(derived)
    alarms = rng.choice(cand, size=min(n_alarms, cand.size), replace=False)
    return alarms.astype(np.int64), truth[alarms].astype(np.int8)


def random_terms(rng: np.random.Generator, b: int, max_terms: int = 6, free: float = 0.3,
                 floor: float = 0.0):
    """A random term list for a factor over b variables: 1..max_terms terms,
    each variable fixed to 0 or 1 or left free (probability `free`), weights
    U(0.1, 1); with floor > 0 a last all-free term of that weight keeps every
    assignment possible.  Returns (indicators [l, b] int8, weights [l] float64)."""
    l = int(rng.integers(1, max_terms + 1))
    ind = rng.integers(0, 2, size=(l, b)).astype(np.int8)
    ind[rng.random((l, b)) < free] = -1
    w = rng.uniform(0.1, 1.0, size=l)
    if floor > 0:
        ind = np.concatenate([ind, np.full((1, b), -1, np.int8)])
        w = np.concatenate([w, [floor]])
    return ind, w


def with_generic_factors(g: FactorGraph, frac: float, seed: int, max_terms: int = 6,
                         free: float = 0.3, floor: float = 0.05) -> FactorGraph:
    """A copy of g in which a random fraction of the factors (those of at
    most 32 variables) are replaced by TERMS factors over the same variables
    with random term lists (random_terms with the given floor)."""
    rng = np.random.default_rng(seed)
    ft = np.array(g.factor_type, copy=True)
    fp = np.asarray(g.factor_ptr)
    n = np.diff(fp)
    pick = (rng.random(ft.shape[0]) < frac) & (n <= 32)
    ft[pick] = TERMS
    tp = np.zeros(ft.shape[0] + 1, np.int64)
    inds, ws = [], []
    for a in range(ft.shape[0]):
        if ft[a] == TERMS:
            ind, w = random_terms(rng, int(n[a]), max_terms, free, floor)
            inds.append(ind.reshape(-1))
            ws.append(w)
            tp[a + 1] = tp[a] + w.shape[0]
        else:
            tp[a + 1] = tp[a]
    ti = np.concatenate(inds) if inds else np.zeros(0, np.int8)
    tw = np.concatenate(ws) if ws else np.zeros(0, np.float64)
    return FactorGraph(g.n_vars, g.factor_ptr, g.factor_vars, ft, g.factor_param, g.prior_p1, g.evidence,
                       g.name + f"_generic{frac:g}", dict(g.meta), (tp, ti, tw))


def fig1_example() -> FactorGraph:
    """The five-variable, five-factor graph of the paper's Fig. 1 (Sec. 2.1),
    with factor rows a1:[v1] a2:[v2] a3:[v1,v3] a4:[v1,v2,v4] a5:[v3,v4,v5]
    (0-based ids).  a1 and a2 are unary prior factors; the others are given
    logical types so that the graph can also be run."""
    rows = [[0], [1], [0, 2], [0, 1, 3], [2, 3, 4]]
    ptr, fv = _csr([np.array(r, np.int32) for r in rows])
    ftype = np.array([PRIOR, PRIOR, NOISY_IMPLY, AND, OR], dtype=np.uint8)
    fparam = np.array([0.3, 0.6, 0.9, 0.0, 0.0], dtype=np.float32)
    return FactorGraph(5, ptr, fv, ftype, fparam, np.full(5, np.nan, np.float32),
                       np.full(5, -1, np.int8), "fig1")


def batched_mix(n_graphs: int = 512, seed: int = 4, lo: float = 1e3, hi: float = 1e5,
                scale: float = 1.0) -> list[FactorGraph]:
    """The batched workload: n_graphs graphs with size N_i log-uniform in
    [lo, hi] (times scale); even i SmartFL-shaped (N_i variables in
    max(10, N_i/1000) layers, run with TOPO_FB), odd i BINGO-shaped (N_i tuples,
    run with PARALL).  Graph i uses seed + i."""
    rng = np.random.default_rng(seed)
    sizes = np.exp(rng.uniform(np.log(lo), np.log(hi), size=n_graphs)) * scale
    out = []
    for i, n in enumerate(sizes):
        n = max(int(n), 40)
        if i % 2 == 0:
            layers = max(10, n // 1000)
            width = max(n // layers, 4)
            g = smartfl(n_layers=layers, width=width, seed=seed + i, name=f"b{i}_smartfl{layers * width}")
        else:
            g = bingo(n_tuples=n, seed=seed + i, name=f"b{i}_bingo{n}")
        out.append(g)
    return out


def serving_sessions(n_sessions: int = 64, seed: int = 5, lo: float = 5e4, hi: float = 5e5,
                     scale: float = 1.0) -> list[FactorGraph]:
    """The served workload's resident sessions: BINGO-shaped graphs with N
    log-uniform in [lo, hi] tuples (times scale); session i uses seed 1000*seed+i."""
    rng = np.random.default_rng(seed)
    sizes = np.exp(rng.uniform(np.log(lo), np.log(hi), size=n_sessions)) * scale
    return [bingo(n_tuples=max(int(n), 40), seed=1000 * seed + i, name=f"s{i}_bingo{int(n)}")
            for i, n in enumerate(sizes)]


def request_stream(sessions: list[FactorGraph], rate: float = 2000.0, duration: float = 30.0,
                   seed: int = 5) -> np.ndarray:
    """Poisson arrivals at `rate` per second for `duration` seconds.  Each request
    picks a session uniformly, then an unobserved tuple of it uniformly (a tuple
    is clamped at most once per session), then a value Bernoulli(0.5).
    Returns a structured array (t, session, var, value) in arrival order."""
    rng = np.random.default_rng(seed + 77)
    n = int(rng.poisson(rate * duration))
    t = np.sort(rng.uniform(0.0, duration, size=n))
    sess = rng.integers(0, len(sessions), size=n)
    val = rng.integers(0, 2, size=n).astype(np.int8)
    var = np.empty(n, dtype=np.int64)
    used: list[set] = [set() for _ in sessions]
    for i in range(n):
        g = sessions[sess[i]]
        nt = g.meta.get("n_tuples", g.n_vars)
        while True:
            v = int(rng.integers(0, nt))
            if v not in used[sess[i]] and g.evidence[v] < 0:
                used[sess[i]].add(v)
                break
        var[i] = v
    rec = np.zeros(n, dtype=[("t", "f8"), ("session", "i4"), ("var", "i8"), ("value", "i1")])
    rec["t"], rec["session"], rec["var"], rec["value"] = t, sess, var, val
    return rec
