"""Pins of the FP64 oracle to things other than itself (CPU only).

Each test names the passage of the paper or the mathematical fact it rests on.
A plausible slip anywhere in the oracle (a dropped term, a wrong index or sign,
a transposed operand, a wrong cut rule) fails at least one of them.
"""
import itertools
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2509_22337_gb300 import gen
from tests import bp_reference_defs as R

TYPES_ARITY = [
    (gen.AND, range(2, 10)), (gen.OR, range(2, 10)), (gen.NOT, [2]), (gen.EQ, range(1, 9)),
    (gen.NOISY_IMPLY, range(2, 10)), (gen.NOISY_AND, range(2, 10)), (gen.PRIOR, [1]),
]


# ---------------------------------------------------------------------------
# Eq. (2) vs Eq. (4) / Algorithm 1: the term lists and the literal Algorithm 1
# reproduce the dense factor-table message for every type and fan-in.
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("ftype,arities", TYPES_ARITY)
def test_alg1_term_lists_equal_dense_eq2(ftype, arities):
    rng = np.random.default_rng(100 + ftype)
    for b in arities:
        for trial in range(3):
            p = float(rng.uniform(0.05, 0.99))
            mu = rng.uniform(0.0, 2.0, size=(b, 2))
            if trial == 2:  # hard inputs too
                mu[rng.random(b) < 0.3] = [0.0, 1.0]
            tab = R.factor_table(ftype, p, b)
            ind, w = O.terms(ftype, b, p)
            for v in range(b):
                want = R.dense_message(tab, mu, v)
                got = np.array([O.alg1(ind, w, mu, v, 0), O.alg1(ind, w, mu, v, 1)])
                np.testing.assert_allclose(got, want, rtol=1e-13, atol=1e-300)


def test_term_counts_match_sec_2_2():
    # Sec. 2.2: BINGO's rule constraint over three premises has five
    # sub-messages per entry (ten per message).
    ind, w = O.terms(gen.NOISY_AND, 4, 0.9)
    assert ind.shape[1] == 5 and w.shape[0] == 5


def test_special_cases_reduce():
    rng = np.random.default_rng(7)
    for b in range(2, 7):
        mu = rng.uniform(0.1, 1.0, size=(b, 2))
        i1, w1 = O.terms(gen.NOISY_AND, b, 1.0)
        i2, w2 = O.terms(gen.AND, b, 0.0)
        for v in range(b):
            for x in (0, 1):
                assert O.alg1(i1, w1, mu, v, x) == pytest.approx(O.alg1(i2, w2, mu, v, x), rel=1e-14)
    # AND and OR with one premise are equality factors
    mu = rng.uniform(0.1, 1.0, size=(2, 2))
    ie, we = O.terms(gen.EQ, 2, 0.0)
    for t in (gen.AND, gen.OR):
        it, wt = O.terms(t, 2, 0.0)
        for v in range(2):
            for x in (0, 1):
                assert O.alg1(it, wt, mu, v, x) == pytest.approx(O.alg1(ie, we, mu, v, x), rel=1e-14)


def test_invalid_arities_rejected():
    with pytest.raises(ValueError):
        O.terms(gen.NOT, 3, 0.0)
    with pytest.raises(ValueError):
        O.terms(gen.PRIOR, 2, 0.5)
    with pytest.raises(ValueError):
        O.terms(gen.AND, 1, 0.0)
    with pytest.raises(ValueError):
        O.terms(99, 3, 0.0)


# ---------------------------------------------------------------------------
# Algorithm 2: the worked example of Sec. 2.1, the PARALL special case, the
# literal scan against the neighbourhood scan, and Theorems 1 and 2.
# ---------------------------------------------------------------------------
def _golden_groups():
    path = os.path.join(os.path.dirname(__file__), "golden", "fig1_seqfix_levels.txt")
    groups = []
    for line in open(path):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        pairs = []
        for tok in line.split():
            a, v = tok.strip("()").split(",")
            pairs.append((int(a[1:]) - 1, int(v[1:]) - 1))
        groups.append(pairs)
    return groups


@pytest.mark.parametrize("literal", [True, False])
def test_alg2_worked_example_sec_2_1(literal):
    g = gen.fig1_example()
    o = O.Oracle(g)
    lp, le = o.levels(o.ranks("SEQFIX"), literal=literal)
    got = [[(int(np.searchsorted(g.factor_ptr, e, side="right") - 1), int(g.factor_vars[e]))
            for e in le[lp[i]:lp[i + 1]]] for i in range(len(lp) - 1)]
    assert got == _golden_groups()


def test_ne_definition_1_on_example():
    # Sec. 2.1: mu_{a4->v1} depends on mu_{a2->v2} (through v2) and on
    # mu_{a5->v4} (through v4); mu_{a2->v2} and mu_{a1->v1} are independent.
    g = gen.fig1_example()
    o = O.Oracle(g)
    e = {(0, 0): 0, (1, 1): 1, (2, 0): 2, (2, 2): 3, (3, 0): 4, (3, 1): 5, (3, 3): 6, (4, 2): 7,
         (4, 3): 8, (4, 4): 9}
    assert o.in_ne(e[(1, 1)], e[(3, 0)])
    assert o.in_ne(e[(4, 3)], e[(3, 0)])
    assert not o.in_ne(e[(0, 0)], e[(1, 1)]) and not o.in_ne(e[(1, 1)], e[(0, 0)])
    assert not o.in_ne(e[(3, 1)], e[(3, 0)])      # same factor: a* != a
    assert o.in_ne(e[(0, 0)], e[(2, 2)])          # (a3,v3) cuts on (a1,v1)
    assert o.in_ne(e[(3, 3)], e[(4, 2)])          # (a5,v3) cuts on (a4,v4)


def test_parall_single_level():
    # Sec. 4.2.2: PARALL puts every edge in one equivalence class, so
    # Algorithm 2 never cuts.
    g = gen.random_loopy(30, 40, seed=3)
    o = O.Oracle(g)
    for literal in (True, False):
        lp, le = o.levels(o.ranks("PARALL"), literal=literal)
        assert lp.tolist() == [0, g.n_edges]
        assert le.tolist() == list(range(g.n_edges))


def _rand_graphs():
    out = [gen.random_loopy(n, m, seed=s) for s, (n, m) in enumerate([(20, 25), (40, 60), (60, 50)])]
    out.append(gen.smartfl(n_layers=8, width=12, seed=11))
    out.append(gen.tiny())
    return out


def _rank_sets(o, g, rng):
    yield "PARALL", o.ranks("PARALL")
    yield "SEQFIX", o.ranks("SEQFIX")
    yield "CUSTOM-perm", rng.permutation(g.n_edges).astype(np.int64)
    yield "CUSTOM-few", rng.integers(0, 4, size=g.n_edges).astype(np.int64)
    try:
        yield "TOPO", o.ranks("TOPO")
        yield "TOPO-back", o.ranks("TOPO", backward=True)
    except ValueError:
        pass


def test_alg2_literal_equals_neighbourhood_scan():
    rng = np.random.default_rng(5)
    for g in _rand_graphs():
        o = O.Oracle(g)
        for name, r in _rank_sets(o, g, rng):
            if g.n_edges > 5000 and name in ("SEQFIX", "CUSTOM-perm"):
                continue  # literal scan is quadratic in the level size
            a = o.levels(r, literal=True)
            b = o.levels(r, literal=False)
            assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1]), (g.name, name)


def _ne_sets(g):
    A = g.n_factors
    fac = np.repeat(np.arange(A), np.diff(g.factor_ptr))
    var = g.factor_vars
    by_var = {}
    for e in range(g.n_edges):
        by_var.setdefault(int(var[e]), []).append(e)
    ne = []
    for e in range(g.n_edges):
        a, v = fac[e], var[e]
        s = set()
        for q in range(int(g.factor_ptr[a]), int(g.factor_ptr[a + 1])):
            vs = int(var[q])
            if vs == v:
                continue
            for f in by_var[vs]:
                if fac[f] != a:
                    s.add(f)
        ne.append(s)
    return ne


def test_theorem_1_and_2_properties():
    rng = np.random.default_rng(9)
    for g in _rand_graphs()[:4]:
        o = O.Oracle(g)
        ne = _ne_sets(g)
        for name, r in _rank_sets(o, g, rng):
            lp, le = o.levels(r)
            lvl = np.empty(g.n_edges, dtype=np.int64)
            for i in range(len(lp) - 1):
                lvl[le[lp[i]:lp[i + 1]]] = i
            # every edge exactly once; canonical (rank, id) order inside the output
            assert sorted(le.tolist()) == list(range(g.n_edges))
            keys = list(zip(r[le].tolist(), le.tolist()))
            assert keys == sorted(keys)
            # classes split across levels (the gap in Theorem 2(2))
            split = {int(c) for c in np.unique(r) if len(np.unique(lvl[r == c])) > 1}
            for e in range(g.n_edges):
                for f in ne[e]:
                    # Theorem 1: delta(e, f) = 1 only towards a strictly earlier class
                    if r[f] < r[e]:
                        assert lvl[f] < lvl[e], (name, e, f)          # Theorem 2(1)
                    if r[e] < r[f]:
                        assert lvl[f] >= lvl[e], (name, e, f)         # Theorem 2(2), strict part
                    if r[e] == r[f] and int(r[e]) not in split:
                        assert lvl[f] == lvl[e]
            if name == "PARALL":
                assert len(lp) == 2


# ---------------------------------------------------------------------------
# Eq. (1)-(3) end to end: exact on trees (Sec. 3.2), equal to textbook
# synchronous / round-robin BP on dense tables on loopy graphs.
# ---------------------------------------------------------------------------
def _tree_cases():
    cases = [gen.tree_subgraph(gen.tiny(), 12)]
    for s in range(12):
        cases.append(gen.random_tree(int(8 + s % 9), seed=s))
    return cases


@pytest.mark.parametrize("strategy", ["PARALL", "SEQFIX", "TOPO", "TOPO_FB", "RESIDUAL"])
def test_bp_exact_on_trees(strategy):
    checked = 0
    for g in _tree_cases():
        exact, Z = R.brute_force_marginals(g)
        if not Z > 0:
            continue
        o = O.Oracle(g)
        try:
            res = o.run(strategy, max_iters=200, tol=1e-15 if strategy != "RESIDUAL" else 1e-13)
        except ValueError:
            continue  # TOPO on a graph whose output convention has a cycle
        p = o.marginals(res["a2v"])
        np.testing.assert_allclose(p, exact, atol=1e-12, err_msg=f"{g.name} {strategy}")
        checked += 1
    assert checked >= 6


def test_tiny_tree_subgraph_is_a_tree_of_12():
    t = gen.tree_subgraph(gen.tiny(), 12)
    assert t.n_vars == 12
    # a factor graph is a tree iff it is connected and |E| = |V| + |A| - 1
    assert t.n_edges == t.n_vars + t.n_factors - 1


def test_parall_equals_textbook_synchronous_bp():
    for s in range(4):
        g = gen.random_loopy(12, 14, seed=20 + s)
        o = O.Oracle(g)
        for iters in (1, 2, 7):
            res = o.run("PARALL", max_iters=iters, tol=0.0)
            want = R.msgs_to_edges(g, R.sync_bp(g, iters))
            np.testing.assert_allclose(res["a2v"], want, atol=1e-13)
            np.testing.assert_allclose(o.marginals(res["a2v"]),
                                       R.marginals_from(g, R.sync_bp(g, iters)), atol=1e-13)


@pytest.mark.parametrize("def2", [True, False])
def test_seqfix_equals_round_robin_sequential_bp(def2):
    # Sec. 2.1: the round-robin asynchronous schedule; Definition 2 with a
    # total order is exactly sequential BP, and the levels of Algorithm 2
    # (Theorem 2) reproduce it.
    rng = np.random.default_rng(4)
    for s in range(4):
        g = gen.random_loopy(10, 12, seed=40 + s)
        fac = np.repeat(np.arange(g.n_factors), np.diff(g.factor_ptr))
        perm = rng.permutation(g.n_edges)
        order = [(int(fac[e]), int(g.factor_vars[e])) for e in perm]
        rank = np.empty(g.n_edges, dtype=np.int64)
        rank[perm] = np.arange(g.n_edges)
        o = O.Oracle(g)
        for iters in (1, 3):
            res = o.run("CUSTOM", max_iters=iters, tol=0.0, custom=rank, def2=def2)
            want = R.msgs_to_edges(g, R.seq_bp(g, iters, order))
            np.testing.assert_allclose(res["a2v"], want, atol=1e-13)


def test_level_mode_equals_definition_2_without_split_classes():
    rng = np.random.default_rng(12)
    for s in range(5):
        g = gen.random_loopy(25, 30, seed=60 + s)
        o = O.Oracle(g)
        for name, r in [("PARALL", o.ranks("PARALL")), ("SEQFIX", o.ranks("SEQFIX")),
                        ("few", rng.integers(0, 3, size=g.n_edges).astype(np.int64))]:
            lp, le = o.levels(r)
            lvl = np.empty(g.n_edges, dtype=np.int64)
            for i in range(len(lp) - 1):
                lvl[le[lp[i]:lp[i + 1]]] = i
            split = any(len(np.unique(lvl[r == c])) > 1 for c in np.unique(r))
            if split:
                continue
            a = o.run("CUSTOM", 6, 0.0, custom=r, def2=True)
            b = o.run("CUSTOM", 6, 0.0, custom=r, def2=False)
            np.testing.assert_allclose(a["a2v"], b["a2v"], atol=1e-12)


# ---------------------------------------------------------------------------
# Eq. (1): prefix/suffix exclusion products equal the literal product.
# ---------------------------------------------------------------------------
def test_v2a_prefix_suffix_equals_literal_product():
    rng = np.random.default_rng(3)
    d = 300
    rows = [np.array([i, d], np.int32) for i in range(d)]  # hub variable d in d factors
    ptr = np.zeros(d + 1, np.int64)
    ptr[1:] = np.cumsum([2] * d)
    g = gen.FactorGraph(d + 1, ptr, np.concatenate(rows), np.full(d, gen.AND, np.uint8),
                        np.zeros(d, np.float32), np.full(d + 1, np.nan, np.float32),
                        np.full(d + 1, -1, np.int8), "star")
    o = O.Oracle(g)
    a2v = rng.uniform(0.01, 1.0, size=(g.n_edges, 2))
    a2v /= a2v.sum(1, keepdims=True)
    lit = o.v2a_row(a2v, d, literal=True)
    fast = o.v2a_row(a2v, d, literal=False)
    hub_edges = np.arange(1, g.n_edges, 2)
    np.testing.assert_allclose(fast[hub_edges], lit[hub_edges], rtol=1e-12)
    # with a hard zero in the row the exclusion is still exact
    a2v[3] = [1.0, 0.0]
    lit = o.v2a_row(a2v, d, literal=True)
    fast = o.v2a_row(a2v, d, literal=False)
    np.testing.assert_allclose(fast[hub_edges], lit[hub_edges], rtol=1e-12, atol=1e-300)


# ---------------------------------------------------------------------------
# Invariants and strategies
# ---------------------------------------------------------------------------
def test_message_invariants_and_clamps():
    g = gen.smartfl(n_layers=10, width=30, seed=5)
    o = O.Oracle(g)
    res = o.run("TOPO_FB", 30, 1e-9)
    m = res["a2v"]
    assert (m >= 0).all()
    np.testing.assert_allclose(m.sum(1), 1.0, atol=1e-14)
    p = o.marginals(m)
    ev = g.evidence >= 0
    # a clamped variable has marginal exactly 0 or 1 unless the guard fired
    ok = (p[ev] == g.evidence[ev]) | (p[ev] == 0.5)
    assert ok.all()


def test_topo_rank_is_layer_depth():
    g = gen.smartfl(n_layers=12, width=20, seed=8)
    o = O.Oracle(g)
    r = o.ranks("TOPO")
    fac_out = g.factor_vars[g.factor_ptr[1:] - 1]
    layer = fac_out // 20
    want = np.repeat(layer, np.diff(g.factor_ptr))
    assert np.array_equal(r, want)
    rb = o.ranks("TOPO", backward=True)
    assert np.array_equal(rb, want.max() - want)


def test_topo_rejects_cycles():
    g = gen.bingo(n_tuples=400, seed=9, back_frac=0.2)
    o = O.Oracle(g)
    with pytest.raises(ValueError):
        o.ranks("TOPO")


def _chain(n, seed):
    """x0 -> x1 -> ... -> x{n-1}: factor i has premise x{i-1} and output x{i};
    every variable has a prior, the last one is observed."""
    rng = np.random.default_rng(seed)
    types = rng.choice([gen.NOT, gen.EQ, gen.AND, gen.OR, gen.NOISY_IMPLY, gen.NOISY_AND], n - 1)
    fv = np.array([[i - 1, i] for i in range(1, n)], np.int32).reshape(-1)
    prior = rng.uniform(0.1, 0.9, n).astype(np.float32)
    ev = np.full(n, -1, np.int8)
    ev[-1] = 1
    param = np.where((types == gen.NOISY_IMPLY) | (types == gen.NOISY_AND), rng.uniform(0.6, 0.95, n - 1), 0)
    return gen.FactorGraph(n, np.arange(0, 2 * n - 1, 2, dtype=np.int64), fv, types.astype(np.uint8),
                           param.astype(np.float32), prior, ev, f"chain{n}")


def test_topo_fb_chain_exact_after_one_sweep():
    """Reading 8 (Table 1's topological order, swept forward then backward):
    on a chain the forward half carries every message towards the outputs
    exactly and the backward half every message towards the premises, so one
    TOPO_FB iteration gives the exact marginals (Sec. 3.2: BP is exact on
    trees).  Two forward halves (or two backward halves) do not."""
    for seed in range(6):
        g = _chain(9, seed)
        exact, Z = R.brute_force_marginals(g)
        assert Z > 0
        o = O.Oracle(g)
        r = o.run("TOPO_FB", 1, 0.0)
        np.testing.assert_allclose(o.marginals(r["a2v"]), exact, atol=1e-12, err_msg=g.name)
        assert r["updates"] == 2 * g.n_edges  # one sweep = both halves, E writes each
        twice_forward = o.marginals(o.run("TOPO", 2, 0.0)["a2v"])
        assert np.abs(twice_forward - exact).max() > 1e-6


def test_topo_fb_iteration_is_forward_levels_then_backward_levels():
    """Reading 8: one TOPO_FB iteration is the TOPO level list (ranks = output
    depth, pinned by test_topo_rank_is_layer_depth) followed by the level list
    of the reversed ranks (max - rank), the second from the messages the first
    left; the iteration's residual (reading 6) is the largest change of either
    half's writes.  The reversed ranks are run as a custom preorder (Table 1)."""
    first_bigger = second_bigger = 0
    for seed in range(4):
        g = gen.smartfl(n_layers=8, width=12, seed=90 + seed, planted=True)
        o = O.Oracle(g)
        fwd = o.ranks("TOPO")
        bwd = fwd.max() - fwd
        m0 = None
        for k in range(4):  # start states: uniform, then after k PARALL iterations
            if k:
                m0 = o.run("PARALL", k, 0.0)["a2v"]
            r = o.run("TOPO_FB", 1, 0.0, a2v=m0)
            rf = o.run("TOPO", 1, 0.0, a2v=m0)
            rb = o.run("CUSTOM", 1, 0.0, custom=bwd, a2v=rf["a2v"])
            assert np.array_equal(r["a2v"], rb["a2v"]), (seed, k)
            assert r["residual"] == max(rf["residual"], rb["residual"]), (seed, k)
            first_bigger += rf["residual"] > rb["residual"]
            second_bigger += rb["residual"] > rf["residual"]
    # both halves set the residual somewhere, so a residual of one half only fails
    assert first_bigger and second_bigger


def test_topo_fb_stops_on_the_pair_residual():
    """The stopping test (reading 6) applies once per forward + backward pair:
    the iteration count is the first pair whose residual is below tol, and the
    recorded history is one residual per pair."""
    g = gen.smartfl(n_layers=8, width=12, seed=95, planted=True)
    o = O.Oracle(g)
    full = o.run("TOPO_FB", 40, 0.0, history=True)
    h = full["res_hist"]
    assert h.shape[0] == 40 and h[-1] < h[0]
    tol = float(h[5]) * 1.000001  # pair 6 is the first below tol only if h[0..4] are above it
    want = next(i for i in range(40) if h[i] < tol) + 1
    r = o.run("TOPO_FB", 40, tol)
    assert r["converged"] and r["iters"] == want
    assert r["updates"] == 2 * g.n_edges * want


def test_residual_classes_by_hand():
    """Reading 9, the residual strategy's classes, on a hand-made graph whose
    previous-iteration changes are set by hand: rho_a is the largest change
    written into ANY of a's variables (by any factor), bucketed >= 1e-2 (0),
    [1e-4, 1e-2) (1), [tol, 1e-4) (2), below tol skipped."""
    tol = 1e-6
    rows = [[0, 1], [2, 3], [4, 5], [6, 7], [8, 9], [10, 11], [1, 16], [12, 13], [13, 14], [14, 15]]
    ptr = np.concatenate([[0], np.cumsum([len(r) for r in rows])]).astype(np.int64)
    fv = np.array([v for r in rows for v in r], np.int32)
    n_a = len(rows)
    g = gen.FactorGraph(17, ptr, fv, np.full(n_a, gen.EQ, np.uint8), np.zeros(n_a, np.float32),
                        np.full(17, np.nan, np.float32), np.full(17, -1, np.int8), "hand")
    dres = np.zeros(g.n_edges + 1)

    def edge(a, v):
        return int(ptr[a] + rows[a].index(v))
    dres[edge(0, 0)] = 0.5      # a0: 0.5 -> class 0
    dres[edge(0, 1)] = 2e-3     # into v1: a6 sees it through v1 only
    dres[edge(1, 3)] = 1e-2     # a1: exactly 1e-2 -> class 0
    dres[edge(2, 4)] = 5e-3     # a2: class 1
    dres[edge(3, 7)] = 1e-4     # a3: exactly 1e-4 -> class 1
    dres[edge(4, 8)] = 5e-5     # a4: class 2
    dres[edge(5, 10)] = 1e-6    # a5: exactly tol -> class 2
    dres[edge(7, 12)] = 9.9e-7  # a7: below tol -> skipped
    dres[edge(8, 14)] = 3e-5    # a8: class 2 from its own write into v14 ...
    dres[edge(9, 15)] = 0.2     # a9: ... while a9 (also at v14) is class 0 from v15
    # a6 ([1, 16]) writes nothing itself: class 1 from a0's write into v1
    want_cls = [0, 0, 1, 1, 2, 2, 1, -1, 2, 0]
    o = O.Oracle(g)
    rank, active = o.residual_classes(dres, tol)
    assert rank.tolist() == [c for a, c in enumerate(want_cls) for _ in rows[a]]
    assert active.tolist() == [e for a, c in enumerate(want_cls) if c >= 0 for e in range(ptr[a], ptr[a + 1])]


def test_residual_reaches_parall_fixed_point():
    g = gen.tiny()
    o = O.Oracle(g)
    a = o.run("PARALL", 500, 1e-10)
    b = o.run("RESIDUAL", 500, 1e-10)
    assert a["converged"] and b["converged"]
    np.testing.assert_allclose(o.marginals(a["a2v"]), o.marginals(b["a2v"]), atol=1e-8)
    assert b["updates"] < a["updates"]


def test_zero_mass_guard_fires_on_contradiction():
    # y = AND(x1, x2) with y observed true and x1 observed false
    ptr = np.array([0, 3], np.int64)
    g = gen.FactorGraph(3, ptr, np.array([0, 1, 2], np.int32), np.array([gen.AND], np.uint8),
                        np.zeros(1, np.float32), np.full(3, np.nan, np.float32),
                        np.array([0, -1, 1], np.int8), "contra")
    o = O.Oracle(g)
    res = o.run("PARALL", 3, 0.0)
    assert res["guards"] > 0
    # to x2 both entries vanish: mu(1) needs x1 = 1, mu(0) needs y = 0
    np.testing.assert_allclose(res["a2v"][1], [0.5, 0.5])
    # to y: (D, Pi1) = (1, 0); to x1: (m_y0 * Pi_s, m_y1 * Pi1 + m_y0 * D) -> (0, 1)
    np.testing.assert_allclose(res["a2v"][2], [1.0, 0.0])
    np.testing.assert_allclose(res["a2v"][0], [0.0, 1.0])
    # y: phi (0,1) times (1,0) has zero mass -> guarded marginal
    assert o.marginals(res["a2v"])[2] == 0.5


def test_invalid_graphs_rejected():
    base = gen.fig1_example()
    bad = gen.FactorGraph(5, base.factor_ptr, base.factor_vars.copy(), base.factor_type,
                          base.factor_param, base.prior_p1, base.evidence)
    bad.factor_vars[3] = 0  # a4 lists v1 twice... (a3 row [v1, v1])
    with pytest.raises(ValueError):
        O.Oracle(bad)
    bad2 = gen.FactorGraph(5, base.factor_ptr, base.factor_vars.copy(), base.factor_type,
                           base.factor_param, base.prior_p1, base.evidence)
    bad2.factor_vars[0] = 7
    with pytest.raises(ValueError):
        O.Oracle(bad2)


# ---------------------------------------------------------------------------
# Generic factors: local structure given explicitly as a term list (the
# indicator array of Sec. 4.3.2), evaluated by Algorithm 1.
# ---------------------------------------------------------------------------
def test_generic_terms_algorithm1_equals_dense_table():
    """Random term lists with free variables: Algorithm 1 on the list equals
    Eq. (2) on the dense table the list defines."""
    rng = np.random.default_rng(60)
    for _ in range(40):
        b = int(rng.integers(1, 7))
        ind, w = gen.random_terms(rng, b, max_terms=7, free=0.35)
        tab = R.terms_table(ind, w)
        mu = rng.uniform(0.0, 1.0, size=(b, 2))
        oind = np.where(ind.T < 0, -1, ind.T).astype(np.int8)  # oracle layout [b, l]
        for v in range(b):
            got = np.array([O.alg1(oind, w, mu, v, 0), O.alg1(oind, w, mu, v, 1)])
            np.testing.assert_allclose(got, R.dense_message(tab, mu, v), rtol=1e-13, atol=1e-15)


def test_generic_factor_with_a_types_terms_equals_the_type():
    """A TERMS factor carrying a typed factor's own term list gives the same
    BP messages as the typed factor."""
    for s in range(3):
        g = gen.random_tree(12, seed=610 + s)
        fp = np.asarray(g.factor_ptr)
        tp = [0]
        inds, ws = [], []
        for a in range(g.n_factors):
            b = int(fp[a + 1] - fp[a])
            ind, w = O.terms(int(g.factor_type[a]), b, float(g.factor_param[a]))
            inds.append(ind.T.reshape(-1))  # [l, b], term after term
            ws.append(w)
            tp.append(tp[-1] + w.shape[0])
        h = gen.FactorGraph(g.n_vars, g.factor_ptr, g.factor_vars, np.full(g.n_factors, gen.TERMS, np.uint8),
                            g.factor_param, g.prior_p1, g.evidence, g.name + "_asterms", {},
                            (np.array(tp, np.int64), np.concatenate(inds).astype(np.int8), np.concatenate(ws)))
        a = O.Oracle(g).run("PARALL", 20, 0.0)
        b_ = O.Oracle(h).run("PARALL", 20, 0.0)
        np.testing.assert_array_equal(a["a2v"], b_["a2v"])


def test_generic_bp_exact_on_trees():
    """On trees with generic factors (random term lists), BP marginals equal
    brute-force exact marginals."""
    checked = 0
    for s in range(8):
        g = gen.with_generic_factors(gen.random_tree(int(8 + s % 7), seed=620 + s), 0.6, seed=630 + s)
        exact, Z = R.brute_force_marginals(g)
        if not Z > 0:
            continue
        o = O.Oracle(g)
        res = o.run("PARALL", max_iters=200, tol=1e-15)
        np.testing.assert_allclose(o.marginals(res["a2v"]), exact, atol=1e-12, err_msg=g.name)
        checked += 1
    assert checked >= 6


def test_generic_terms_rejected_when_malformed():
    g = gen.with_generic_factors(gen.random_loopy(10, 8, seed=640), 1.0, seed=641)
    tp, ti, tw = g.terms
    bad = [(tp, np.where(ti == 0, 2, ti).astype(np.int8), tw), (tp, ti, -tw)]
    for terms in bad:
        h = gen.FactorGraph(g.n_vars, g.factor_ptr, g.factor_vars, g.factor_type, g.factor_param,
                            g.prior_p1, g.evidence, "bad", {}, terms)
        with pytest.raises(ValueError):
            O.Oracle(h)


def test_oracle_threads_give_the_same_results():
    """The oracle's multi-threaded mode (each level's independent updates on
    several host threads, used to time it on every core) computes exactly the
    one-thread run: messages, residual history, guards and range diagnostic."""
    cases = [(gen.tiny(), "PARALL"), (gen.smartfl(n_layers=12, width=40, seed=5), "TOPO_FB"),
             (gen.bingo(n_tuples=3000, seed=8), "PARALL"), (gen.bingo(n_tuples=2000, seed=9), "RESIDUAL")]
    for g, strategy in cases:
        o = O.Oracle(g)
        a = o.run(strategy, 8, 0.0, history=True)
        b = o.run(strategy, 8, 0.0, history=True, threads=4)
        assert np.array_equal(a["a2v"], b["a2v"]), (g.name, strategy)
        assert np.array_equal(a["res_hist"], b["res_hist"]) and a["guards"] == b["guards"]
        assert a["min_pos"] == b["min_pos"] and a["updates"] == b["updates"]
