"""The alarm-ranking loop's host side (Sec. 5.3): the quality measures against
their definitions counted by brute force, and the planted ground truth against
properties that fix it (no GPU)."""
import itertools

import numpy as np
import pytest

from paper_2509_22337_gb300 import gen, ranking


def _inversions_brute(lab):
    # every pair (i, j), i before j, with a false alarm at i and a true one at j
    return sum(1 for i, j in itertools.combinations(range(len(lab)), 2) if lab[i] == 0 and lab[j] == 1)


def test_inversions_match_pair_count():
    rng = np.random.default_rng(3)
    for n in (0, 1, 2, 7, 40):
        for _ in range(20):
            lab = rng.integers(0, 2, size=n)
            assert ranking.inversions(lab) == _inversions_brute(lab)
    assert ranking.inversions([1, 1, 0, 0]) == 0          # true alarms first: no inversion
    assert ranking.inversions([0, 0, 1, 1]) == 4          # every false before every true


def test_rank_t():
    lab = [1, 0, 1, 1, 0]
    assert ranking.rank_t(lab, 1.0) == 4                  # the third true alarm is the 4th inspected
    assert ranking.rank_t(lab, 0.9) == 4                  # ceil(0.9 * 3) = 3
    lab10 = [1] * 9 + [0] * 5 + [1]                       # 10 true alarms
    assert ranking.rank_t(lab10, 0.9) == 9                # ceil(0.9 * 10) = 9: not 10 by rounding
    assert ranking.rank_t(lab10, 1.0) == 15
    assert ranking.rank_t([0, 0, 0], 1.0) == 0


def test_next_alarm_breaks_ties_by_list_order():
    p = np.array([0.2, 0.9, 0.9, 0.5])
    alarms = np.array([3, 2, 1])
    assert ranking.next_alarm(p, alarms, np.zeros(3, bool)) == 1          # alarm 2 before alarm 1
    assert ranking.next_alarm(p, alarms, np.array([False, True, False])) == 2


def _graph(rows, types, params, n_tuples, prior=None):
    ptr = np.zeros(len(rows) + 1, np.int64)
    ptr[1:] = np.cumsum([len(r) for r in rows])
    n_vars = int(max(max(r) for r in rows)) + 1
    pr = np.full(n_vars, np.nan, np.float32) if prior is None else prior
    return gen.FactorGraph(n_vars, ptr, np.concatenate(rows).astype(np.int32), np.array(types, np.uint8),
                           np.array(params, np.float32), pr, np.full(n_vars, -1, np.int8), "hand",
                           dict(n_tuples=n_tuples))


def test_planted_truth_is_the_least_fixed_point():
    # tuples 0, 1 base; rules: r0: 0 -> d3 -> OR -> 2; a cycle 4 <-> 5 with no base support:
    # r1: 5 -> d6 -> OR -> 4, r2: 4 -> d7 -> OR -> 5
    rows = [[0, 8], [8, 2], [5, 9], [9, 4], [4, 10], [10, 5]]
    types = [gen.NOISY_AND, gen.OR] * 3
    g = _graph(rows, types, [0.99, 0, 0.99, 0, 0.99, 0], n_tuples=8)
    alarms, lab = gen.planted_alarms(g, 3, seed=1, fire=1.0, base_true=1.0)
    truth = dict(zip(alarms.tolist(), lab.tolist()))
    assert sorted(truth) == [2, 4, 5]                     # the derived tuples
    assert truth[2] == 1                                  # derived from a true base fact
    assert truth[4] == 0 and truth[5] == 0                # a cycle does not support itself
    _, lab0 = gen.planted_alarms(g, 3, seed=1, fire=0.0, base_true=1.0)
    assert (lab0 == 0).all()                              # no rule fires: nothing derived


def test_planted_alarms_are_distinct_derived_and_seeded():
    g = gen.bingo(n_tuples=600, seed=41, back_frac=0.05)
    a1, l1 = gen.planted_alarms(g, 40, seed=42)
    a2, l2 = gen.planted_alarms(g, 40, seed=42)
    assert np.array_equal(a1, a2) and np.array_equal(l1, l2)
    assert len(set(a1.tolist())) == 40 and (a1 < g.meta["n_tuples"]).all()
    ors = np.flatnonzero(g.factor_type == gen.OR)
    concl = set(g.factor_vars[g.factor_ptr[ors + 1] - 1].tolist())
    assert set(a1.tolist()) <= concl
    assert 0 < l1.mean() < 1                              # both kinds of alarm
