"""Argument validation of fbp_graph_create runs before any device call, so
these error paths are checked on the CPU."""
import numpy as np
import pytest

from paper_2509_22337_gb300 import build as B
from paper_2509_22337_gb300 import fbp as F
from paper_2509_22337_gb300 import gen


@pytest.fixture(scope="module")
def lib():
    B.build()
    return F.load()


def _create(g, **kw):
    args = dict(n_vars=g.n_vars, n_factors=g.n_factors, factor_ptr=g.factor_ptr,
                factor_vars=g.factor_vars, factor_type=g.factor_type, factor_param=g.factor_param,
                prior_p1=g.prior_p1, evidence=g.evidence, alloc=None, stream=0)
    args.update(kw)
    return F.fbp_graph_create(**args)


@pytest.mark.parametrize("mutate,msg", [
    (lambda g: dict(factor_vars=np.where(np.arange(g.n_edges) == 3, 99, g.factor_vars)), "out of range"),
    (lambda g: dict(factor_vars=np.where(np.arange(g.n_edges) == 3, 0, g.factor_vars)), "twice"),
    (lambda g: dict(factor_type=np.array([6, 6, 4, 0, 9], np.uint8)), "unknown type"),
    (lambda g: dict(factor_type=np.array([6, 2, 4, 0, 1], np.uint8)), "arity"),
    (lambda g: dict(factor_param=np.array([1.5, 0.6, 0.9, 0, 0], np.float32)), "outside"),
    (lambda g: dict(factor_ptr=np.array([0, 1, 2, 1, 7, 10], np.int64)), "decreases"),
    (lambda g: dict(prior_p1=np.array([2, 0, 0, 0, 0], np.float32)), "prior"),
    (lambda g: dict(evidence=np.array([3, 0, 0, 0, 0], np.int8)), "evidence"),
    (lambda g: dict(n_vars=-1), "negative"),
])
def test_invalid_graph_rejected(lib, mutate, msg):
    g = gen.fig1_example()
    with pytest.raises(F.FbpError) as ei:
        _create(g, **mutate(g))
    assert ei.value.code == F.FBP_ERR_INVALID_ARG
    assert msg in str(ei.value)


def test_batch_rejects_bad_member_before_any_device_work(lib):
    from paper_2509_22337_gb300 import fbp_batch as B
    good = gen.fig1_example()
    bad = gen.FactorGraph(5, good.factor_ptr, good.factor_vars.copy(), good.factor_type, good.factor_param,
                          good.prior_p1, good.evidence)
    bad.factor_vars[2] = 9
    with pytest.raises(F.FbpError) as ei:
        B.fbp_batch_create([good, bad], ["PARALL", "PARALL"], [10, 10], [0.0, 0.0], alloc=None, stream=0)
    assert ei.value.code == F.FBP_ERR_INVALID_ARG and "batch graph 1" in str(ei.value)
    with pytest.raises(F.FbpError):
        B.fbp_batch_create([good], ["RESIDUAL"], [10], [0.0], alloc=None, stream=0)


def test_generic_factor_arity_and_batches(lib):
    """Generic (FBP_TERMS) factors: at most 32 variables; single graphs only."""
    from paper_2509_22337_gb300 import fbp_batch as B
    wide = gen.FactorGraph(40, np.array([0, 40], np.int64), np.arange(40, dtype=np.int32),
                           np.array([gen.TERMS], np.uint8), np.zeros(1, np.float32),
                           np.full(40, np.nan, np.float32), np.full(40, -1, np.int8))
    with pytest.raises(F.FbpError) as ei:
        _create(wide)
    assert ei.value.code == F.FBP_ERR_INVALID_ARG and "arity" in str(ei.value)
    g = gen.with_generic_factors(gen.random_loopy(12, 10, seed=650), 0.5, seed=651)
    with pytest.raises(F.FbpError) as ei:
        B.fbp_batch_create([g], ["PARALL"], [10], [0.0], alloc=None, stream=0)
    assert ei.value.code == F.FBP_ERR_INVALID_ARG and "generic" in str(ei.value)


def test_lowest_bad_factor_is_reported(lib):
    """Factors are checked on several host threads; the error still names the
    lowest-numbered bad factor, wherever the parts of the range fall."""
    n = 200_000
    fp = np.arange(0, 2 * n + 1, 2, dtype=np.int64)
    fv = np.arange(2 * n, dtype=np.int32) % (n + 1)
    g = gen.FactorGraph(n + 1, fp, fv, np.full(n, gen.AND, np.uint8), np.zeros(n, np.float32),
                        np.full(n + 1, np.nan, np.float32), np.full(n + 1, -1, np.int8), "pairs")
    bad = fv.copy()
    bad[2 * 150_000 + 1] = n + 7      # factor 150000: variable out of range
    bad[2 * 40_000 + 1] = bad[2 * 40_000]  # factor 40000: a variable twice
    with pytest.raises(F.FbpError) as ei:
        _create(g, factor_vars=bad)
    assert "factor 40000 lists variable" in str(ei.value)


def test_duplicate_in_a_wide_factor_names_the_first_repeat(lib):
    """A factor wider than 64 variables is checked by sorting a copy; the
    message names the first variable that repeats in row order."""
    n = 100
    row = np.arange(n, dtype=np.int32)
    row[70] = 5   # repeats variable 5 (first repeat in row order)
    row[90] = 3   # a later repeat of a smaller variable
    g = gen.FactorGraph(n, np.array([0, n], np.int64), row, np.array([gen.EQ], np.uint8),
                        np.zeros(1, np.float32), np.full(n, np.nan, np.float32), np.full(n, -1, np.int8), "wide")
    with pytest.raises(F.FbpError) as ei:
        _create(g)
    assert "lists variable 5 twice" in str(ei.value)
