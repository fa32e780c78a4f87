"""CPU-side checks of the CUDA library: it loads, exports every entry point
its headers declare, and its host-side dependency analysis (Algorithm 2)
matches the oracle's bit for bit.  No device computation runs here."""
import glob
import os
import re

import numpy as np
import pytest

from oracle import oracle as O
from paper_2509_22337_gb300 import build as B
from paper_2509_22337_gb300 import fbp as F
from paper_2509_22337_gb300 import gen

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return F.load()


def declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"\b(fbp_\w+)\s*\(", src):
            names.add(m.group(1))
    return sorted(names)


def test_library_exports_every_declared_symbol(lib):
    names = declared_symbols()
    assert len(names) >= 12
    for n in names:
        assert hasattr(lib, n), n


def test_missing_library_fails_loudly(tmp_path):
    with pytest.raises(RuntimeError):
        F.load.__wrapped__(str(tmp_path / "nope.so")) if hasattr(F.load, "__wrapped__") else \
            _load_missing(str(tmp_path / "nope.so"))


def _load_missing(path):
    saved = F._lib
    F._lib = None
    try:
        F.load(path)
    finally:
        F._lib = saved


def _graphs():
    yield gen.fig1_example()
    for s in range(3):
        yield gen.random_loopy(40, 50, seed=200 + s)
    yield gen.tiny()
    yield gen.smartfl(n_layers=20, width=50, seed=12)
    yield gen.smartfl(n_layers=200, width=1000, seed=2)


def _custom_ranks(kind, rng, n):
    """CUSTOM: seven classes (the library places them by counting sort);
    CUSTOM_WIDE: seven classes spread over +-3 * 2^40 (comparison sort of
    (rank, id) pairs); CUSTOM_EXTREME: int64 minimum, zero and maximum."""
    k = rng.integers(0, 7, size=n).astype(np.int64)
    if kind == "CUSTOM":
        return k
    if kind == "CUSTOM_WIDE":
        return (k - 3) * (np.int64(1) << 40)
    i64 = np.iinfo(np.int64)
    return np.choose(k % 3, [np.int64(i64.min), np.int64(0), np.int64(i64.max)]).astype(np.int64)


@pytest.mark.parametrize("strategy", ["PARALL", "SEQFIX", "TOPO", "TOPO_FB", "CUSTOM", "CUSTOM_WIDE",
                                      "CUSTOM_EXTREME"])
def test_levels_bit_exact_vs_oracle(lib, strategy):
    rng = np.random.default_rng(1)
    custom_kind = strategy if strategy.startswith("CUSTOM") else None
    if custom_kind:
        strategy = "CUSTOM"
    for g in _graphs():
        if g.n_edges > 100000 and strategy in ("SEQFIX", "CUSTOM"):
            continue
        o = O.Oracle(g)
        halves = [False, True] if strategy == "TOPO_FB" else [False]
        custom = _custom_ranks(custom_kind, rng, g.n_edges) if custom_kind else None
        for back in halves:
            ostrat = "TOPO" if strategy == "TOPO_FB" else strategy
            try:
                r = o.ranks(ostrat, custom=custom, backward=back)
            except ValueError:  # cyclic graph: both sides must refuse TOPO
                with pytest.raises(F.FbpError) as ei:
                    F.fbp_schedule_build_host(g.n_vars, g.n_factors, g.factor_ptr, g.factor_vars,
                                              strategy, backward=back)
                assert ei.value.code == F.FBP_ERR_SCHEDULE
                continue
            want = o.levels(r)
            got = F.fbp_schedule_build_host(g.n_vars, g.n_factors, g.factor_ptr, g.factor_vars,
                                            strategy, edge_rank=custom, backward=back)
            assert np.array_equal(got[0], want[0]), (g.name, strategy, back)
            assert np.array_equal(got[1], want[1]), (g.name, strategy, back)


def test_levels_worked_example(lib):
    g = gen.fig1_example()
    lp, le = F.fbp_schedule_build_host(g.n_vars, g.n_factors, g.factor_ptr, g.factor_vars, "SEQFIX")
    assert lp.tolist() == [0, 3, 7, 10]
    assert le.tolist() == list(range(10))


def test_topo_cycle_is_schedule_error(lib):
    g = gen.bingo(n_tuples=500, seed=9, back_frac=0.2)
    with pytest.raises(F.FbpError) as ei:
        F.fbp_schedule_build_host(g.n_vars, g.n_factors, g.factor_ptr, g.factor_vars, "TOPO")
    assert ei.value.code == F.FBP_ERR_SCHEDULE


def test_custom_without_ranks_is_invalid(lib):
    g = gen.fig1_example()
    with pytest.raises(F.FbpError) as ei:
        F.fbp_schedule_build_host(g.n_vars, g.n_factors, g.factor_ptr, g.factor_vars, "CUSTOM")
    assert ei.value.code == F.FBP_ERR_INVALID_ARG
