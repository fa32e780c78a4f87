"""The belief-form sequential engine (FBP_OPT_ENGINE = 3): static schedules
run level by level with every variable's belief kept current (v->a = belief
/ own message), for graphs whose hubs make the row walk of the level engine
too slow.  Compared with the FP64 oracle's in-place level execution (Sec. 4.3,
Algorithm 2's levels): the same iterations, marginals within 1e-5; at
BINGO-1M size, sampled levels of a SEQFIX sweep message by message."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2509_22337_gb300 import gen
from tests.test_gpu_parity import TOL_P, assert_parity, assert_same_stop, in_fp32_range, oracle_run

pytestmark = pytest.mark.gpu

SEQ = 3  # FBP_OPT_ENGINE value of the belief-form sequential engine


def seq_run(F, g, strategy, iters, tol, custom=None):
    G = F.Graph(g, strategy, edge_rank=custom)
    G.set_option(F.FBP_OPT_ENGINE, SEQ)
    status, it, res = G.run(iters, tol)
    out = dict(status=status, iters=it, residual=res, p=G.marginals().astype(np.float64), stats=G.stats(),
               a2v=G.messages().astype(np.float64))
    lp, _ = G.levels()
    out["widest"] = int(np.diff(np.asarray(lp)).max()) if len(lp) > 1 else 0
    G.close()
    return out


def _graphs():
    return [gen.random_loopy(50, 60, seed=400), gen.random_loopy(50, 60, seed=401),
            gen.smartfl(n_layers=12, width=40, seed=21), gen.bingo(n_tuples=300, seed=22, back_frac=0.0),
            gen.smartfl(n_layers=8, width=400, seed=23)]


@pytest.mark.parametrize("strategy", ["SEQFIX", "TOPO", "TOPO_FB", "CUSTOM"])
def test_seq_engine_matches_oracle(fbp, strategy):
    rng = np.random.default_rng(12)
    checked, wide = 0, False
    for g in _graphs():
        custom = rng.integers(0, 5, size=g.n_edges).astype(np.int64) if strategy == "CUSTOM" else None
        try:
            b = oracle_run(g, strategy, 20, 0.0, custom=custom)
        except ValueError:
            continue  # TOPO on a cyclic graph
        a = seq_run(fbp, g, strategy, 20, 0.0, custom=custom)
        assert a["iters"] == b["iters"]
        assert np.isfinite(a["p"]).all() and (a["p"] >= 0).all() and (a["p"] <= 1).all()
        wide = wide or a["widest"] > 256
        if not in_fp32_range(b):
            print(f"{g.name} {strategy}: FP64 run leaves FP32 range (min entry {b['min_pos']:.2e})")
            continue
        assert_parity(a, b, f"{g.name} {strategy} (belief-form engine)")
        checked += 1
    assert checked >= 2
    if strategy in ("TOPO", "TOPO_FB"):
        assert wide  # a level wider than the block stages its messages


@pytest.mark.parametrize("strategy", ["SEQFIX", "TOPO_FB"])
def test_seq_engine_stops_where_the_oracle_does(fbp, strategy):
    for g in (gen.tiny(), gen.smartfl(n_layers=15, width=40, seed=77)):
        tol = 1e-6
        b = oracle_run(g, strategy, 200, tol)
        a = seq_run(fbp, g, strategy, 200, tol)
        assert_same_stop(a, b, tol, f"{g.name} {strategy}")
        assert a["status"] == 0 and a["residual"] < tol


def test_seq_engine_hub_rows_vs_oracle(fbp):
    """Rows longer than 256 entries (block combine) and of 9..256 entries
    (one-thread combine) are kept current level by level.  Four sweeps: on
    BINGO-shaped graphs FP32 runs drift from the FP64 one over many sweeps
    whichever engine runs them (messages reach 1e-17), which the sampled-level
    tests below sidestep."""
    g = gen.bingo(n_tuples=3000, seed=78)
    deg = np.bincount(g.factor_vars, minlength=g.n_vars)
    assert (deg > 256).any() and ((deg > 8) & (deg <= 256)).any()
    b = oracle_run(g, "SEQFIX", 4, 0.0)
    a = seq_run(fbp, g, "SEQFIX", 4, 0.0)
    assert a["iters"] == b["iters"] == 4
    if not in_fp32_range(b):
        pytest.skip(f"FP64 run leaves FP32 range (min entry {b['min_pos']:.2e}); the sampled-level tests cover it")
    assert_parity(a, b, "bingo3000 SEQFIX (belief-form engine)")
    assert np.abs(a["a2v"] - b["a2v"]).max() <= TOL_P


def _sampled_levels(fbp, g, n_levels_sampled, seed):
    """Two SEQFIX sweeps on the GPU; every edge is written once per sweep at
    its level, so the state level L of the second sweep started from is the
    first sweep's messages with the second sweep's for the edges of earlier
    levels.  Returns (state before, GPU result) for each sampled level."""
    G = fbp.Graph(g, "SEQFIX")
    G.set_option(fbp.FBP_OPT_ENGINE, SEQ)
    G.run(1, 0.0)
    s1 = G.messages().astype(np.float64)
    G.run(1, 0.0)
    s2 = G.messages().astype(np.float64)
    lp, le = (np.asarray(x) for x in G.levels())
    G.close()
    level_of = np.empty(g.n_edges, np.int64)
    level_of[le] = np.repeat(np.arange(len(lp) - 1), np.diff(lp))
    rng = np.random.default_rng(seed)
    deg = np.bincount(g.factor_vars, minlength=g.n_vars)
    hub = int(np.argmax(deg))
    hub_levels = np.unique(level_of[g.factor_vars == hub])
    picks = np.unique(np.concatenate([rng.choice(len(lp) - 1, size=n_levels_sampled, replace=False),
                                      rng.choice(hub_levels, size=min(5, hub_levels.size), replace=False),
                                      [len(lp) - 2]]))
    for L in picks:
        edges = le[lp[L]:lp[L + 1]].astype(np.int64)
        state = np.where((level_of < L)[:, None], s2, s1)
        yield L, state, edges, s2[edges]


def test_seq_engine_mid_size_sampled_levels(fbp):
    g = gen.bingo(n_tuples=20000, seed=79)
    o = O.Oracle(g)
    for L, state, edges, got in _sampled_levels(fbp, g, 30, 3):
        want = o.update_edges(state, edges)
        assert np.abs(got[:, 1] - want[:, 1]).max() <= TOL_P, L


def test_seq_engine_bingo_1m_sampled_levels(fbp):
    """BINGO-1M SEQFIX end to end (two sweeps of ~880k levels); 40 sampled
    levels of the second sweep, and levels that touch the largest hub (a row
    of ~1e5 entries), recomputed by the oracle from the state they started
    from."""
    g = gen.bingo()
    o = O.Oracle(g)
    n = 0
    for L, state, edges, got in _sampled_levels(fbp, g, 40, 4):
        want = o.update_edges(state, edges)
        assert np.abs(got[:, 1] - want[:, 1]).max() <= TOL_P, L
        n += edges.size
    assert n > 0
