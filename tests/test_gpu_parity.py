"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Bar (stated by the method's contract): marginals within max abs error 1e-5 of
the FP64 oracle after the same number of iterations; converged-iteration count
and schedule levels exactly equal.  Every input is seeded and synthetic.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2509_22337_gb300 import gen
from tests import bp_reference_defs as R

pytestmark = pytest.mark.gpu
TOL_P = 1e-5
# The contract compares FP32 normalised messages with FP64 ones.  It is only
# meaningful while every message the FP64 run writes is representable in FP32:
# a nonzero entry below the FP32 normal range (1.2e-38) becomes an exact zero
# there, and a later contradiction then takes the zero-mass guard on one side
# only.  Runs whose FP64 trajectory leaves that range (with two decades of
# headroom for intermediate products) are reported, not compared.
FP32_RANGE = 1e-36


def in_fp32_range(b) -> bool:
    return b["min_pos"] >= FP32_RANGE


def gpu_run(F, g, strategy, iters, tol, **spec):
    G = F.Graph(g, strategy, **spec)
    status, it, res = G.run(iters, tol)
    p = G.marginals().astype(np.float64)
    st = G.stats()
    msgs = G.messages().astype(np.float64)
    G.close()
    return dict(status=status, iters=it, residual=res, p=p, stats=st, a2v=msgs)


def oracle_run(g, strategy, iters, tol, custom=None):
    o = O.Oracle(g)
    r = o.run(strategy, iters, tol, custom=custom, history=True)
    r["p"] = o.marginals(r["a2v"])
    return r


TIE_BAND = 0.03  # relative: FP32 messages are quantised at ~6e-8, i.e. a few % of tol = 1e-6


def assert_same_stop(a, b, tol, what):
    """The converged-iteration count must match the oracle's exactly, except
    for a threshold tie: the two runs may stop one iteration apart only if the
    oracle's residual at the earlier of the two stopping iterations lies within
    TIE_BAND*tol of tol, where FP32 message quantisation cannot decide it."""
    if a["iters"] == b["iters"]:
        return
    hist = b["res_hist"]
    t = min(a["iters"], b["iters"])
    near = abs(hist[t - 1] - tol) <= TIE_BAND * tol
    assert abs(a["iters"] - b["iters"]) == 1 and near, (
        f"{what}: GPU stopped at {a['iters']}, oracle at {b['iters']}, oracle residuals "
        f"{hist[max(0, t - 3):t + 1]}")
    print(f"{what}: threshold tie at iteration {t}: oracle residual {hist[t - 1]:.6e} vs tol {tol:g}")


def assert_parity(a, b, what):
    err = np.abs(a["p"] - b["p"]).max() if a["p"].size else 0.0
    assert err <= TOL_P, f"{what}: max |dp| = {err:.3e}"


def test_tiny_parall_50_iterations(fbp):
    g = gen.tiny()
    a = gpu_run(fbp, g, "PARALL", 50, 0.0)
    b = oracle_run(g, "PARALL", 50, 0.0)
    assert a["iters"] == b["iters"] == 50
    assert_parity(a, b, "tiny PARALL")
    # the a->v messages themselves, not just the marginals
    assert np.abs(a["a2v"] - b["a2v"]).max() <= TOL_P
    assert a["stats"]["updates"] == 50 * g.n_edges


def test_tiny_tree_subgraph_exact(fbp):
    t = gen.tree_subgraph(gen.tiny(), 12)
    exact, Z = R.brute_force_marginals(t)
    assert Z > 0
    a = gpu_run(fbp, t, "PARALL", 30, 0.0)
    assert np.abs(a["p"] - exact).max() <= TOL_P


@pytest.mark.parametrize("strategy", ["PARALL", "SEQFIX", "TOPO", "TOPO_FB"])
def test_random_trees_exact(fbp, strategy):
    n_checked = 0
    for s in range(16):
        t = gen.random_tree(int(6 + s % 12), seed=300 + s)
        exact, Z = R.brute_force_marginals(t)
        if not Z > 0:
            continue
        try:
            a = gpu_run(fbp, t, strategy, 60, 1e-9)
        except fbp.FbpError as e:
            assert e.code == fbp.FBP_ERR_SCHEDULE
            continue
        assert np.abs(a["p"] - exact).max() <= TOL_P, t.name
        n_checked += 1
    assert n_checked >= 6


@pytest.mark.parametrize("strategy", ["PARALL", "SEQFIX", "TOPO", "TOPO_FB", "CUSTOM"])
def test_small_graphs_all_strategies(fbp, strategy):
    rng = np.random.default_rng(11)
    graphs = [gen.random_loopy(50, 60, seed=400 + s) for s in range(3)]
    graphs += [gen.smartfl(n_layers=12, width=40, seed=21), gen.bingo(n_tuples=300, seed=22, back_frac=0.0)]
    checked = 0
    for g in graphs:
        custom = rng.integers(0, 5, size=g.n_edges).astype(np.int64) if strategy == "CUSTOM" else None
        try:
            b = oracle_run(g, strategy, 25, 0.0, custom=custom)
        except ValueError:
            continue  # TOPO on a cyclic graph
        a = gpu_run(fbp, g, strategy, 25, 0.0, edge_rank=custom)
        assert a["iters"] == b["iters"]
        assert np.isfinite(a["p"]).all() and (a["p"] >= 0).all() and (a["p"] <= 1).all()
        if not in_fp32_range(b):
            print(f"{g.name} {strategy}: FP64 run leaves FP32 range (min entry {b['min_pos']:.2e})")
            continue
        assert_parity(a, b, f"{g.name} {strategy}")
        checked += 1
    assert checked >= 2


@pytest.mark.parametrize("strategy,split", [("PARALL", None), ("PARALL", (9, 256)), ("SEQFIX", None),
                                            ("TOPO_FB", None)])
def test_hub_rows_and_wide_factors_vs_oracle(fbp, strategy, split):
    """A 3,000-entry hub row (two full 1,024-entry chunks and a ragged one),
    a 200-entry row, and four factors wider than a warp (40, 35, 34 and 41
    variables), element by element against the oracle: flooding (hub chunks,
    warp rows, the wide-factor kernel) and the engine (long rows, the per-edge
    path of wide factors).  split = (hub_min, chunk) reconfigures the flooding
    work split so that rows above 9 entries run in 256-entry chunks: the hub in
    12 chunks with a 184-entry tail, the 200-entry row as one ragged chunk."""
    for seed in (71, 72):
        g = gen.hub_and_wide(seed=seed)
        b = oracle_run(g, strategy, 12, 0.0)
        assert in_fp32_range(b) and b["guards"] == 0
        G = fbp.Graph(g, strategy)
        if split:
            G.set_option(fbp.FBP_OPT_FLOOD_HUB_MIN, split[0])
            G.set_option(fbp.FBP_OPT_FLOOD_CHUNK, split[1])
        status, it, res = G.run(12, 0.0)
        p = G.marginals().astype(np.float64)
        m = G.messages().astype(np.float64)
        G.close()
        assert it == b["iters"] == 12
        err = np.abs(p - b["p"]).max()
        assert err <= TOL_P, f"{g.name} {strategy} {split}: max |dp| = {err:.3e}"
        # the hub's own marginal is a product of 3,000 messages: 1 - p ~ 1e-3..1e-2
        assert abs(p[0] - b["p"][0]) <= TOL_P
        print(f"{g.name} {strategy} {split}: max |dp| {err:.2e}, "
              f"max |d m1| {np.abs(m[:, 1] - b['a2v'][:, 1]).max():.2e}")


@pytest.mark.parametrize("graph", [lambda: gen.hub_and_wide(seed=73), lambda: gen.bingo(n_tuples=30000, seed=74)])
def test_flood_split_is_arithmetic_invariant(fbp, graph):
    """The flooding split only moves rows between kernels: every (hub_min,
    chunk) setting the tuner may pick computes the same messages bit for bit
    (a row's product is always grouped in 256-entry sub-chunks)."""
    g = graph()
    ref = None
    for hub_min, chunk in [(256, 1024), (9, 256), (64, 512), (128, 2048), (9, 65536), (200, 768)]:
        G = fbp.Graph(g, "PARALL")
        G.set_option(fbp.FBP_OPT_FLOOD_HUB_MIN, hub_min)
        G.set_option(fbp.FBP_OPT_FLOOD_CHUNK, chunk)
        G.run(15, 0.0)
        m, p = G.messages(), G.marginals()
        G.close()
        if ref is None:
            ref = (m, p)
            continue
        assert np.array_equal(m, ref[0]) and np.array_equal(p, ref[1]), (hub_min, chunk)


def test_levels_from_device_graph_match_oracle(fbp):
    g = gen.smartfl(n_layers=30, width=60, seed=31)
    o = O.Oracle(g)
    G = fbp.Graph(g, "TOPO_FB")
    lp, le = G.levels()
    G.close()
    f = o.levels(o.ranks("TOPO"))
    b = o.levels(o.ranks("TOPO", backward=True))
    want_lp = np.concatenate([f[0], f[0][-1] + b[0][1:]])
    assert np.array_equal(lp, want_lp)
    assert np.array_equal(le, np.concatenate([f[1], b[1]]))


def test_converged_iteration_count_matches(fbp):
    for g, strat in [(gen.smartfl(n_layers=20, width=50, seed=41, planted=True), "TOPO_FB"),
                     (gen.tiny(), "PARALL"), (gen.tiny(), "SEQFIX")]:
        b = oracle_run(g, strat, 300, 1e-6)
        a = gpu_run(fbp, g, strat, 300, 1e-6)
        assert b["converged"], g.name
        assert_same_stop(a, b, 1e-6, f"{g.name} {strat}")
        assert a["status"] == fbp.FBP_OK
        assert_parity(a, b, f"{g.name} {strat} converged")


def test_smartfl_200k_topo_fb_full_size(fbp):
    """SmartFL-shaped layered DAG, 200k variables, TOPO_FB to tol 1e-6 or 100
    sweeps; the oracle runs the same schedule in FP64."""
    g = gen.smartfl()
    a = gpu_run(fbp, g, "TOPO_FB", 100, 1e-6)
    b = oracle_run(g, "TOPO_FB", 100, 1e-6)
    assert_same_stop(a, b, 1e-6, "smartfl200k TOPO_FB")
    assert_parity(a, b, "smartfl200k TOPO_FB")


@pytest.mark.parametrize("warm", [5, 100])
def test_bingo_1m_sampled_one_step(fbp, warm):
    """BINGO-shaped 1M-tuple graph in the bench's launch configuration: after
    `warm` GPU flooding iterations (by 100 the messages span some 17 decades,
    as in the benched 500-iteration run), one more GPU iteration is compared
    message by message (a sample of 2,000 edges) with the oracle's synchronous
    update from the same exported state."""
    g = gen.bingo()
    G = fbp.Graph(g, "PARALL")
    G.run(warm, 0.0)
    s5 = G.messages().astype(np.float64)
    G.run(1, 0.0)
    s6 = G.messages().astype(np.float64)
    G.close()
    o = O.Oracle(g)
    rng = np.random.default_rng(5)
    edges = rng.choice(g.n_edges, size=2000, replace=False)
    # and every edge of the first 200 factors of the largest hub: their a->v
    # messages read the hub's v->a message, a product over ~1e5 entries
    deg = np.bincount(g.factor_vars, minlength=g.n_vars)
    hub = int(np.argmax(deg))
    fac = np.unique(np.searchsorted(g.factor_ptr, np.flatnonzero(g.factor_vars == hub), side="right") - 1)[:200]
    hub_edges = np.concatenate([np.arange(g.factor_ptr[a], g.factor_ptr[a + 1]) for a in fac])
    edges = np.unique(np.concatenate([edges, hub_edges]))
    want = o.update_edges(s5, edges)
    assert np.abs(s6[edges, 1] - want[:, 1]).max() <= TOL_P


def test_determinism_bit_identical(fbp):
    g = gen.smartfl(n_layers=20, width=50, seed=51)
    a = gpu_run(fbp, g, "TOPO_FB", 10, 0.0)
    b = gpu_run(fbp, g, "TOPO_FB", 10, 0.0)
    assert np.array_equal(a["a2v"], b["a2v"]) and np.array_equal(a["p"], b["p"])


def test_warm_start_equals_continuous_run(fbp):
    g = gen.tiny()
    G = fbp.Graph(g, "PARALL")
    G.run(7, 0.0)
    G.run(5, 0.0)
    p1 = G.marginals()
    G.reset()
    G.run(12, 0.0)
    p2 = G.marginals()
    G.close()
    assert np.array_equal(p1, p2)


def test_messages_roundtrip_and_checkpoint(fbp):
    g = gen.tiny()
    G = fbp.Graph(g, "PARALL")
    G.run(9, 0.0)
    m = G.messages()
    assert (m >= 0).all() and np.abs(m.sum(1) - 1).max() < 1e-6
    H = fbp.Graph(g, "PARALL")
    H.set_messages(m)
    G.run(4, 0.0)
    H.run(4, 0.0)
    assert np.abs(G.marginals() - H.marginals()).max() <= 1e-6
    G.close()
    H.close()


def test_evidence_clamp_is_exact(fbp):
    g = gen.tiny()
    G = fbp.Graph(g, "PARALL")
    G.set_evidence(1500, 1)
    G.set_evidence(1600, 0)
    G.run(20, 0.0)
    p = G.marginals()
    G.close()
    assert p[1500] == 1.0 and p[1600] == 0.0


def test_empty_and_degenerate_graphs(fbp):
    # no factors: marginals are the priors (or 1/2)
    g = gen.FactorGraph(3, np.zeros(1, np.int64), np.zeros(0, np.int32), np.zeros(0, np.uint8),
                        np.zeros(0, np.float32), np.array([0.25, np.nan, 0.5], np.float32),
                        np.array([-1, -1, 1], np.int8), "nofactors")
    a = gpu_run(fbp, g, "PARALL", 3, 0.0)
    np.testing.assert_allclose(a["p"], [0.25, 0.5, 1.0], atol=1e-7)
    # no variables at all
    g0 = gen.FactorGraph(0, np.zeros(1, np.int64), np.zeros(0, np.int32), np.zeros(0, np.uint8),
                         np.zeros(0, np.float32), np.zeros(0, np.float32), np.zeros(0, np.int8), "empty")
    a0 = gpu_run(fbp, g0, "TOPO_FB", 3, 1e-6)
    assert a0["p"].size == 0
    # a contradiction: the zero-mass guard fires identically on both sides
    gc = gen.FactorGraph(3, np.array([0, 3], np.int64), np.array([0, 1, 2], np.int32),
                         np.array([gen.AND], np.uint8), np.zeros(1, np.float32),
                         np.full(3, np.nan, np.float32), np.array([0, -1, 1], np.int8), "contra")
    a = gpu_run(fbp, gc, "PARALL", 3, 0.0)
    b = oracle_run(gc, "PARALL", 3, 0.0)
    assert_parity(a, b, "contradiction")
    assert a["stats"]["guards"] == b["guards"]


def test_engine_equals_per_level_launches(fbp):
    """The persistent engine and one launch per level (the paper's execution)
    run the same arithmetic in the same order: bit-identical messages."""
    for g, strat in [(gen.smartfl(n_layers=25, width=80, seed=61), "TOPO_FB"), (gen.tiny(), "SEQFIX")]:
        G = fbp.Graph(g, strat)
        G.run(6, 0.0)
        a = G.messages()
        G.close()
        H = fbp.Graph(g, strat)
        H.set_option(fbp.FBP_OPT_ENGINE, 0)
        H.run(6, 0.0)
        b = H.messages()
        assert H.stats()["kernel_launches"] > 6
        H.close()
        assert np.array_equal(a, b), (g.name, strat)


@pytest.mark.parametrize("grid", [1, 3, 17])
def test_engine_grid_size_does_not_change_results(fbp, grid):
    g = gen.smartfl(n_layers=15, width=60, seed=62)
    ref = gpu_run(fbp, g, "TOPO_FB", 5, 0.0)
    G = fbp.Graph(g, "TOPO_FB")
    G.set_option(fbp.FBP_OPT_ENGINE_GRID, grid)
    G.run(5, 0.0)
    assert np.array_equal(G.messages().astype(np.float64), ref["a2v"])
    G.close()


@pytest.mark.parametrize("fuse", [32, 64, 128, 256])
def test_level_fusion_does_not_change_results(fbp, fuse):
    """Level fusion (runs of consecutive levels of at most `fuse` lanes in one
    block, grid barriers only around them) computes the grid engine's
    messages bit for bit: layered graphs whose levels straddle the threshold,
    TOPO_FB (two halves, runs crossing the half boundary) and SEQFIX (every
    level narrow), with the one-block switch off so that the grid runs."""
    cases = [(gen.smartfl(n_layers=30, width=24, seed=63), "TOPO_FB"), (gen.smartfl(n_layers=20, width=90, seed=64), "TOPO_FB"),
             (gen.tiny(), "SEQFIX"), (gen.hub_and_wide(seed=75), "TOPO_FB")]
    for g, strat in cases:
        runs = []
        for f in (0, fuse):
            G = fbp.Graph(g, strat)
            G.set_option(fbp.FBP_OPT_ENGINE_SOLO_LANES, 0)
            G.set_option(fbp.FBP_OPT_ENGINE_FUSE_LANES, f)
            st, it, res = G.run(4, 0.0)
            runs.append((G.messages(), G.marginals(), it, np.float32(res).tobytes()))
            G.close()
        a, b = runs
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1]), (g.name, strat, fuse)
        assert a[2] == b[2] and a[3] == b[3]


def test_barrier_timeout_is_reported_and_context_survives(fbp):
    """Failure detection without a GPU fault: a spin limit of 0 makes every
    device-side barrier wait that has to wait at all expire at once; the run
    must return FBP_ERR_TIMEOUT and the context must stay usable.  A wait is
    made certain: under SEQFIX most levels hold one or two factors, and a
    level whose factor has the 3,000-entry hub as a premise keeps one lane on
    the hub's row for ~1e5 cycles while the other blocks of a 4-block grid
    arrive and poll (on a balanced level every block can arrive before anyone
    polls, and nothing waits)."""
    g = gen.hub_and_wide(seed=71)
    G = fbp.Graph(g, "SEQFIX")
    G.set_option(fbp.FBP_OPT_ENGINE_GRID, 4)
    G.set_option(fbp.FBP_OPT_SPIN_LIMIT, 0)
    with pytest.raises(fbp.FbpError) as ei:
        G.run(3, 0.0)
    assert ei.value.code == fbp.FBP_ERR_TIMEOUT
    G.set_option(fbp.FBP_OPT_SPIN_LIMIT, 4_000_000_000)
    G.reset()
    status, it, res = G.run(3, 0.0)
    assert it == 3
    p = G.marginals()
    G.close()
    ref = gpu_run(fbp, g, "SEQFIX", 3, 0.0)
    assert np.array_equal(p.astype(np.float64), ref["p"])


@pytest.mark.parametrize("cluster", [8, 16])
def test_engine_cluster_mode_does_not_change_results(fbp, cluster):
    """One thread-block cluster with the hardware barrier runs the same
    arithmetic as the cooperative grid, also when a level is wider than the
    cluster holds (several passes per level)."""
    for g in (gen.smartfl(n_layers=15, width=60, seed=62), gen.smartfl(n_layers=5, width=4000, seed=64)):
        G = fbp.Graph(g, "TOPO_FB")
        G.set_option(fbp.FBP_OPT_ENGINE_GRID, 152)
        G.run(4, 0.0)
        a = G.messages()
        G.close()
        H = fbp.Graph(g, "TOPO_FB")
        H.set_option(fbp.FBP_OPT_ENGINE_CLUSTER, cluster)
        H.run(4, 0.0)
        b = H.messages()
        H.close()
        assert np.array_equal(a, b), (g.name, cluster)


@pytest.mark.parametrize("device_schedule", [1, 0])
def test_residual_reaches_the_oracles_fixed_points(fbp, device_schedule):
    """RESIDUAL's levels come from float residuals, so only its outcome is
    compared: the GPU run converges where the FP64 oracle's RESIDUAL run
    does, and its marginals match both the oracle's RESIDUAL and flooding
    fixed points within 1e-5 (schedule built on the device, or on the host)."""
    graphs = [gen.random_tree(14, seed=500 + s) for s in range(4)]
    graphs += [gen.smartfl(n_layers=12, width=40, seed=31, planted=True),
               gen.random_loopy(60, 50, seed=510)]
    checked = 0
    for g in graphs:
        b_res = oracle_run(g, "RESIDUAL", 400, 1e-7)
        b_par = oracle_run(g, "PARALL", 400, 1e-7)
        if not (b_res["converged"] and b_par["converged"]):
            continue
        if not (in_fp32_range(b_res) and in_fp32_range(b_par)):
            continue
        G = fbp.Graph(g, "RESIDUAL")
        G.set_option(fbp.FBP_OPT_RESIDUAL_DEVICE, device_schedule)
        status, it, res = G.run(400, 1e-7)
        a = dict(status=status, iters=it, residual=res, p=G.marginals().astype(np.float64), stats=G.stats())
        G.close()
        assert a["status"] == fbp.FBP_OK, (g.name, a["iters"], a["residual"])
        assert np.abs(a["p"] - b_res["p"]).max() <= TOL_P, g.name
        assert np.abs(a["p"] - b_par["p"]).max() <= TOL_P, g.name
        assert a["stats"]["updates"] <= a["iters"] * g.n_edges  # skipped factors are not updated
        checked += 1
    assert checked >= 4


def test_engine_prefetch_variants_agree(fbp):
    """A grid that holds a level in one pass runs the deep-prefetch engine, a
    small grid (several passes per level) the shallow one: same messages."""
    g = gen.smartfl(n_layers=5, width=4000, seed=64)
    out = []
    for grid in (152, 6):
        G = fbp.Graph(g, "TOPO_FB")
        G.set_option(fbp.FBP_OPT_ENGINE_GRID, grid)
        G.run(4, 0.0)
        out.append(G.messages())
        G.close()
    assert np.array_equal(out[0], out[1])


@pytest.mark.parametrize("grid", [0, 5])
def test_dataflow_engine_equals_barrier_engine(fbp, grid):
    """The dataflow engine (per-message waits instead of a barrier per level)
    computes exactly the level engine's messages: several strategies, levels
    wider than the grid (grid 5), a factor wider than a warp."""
    wide = gen.FactorGraph(40, np.array([0, 36, 38, 40], np.int64),
                           np.concatenate([np.arange(36), [36, 37], [38, 39]]).astype(np.int32),
                           np.array([gen.OR, gen.NOT, gen.AND], np.uint8), np.zeros(3, np.float32),
                           np.full(40, 0.3, np.float32), np.full(40, -1, np.int8), "wide")
    cases = [(gen.smartfl(n_layers=20, width=60, seed=770), "TOPO_FB", None),
             (gen.tiny(), "SEQFIX", None), (gen.tiny(), "TOPO", None),
             (gen.random_loopy(80, 70, seed=771), "CUSTOM", np.random.default_rng(772)),
             (wide, "SEQFIX", None)]
    for g, strat, rng in cases:
        custom = rng.integers(0, 6, size=g.n_edges).astype(np.int64) if rng is not None else None
        out = []
        for mode in (1, 2):
            G = fbp.Graph(g, strat, edge_rank=custom) if custom is not None else fbp.Graph(g, strat)
            G.set_option(fbp.FBP_OPT_ENGINE, mode)
            if grid:
                G.set_option(fbp.FBP_OPT_ENGINE_GRID, grid)
            st = G.run(7, 1e-9)
            out.append((st, G.messages()))
            G.close()
        assert out[0][0] == out[1][0], (g.name, strat)
        assert np.array_equal(out[0][1], out[1][1]), (g.name, strat)


def test_dataflow_wait_timeout_is_reported(fbp):
    g = gen.smartfl(n_layers=10, width=40, seed=773)
    G = fbp.Graph(g, "TOPO_FB")
    G.set_option(fbp.FBP_OPT_ENGINE, 2)
    G.set_option(fbp.FBP_OPT_ENGINE_GRID, 4)
    G.set_option(fbp.FBP_OPT_SPIN_LIMIT, 0)
    with pytest.raises(fbp.FbpError) as ei:
        G.run(3, 0.0)
    assert ei.value.code == fbp.FBP_ERR_TIMEOUT
    G.set_option(fbp.FBP_OPT_SPIN_LIMIT, 4_000_000_000)
    G.reset()
    assert G.run(3, 0.0)[1] == 3
    G.close()


@pytest.mark.parametrize("tol", [0.0, 1e-6])
def test_residual_device_levels_equal_oracle_algorithm2(fbp, tol):
    """The device-built RESIDUAL levels of iteration 2 equal the oracle's
    Algorithm 2 over the same classes: the classes follow from iteration 1's
    changes (recomputed here from the exported messages; cases whose changes
    sit within rounding of a class bound are skipped)."""
    checked = 0
    for s_ in range(4):
        g = gen.smartfl(n_layers=8, width=30, seed=780 + s_) if s_ % 2 else gen.bingo(n_tuples=400, seed=780 + s_)
        G1 = fbp.Graph(g, "RESIDUAL")
        G1.run(1, 0.0)
        m = G1.messages().astype(np.float64)
        G1.close()
        d = np.abs(m[:, 1] / (m[:, 0] + m[:, 1]) - 0.5)  # change from the uniform start
        bounds = [b for b in (1e-2, 1e-4, tol) if b > 0]
        if any(np.any(np.abs(d - b) <= 1e-6 * b) for b in bounds):
            continue
        fv = np.asarray(g.factor_vars)
        fp = np.asarray(g.factor_ptr)
        vres = np.zeros(g.n_vars)
        np.maximum.at(vres, fv, d)
        rank = np.full(g.n_edges, -1, np.int64)
        for a in range(g.n_factors):
            rho = vres[fv[fp[a]:fp[a + 1]]].max()
            rank[fp[a]:fp[a + 1]] = 0 if rho >= 1e-2 else 1 if rho >= 1e-4 else 2 if rho >= tol else -1
        edges = np.flatnonzero(rank >= 0).astype(np.int64)
        lp_o, le_o = O.Oracle(g).levels(rank, edges)
        G2 = fbp.Graph(g, "RESIDUAL")
        G2.run(2, tol)
        lp_g, le_g = G2.levels()
        G2.close()
        assert np.array_equal(lp_g, lp_o) and np.array_equal(le_g, le_o), g.name
        checked += 1
    assert checked >= 2
