"""Generic factors (FBP_TERMS: local structure as an explicit term list, the
indicator array of Sec. 4.3.2, evaluated by Algorithm 1) on the GPU against
the FP64 oracle, through the C ABI, in both execution paths (flooding and
the persistent level engine).  Bar as for every factor: marginals within
1e-5 after the same iterations, exact on trees."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2509_22337_gb300 import gen
from tests import bp_reference_defs as R

pytestmark = pytest.mark.gpu
TOL_P = 1e-5


def _run_gpu(fbp, g, strategy, iters, tol=0.0):
    G = fbp.Graph(g, strategy)
    status, it, res = G.run(iters, tol)
    p = G.marginals().astype(np.float64)
    G.close()
    return it, p


def _run_oracle(g, strategy, iters, tol=0.0):
    o = O.Oracle(g)
    r = o.run(strategy, iters, tol)
    return r, o.marginals(r["a2v"])


@pytest.mark.parametrize("strategy", ["PARALL", "SEQFIX", "TOPO_FB"])
def test_generic_factors_match_oracle(fbp, strategy):
    graphs = [gen.with_generic_factors(gen.random_loopy(60, 50, seed=700 + s), 0.5, seed=710 + s)
              for s in range(3)]
    graphs += [gen.with_generic_factors(gen.smartfl(n_layers=10, width=40, seed=720, planted=True), 0.3, seed=721)]
    checked = 0
    for g in graphs:
        try:
            r, pb = _run_oracle(g, strategy, 30)
        except ValueError:
            continue  # TOPO on a cyclic graph
        it, pa = _run_gpu(fbp, g, strategy, 30)
        assert it == r["iters"] == 30
        if r["min_pos"] < 1e-36:
            continue
        assert np.abs(pa - pb).max() <= TOL_P, (g.name, strategy, np.abs(pa - pb).max())
        checked += 1
    assert checked >= 2


def test_generic_factors_exact_on_trees(fbp):
    checked = 0
    for s in range(6):
        g = gen.with_generic_factors(gen.random_tree(int(8 + s % 7), seed=730 + s), 0.6, seed=740 + s)
        exact, Z = R.brute_force_marginals(g)
        if not Z > 0:
            continue
        for strategy in ("PARALL", "SEQFIX"):
            it, p = _run_gpu(fbp, g, strategy, 60)
            assert np.abs(p - exact).max() <= TOL_P, (g.name, strategy)
        checked += 1
    assert checked >= 4


def test_generic_with_a_types_terms_matches_the_type(fbp):
    """A graph whose factors all carry their own type's term list as generic
    factors gives the typed graph's marginals (two arithmetic routes: the
    closed forms and Algorithm 1)."""
    g = gen.smartfl(n_layers=8, width=30, seed=750, planted=True)
    fp = np.asarray(g.factor_ptr)
    tp, inds, ws = [0], [], []
    for a in range(g.n_factors):
        ind, w = O.terms(int(g.factor_type[a]), int(fp[a + 1] - fp[a]), float(g.factor_param[a]))
        inds.append(ind.T.reshape(-1))
        ws.append(w)
        tp.append(tp[-1] + w.shape[0])
    h = gen.FactorGraph(g.n_vars, g.factor_ptr, g.factor_vars, np.full(g.n_factors, gen.TERMS, np.uint8),
                        g.factor_param, g.prior_p1, g.evidence, "asterms", {},
                        (np.array(tp, np.int64), np.concatenate(inds).astype(np.int8), np.concatenate(ws)))
    for strategy in ("PARALL", "TOPO_FB"):
        _, pa = _run_gpu(fbp, g, strategy, 20)
        _, pb = _run_gpu(fbp, h, strategy, 20)
        assert np.abs(pa - pb).max() <= 1e-6, strategy


def test_generic_terms_required_and_validated(fbp):
    g = gen.with_generic_factors(gen.random_loopy(20, 15, seed=760), 1.0, seed=761)
    bare = gen.FactorGraph(g.n_vars, g.factor_ptr, g.factor_vars, g.factor_type, g.factor_param,
                           g.prior_p1, g.evidence, "bare")
    G = fbp.Graph(bare)
    with pytest.raises(fbp.FbpError) as ei:
        G.run(3, 0.0)
    assert ei.value.code == fbp.FBP_ERR_INVALID_ARG and "terms" in str(ei.value)
    S = fbp.Graph(bare, "SEQFIX")
    with pytest.raises(fbp.FbpError) as ei:
        S.run_fixed_scratch(3, 0.0)
    assert ei.value.code == fbp.FBP_ERR_INVALID_ARG and "terms" in str(ei.value)
    S.close()
    tp, ti, tw = g.terms
    for bad in [(tp, np.where(ti == 1, 3, ti), tw), (tp, ti, -np.asarray(tw)), (tp + 1, ti, tw)]:
        with pytest.raises(fbp.FbpError) as ei:
            fbp.fbp_set_factor_terms(G.h, *bad)
        assert ei.value.code == fbp.FBP_ERR_INVALID_ARG
    fbp.fbp_set_factor_terms(G.h, tp, ti, tw)
    status, it, res = G.run(3, 0.0)
    assert it == 3
    G.close()


@pytest.mark.parametrize("device_schedule", [1, 0])
def test_generic_factors_under_residual(fbp, device_schedule):
    """Generic factors under RESIDUAL (classes and levels built on the device,
    or on the host): the run converges and its marginals match the oracle's
    RESIDUAL and flooding fixed points within 1e-5."""
    graphs = [gen.with_generic_factors(gen.random_tree(14, seed=730 + s), 0.6, seed=740 + s) for s in range(4)]
    graphs += [gen.with_generic_factors(gen.smartfl(n_layers=10, width=40, seed=750, planted=True), 0.3, seed=751),
               gen.with_generic_factors(gen.random_loopy(60, 50, seed=760), 0.5, seed=761)]
    checked = 0
    for g in graphs:
        o = O.Oracle(g)
        r_res = o.run("RESIDUAL", 400, 1e-7)
        r_par = o.run("PARALL", 400, 1e-7)
        if not (r_res["converged"] and r_par["converged"]) or min(r_res["min_pos"], r_par["min_pos"]) < 1e-36:
            continue
        G = fbp.Graph(g, "RESIDUAL")
        G.set_option(fbp.FBP_OPT_RESIDUAL_DEVICE, device_schedule)
        status, it, res = G.run(400, 1e-7)
        pa = G.marginals().astype(np.float64)
        G.close()
        assert status == fbp.FBP_OK, (g.name, it, res)
        assert np.abs(pa - o.marginals(r_res["a2v"])).max() <= TOL_P, g.name
        assert np.abs(pa - o.marginals(r_par["a2v"])).max() <= TOL_P, g.name
        checked += 1
    assert checked >= 5
