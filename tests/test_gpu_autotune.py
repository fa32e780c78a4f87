"""The single-graph autotuner: it picks one of its candidate launch shapes,
and the run it tunes computes the same messages bit for bit (neither the
level engine's shapes nor the flooding split change the arithmetic)."""
import numpy as np
import pytest

from paper_2509_22337_gb300 import autotune, gen

pytestmark = pytest.mark.gpu


def _run(G, iters):
    G.reset()
    G.run(iters, 0.0)
    return G.messages(), G.marginals()


@pytest.mark.parametrize("strategy,graph", [
    ("SEQFIX", lambda: gen.tiny()),
    ("TOPO_FB", lambda: gen.smartfl(n_layers=20, width=50, seed=81)),
    ("PARALL", lambda: gen.bingo(n_tuples=3000, seed=82)),
])
def test_tuned_shape_is_a_candidate_and_keeps_results(fbp, tmp_path, monkeypatch, strategy, graph):
    monkeypatch.setattr(autotune, "CACHE", str(tmp_path / "tune.json"))
    g = graph()
    G = fbp.Graph(g, strategy)
    m0, p0 = _run(G, 10)
    opts = autotune.tune_graph(G, g, strategy, sample_iters=3)
    assert opts in list(autotune.graph_candidates(strategy))
    m1, p1 = _run(G, 10)
    assert np.array_equal(m1, m0) and np.array_equal(p1, p0)
    # a second graph of the same shape takes the cached choice without a search
    # (its signature counts levels, which a handle knows after its first run)
    H = fbp.Graph(g, strategy)
    H.run(1, 0.0)
    assert autotune.tune_graph(H, g, strategy, sample_iters=3) == opts
    G.close()
    H.close()
