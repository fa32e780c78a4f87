"""Batched form: many independent graphs in one run must give, for every
member, exactly what a single-graph run of it gives (same iterations, same
messages, same marginals), and match the FP64 oracle like a single run; in
both of its forms (one persistent launch of thread-block clusters taking
members from a queue; static members in that queue beside the whole-GPU
flooding kernels; static members in one level-engine launch beside them)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2509_22337_gb300 import gen

pytestmark = pytest.mark.gpu

FORMS = [pytest.param(True, None, id="one_launch"), pytest.param(False, True, id="static_queue"),
         pytest.param(False, False, id="engine")]


def _mixed_graphs():
    gs, sch, mi, tol = [], [], [], []
    for i, n in enumerate([300, 1200, 4000, 700, 2500, 9000]):
        layers = max(5, n // 300)
        gs.append(gen.smartfl(n_layers=layers, width=max(n // layers, 4), seed=900 + i))
        sch.append("TOPO_FB")
        mi.append([40, 100, 60, 100, 25, 100][i])
        tol.append([1e-6, 1e-6, 1e-4, 1e-6, 0.0, 1e-5][i])
    for i, n in enumerate([200, 1500, 6000, 400, 3000]):
        gs.append(gen.bingo(n_tuples=n, seed=950 + i))
        sch.append("PARALL")
        mi.append([30, 80, 50, 200, 40][i])
        tol.append([1e-6, 1e-5, 1e-6, 1e-4, 0.0][i])
    gs.append(gen.tiny())
    sch.append("SEQFIX")
    mi.append(60)
    tol.append(1e-6)
    gs.append(gen.smartfl(n_layers=12, width=50, seed=990))
    sch.append("TOPO")
    mi.append(30)
    tol.append(1e-6)
    return gs, sch, mi, tol


@pytest.mark.parametrize("one_launch,static_queue", FORMS)
def test_batch_equals_single_runs(fbp, one_launch, static_queue):
    from paper_2509_22337_gb300 import fbp_batch as B
    gs, sch, mi, tol = _mixed_graphs()
    bt = B.Batch(gs, sch, mi, tol, one_launch=one_launch, static_queue=static_queue)
    assert bt.one_launch == one_launch
    rc, iters, res, status = bt.run()
    if one_launch:  # the whole batch: the queue kernel and the refresh of the flooding members' copy
        assert bt.stats()["kernel_launches"] == 2
    for i, g in enumerate(gs):
        G = fbp.Graph(g, sch[i])
        st, it, r = G.run(mi[i], tol[i])
        assert iters[i] == it, (i, sch[i], iters[i], it)
        assert status[i] == st, i
        assert np.float32(res[i]).tobytes() == np.float32(r).tobytes(), (i, sch[i], res[i], r)
        assert np.array_equal(bt.messages(i), G.messages()), (i, sch[i])
        assert np.array_equal(bt.marginals(i), G.marginals()), (i, sch[i])
        G.close()
    # a second run continues from the current messages, like fbp_run does
    bt.reset()
    rc2, iters2, _, _ = bt.run()
    assert np.array_equal(iters, iters2)
    bt.close()


@pytest.mark.parametrize("static_queue,engine_cluster,queue_clusters",
                         [(False, 1, 0), (False, 16, 0), (True, 8, 1), (True, 16, 3), (True, 8, 1 << 20)])
def test_batch_tuning_does_not_change_results(fbp, static_queue, engine_cluster, queue_clusters):
    from paper_2509_22337_gb300 import fbp_batch as B
    gs, sch, mi, tol = _mixed_graphs()
    ref = B.Batch(gs, sch, mi, tol, one_launch=False, static_queue=False)
    ref.run()
    bt = B.Batch(gs, sch, mi, tol, one_launch=False, static_queue=static_queue)
    bt.tune(engine_grid=0, engine_cluster=engine_cluster, queue_clusters=queue_clusters)
    bt.run()
    for i in range(len(gs)):
        assert np.array_equal(ref.messages(i), bt.messages(i)), i
    ref.close()
    bt.close()


@pytest.mark.parametrize("one_launch,static_queue", FORMS)
def test_batch_members_match_oracle(fbp, one_launch, static_queue):
    from paper_2509_22337_gb300 import fbp_batch as B
    gs = [gen.tiny(), gen.smartfl(n_layers=15, width=40, seed=77), gen.bingo(n_tuples=500, seed=78)]
    sch = ["PARALL", "TOPO_FB", "PARALL"]
    mi = [50, 30, 20]
    tol = [0.0, 0.0, 0.0]
    bt = B.Batch(gs, sch, mi, tol, one_launch=one_launch, static_queue=static_queue)
    rc, iters, res, status = bt.run()
    for i, g in enumerate(gs):
        o = O.Oracle(g)
        r = o.run(sch[i], mi[i], tol[i])
        assert iters[i] == r["iters"]
        if r["min_pos"] < 1e-36:
            continue
        p = o.marginals(r["a2v"])
        assert np.abs(bt.marginals(i).astype(np.float64) - p).max() <= 1e-5, i
    bt.close()


@pytest.mark.parametrize("one_launch,static_queue", FORMS)
def test_batch_single_kind_and_empty_member(fbp, one_launch, static_queue):
    from paper_2509_22337_gb300 import fbp_batch as B
    empty = gen.FactorGraph(4, np.zeros(1, np.int64), np.zeros(0, np.int32), np.zeros(0, np.uint8),
                            np.zeros(0, np.float32), np.array([0.2, np.nan, 0.7, np.nan], np.float32),
                            np.full(4, -1, np.int8), "empty")
    gs = [gen.smartfl(n_layers=8, width=30, seed=5), empty, gen.smartfl(n_layers=6, width=20, seed=6)]
    bt = B.Batch(gs, ["TOPO_FB"] * 3, [20, 20, 20], [1e-6] * 3, one_launch=one_launch, static_queue=static_queue)
    rc, iters, res, status = bt.run()
    np.testing.assert_allclose(bt.marginals(1), [0.2, 0.5, 0.7, 0.5], atol=1e-7)
    assert iters[1] == 1
    bt.close()


def test_many_graphs_of_different_sizes_interleaved(fbp):
    """Graph handles of different sizes used in any order (kernel attributes
    shared by all graphs must not be lowered by a smaller graph)."""
    big = gen.bingo(n_tuples=20000, seed=31)
    small = gen.bingo(n_tuples=300, seed=32)
    A, Bh = fbp.Graph(big, "PARALL"), fbp.Graph(small, "PARALL")
    A.run(2, 0.0)
    Bh.run(2, 0.0)
    A.run(2, 0.0)
    Bh.run(2, 0.0)
    A.close()
    Bh.close()


@pytest.mark.parametrize("one_launch,static_queue", FORMS)
def test_batch_autotuner(fbp, tmp_path, monkeypatch, one_launch, static_queue):
    """The batch tuner picks one of its candidates, and the tuned batch
    computes what the untuned one does, bit for bit for every member (no
    launch shape changes the arithmetic); a second call answers from the
    cache."""
    from paper_2509_22337_gb300 import autotune, fbp_batch as B
    monkeypatch.setattr(autotune, "CACHE", str(tmp_path / "tune.json"))
    gs, sch, mi, tol = _mixed_graphs()
    ref = B.Batch(gs, sch, mi, tol, one_launch=False, static_queue=False)
    ref.run()
    bt = B.Batch(gs, sch, mi, tol, one_launch=one_launch, static_queue=static_queue)
    best = autotune.tune_batch(bt, gs, sch)
    assert best in list(autotune.batch_candidates(bt.form))
    bt.reset()
    bt.run()
    for i in range(len(gs)):
        assert np.array_equal(ref.messages(i), bt.messages(i)), i
        assert np.array_equal(ref.marginals(i), bt.marginals(i)), i
    assert autotune.tune_batch(bt, gs, sch) == best
    ref.close()
    bt.close()


def test_one_launch_cluster_sizes_agree(fbp):
    """The one-launch form with 8-block and 16-block clusters computes the
    same messages, iterations and residuals (a cluster only carries a member)."""
    from paper_2509_22337_gb300 import fbp_batch as B
    gs, sch, mi, tol = _mixed_graphs()
    runs = []
    for cluster in (8, 16):
        bt = B.Batch(gs, sch, mi, tol, one_launch=True)
        bt.tune(engine_cluster=cluster)
        rc, iters, res, status = bt.run()
        runs.append(([bt.messages(i) for i in range(len(gs))], iters, res))
        bt.close()
    (m8, i8, r8), (m16, i16, r16) = runs
    assert np.array_equal(i8, i16) and np.array_equal(np.float32(r8), np.float32(r16))
    assert all(np.array_equal(a, b) for a, b in zip(m8, m16))
