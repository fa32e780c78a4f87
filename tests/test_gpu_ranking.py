"""The alarm-ranking loop (Sec. 5.3) on the GPU against the FP64 oracle.

The oracle replays the GPU's inspection sequence.  Before every question the
alarms' marginals agree within 1e-5, and the GPU's choice is a valid one: its
oracle marginal lies within 1e-5 of the best uninspected alarm's, since
alarms of equal probability may be taken in either order.  The oracle then
clamps the same answer and re-runs warm, as the GPU did.  Synchronous BP
(PARALL) does not always converge again after an answer; an oscillating run
has no fixed point to compare, so the replay compares up to the first answer
after which the oracle's run did not converge (or left FP32's range)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2509_22337_gb300 import gen, ranking

pytestmark = pytest.mark.gpu
TOL_P = 1e-5


def replay_on_oracle(g, strategy, alarms, run, max_iters, tol):
    """Returns the number of questions compared."""
    o = O.Oracle(g)
    r = o.run(strategy, max_iters, tol)
    a2v = r["a2v"]
    inspected = np.zeros(alarms.size, bool)
    where = {int(a): k for k, a in enumerate(alarms)}
    for t, (a, lab) in enumerate(zip(run["order"], run["labels"])):
        if not r["converged"] or r["min_pos"] < 1e-36:  # no fixed point, or outside FP32's range
            return t
        p = o.marginals(a2v)[alarms]
        err = np.abs(p - run["p_alarms"][t]).max()
        assert err <= TOL_P, f"{g.name} {strategy}: step {t}, max |dp| over alarms {err:.2e}"
        k = where[a]
        best = np.where(inspected, -np.inf, p).max()
        assert not inspected[k] and p[k] >= best - TOL_P, f"{g.name} {strategy}: step {t} chose {a}"
        inspected[k] = True
        o.set_evidence(a, lab)
        r = o.run(strategy, max_iters, tol, a2v=a2v)
        a2v = r["a2v"]
    return len(run["order"])


@pytest.mark.parametrize("strategy", ["PARALL", "SEQFIX"])
def test_ranking_loop_matches_oracle(fbp, strategy):
    """Derivation DAGs of the tiny configuration's shape: BP converges again
    after every answer, so all 30 questions are compared."""
    for seed in (1, 2):
        g = gen.tiny(seed=seed)
        alarms, truth = gen.planted_alarms(g, 30, seed=5, fire=0.8)
        run = _gpu_loop(fbp, g, strategy, alarms, truth)
        compared = replay_on_oracle(g, strategy, alarms, run, 500, 1e-6)
        assert compared == alarms.size
        _report(g, strategy, compared, run)


def test_ranking_loop_bingo_shaped(fbp):
    """A cyclic BINGO-shaped graph under asynchronous BP (SEQFIX): compared up
    to the first answer after which the oracle does not converge again."""
    g = gen.bingo(n_tuples=600, seed=47, back_frac=0.05)
    alarms, truth = gen.planted_alarms(g, 30, seed=48)
    run = _gpu_loop(fbp, g, "SEQFIX", alarms, truth)
    compared = replay_on_oracle(g, "SEQFIX", alarms, run, 500, 1e-6)
    assert compared >= 10
    _report(g, "SEQFIX", compared, run)


def _gpu_loop(fbp, g, strategy, alarms, truth):
    G = fbp.Graph(g, strategy)
    G.run(500, 1e-6)
    run = ranking.run_loop(G, alarms, truth, 500, 1e-6, record=True)
    G.close()
    assert sorted(run["order"]) == sorted(alarms.tolist())
    return run


def _report(g, strategy, compared, run):
    print(f"{g.name} {strategy}: {compared} questions compared; inversions {run['inversions']}, "
          f"Rank-100%-T {run['rank100']}, Rank-90%-T {run['rank90']}, "
          f"BP iterations per answer {np.mean(run['iters']):.1f}")
