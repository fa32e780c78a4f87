"""Alarm ranking with user feedback: the interactive loop of a Bayesian program
analysis such as BINGO, as the paper's evaluation runs it (Sec. 5.3).

In each interaction the user is asked about the uninspected alarm with the
highest P(x = 1); the answer is clamped on that variable as evidence, and BP
re-runs warm from the stored messages (fbp_set_evidence + fbp_run).  The
quality of a run is measured on the sequence of answers l_1 .. l_n (Sec. 5.3):

* Inversion(l) = sum_i (1 - l_i) * sum_{j > i} l_j, the pairs in which a false
  alarm is inspected before a true one;
* Rank-100%-T and Rank-90%-T, the interactions needed to find all, and 90%, of
  the true alarms.

Every BP step runs in the library's kernels; this module only chooses the next
alarm and counts.
"""
from __future__ import annotations

import math
import time

import numpy as np


def inversions(labels) -> int:
    """sum_i (1 - l_i) * (number of true alarms inspected after i)."""
    lab = np.asarray(labels, dtype=np.int64)
    after = np.concatenate([np.cumsum(lab[::-1])[::-1][1:], [0]])  # true alarms after each position
    return int(((1 - lab) * after).sum())


def rank_t(labels, frac: float) -> int:
    """Interactions until ceil(frac * #true) true alarms have been found (0 when
    there are no true alarms)."""
    lab = np.asarray(labels, dtype=np.int64)
    need = math.ceil(frac * int(lab.sum()) - 1e-9)
    if need <= 0:
        return 0
    return int(np.searchsorted(np.cumsum(lab), need) + 1)


def next_alarm(p1: np.ndarray, alarms: np.ndarray, inspected: np.ndarray) -> int:
    """Index (into alarms) of the uninspected alarm with the highest P(x = 1);
    ties go to the earlier alarm in the list."""
    score = np.where(inspected, -np.inf, p1[alarms].astype(np.float64))
    return int(np.argmax(score))


def run_loop(graph, alarms, truth, max_iters: int, tol: float, steps: int | None = None,
             record: bool = False) -> dict:
    """The loop on a library graph handle (fbp.Graph: marginals, set_evidence,
    run) whose messages already hold the run before the first question.
    Returns the inspection order, the answers, BP iterations per interaction,
    the host wall time per interaction and the three quality measures; with
    record, also the alarms' marginals before each question."""
    alarms = np.asarray(alarms, np.int64)
    truth = np.asarray(truth, np.int8)
    n = alarms.size if steps is None else min(steps, alarms.size)
    inspected = np.zeros(alarms.size, bool)
    order, answers, iters, wall, seen = [], [], [], [], []
    launches = updates = 0
    device_ms = 0.0
    for _ in range(n):
        t0 = time.perf_counter()
        p1 = graph.marginals()
        if record:
            seen.append(np.asarray(p1[alarms], np.float64).copy())
        k = next_alarm(p1, alarms, inspected)
        inspected[k] = True
        graph.set_evidence(int(alarms[k]), int(truth[k]))
        status, it, res = graph.run(max_iters, tol)
        wall.append(time.perf_counter() - t0)
        if hasattr(graph, "stats"):
            st = graph.stats()
            launches += int(st["kernel_launches"])
            updates += int(st["updates"])
            device_ms += float(st["run_ms"])
        order.append(int(alarms[k]))
        answers.append(int(truth[k]))
        iters.append(int(it))
    out = dict(order=order, labels=answers, iters=iters, seconds=wall, launches=launches, updates=updates,
               device_ms=device_ms,
               inversions=inversions(answers), rank100=rank_t(answers, 1.0), rank90=rank_t(answers, 0.9))
    if record:
        out["p_alarms"] = seen
    return out
