"""Served form (include/fbp_serve.h) through the C ABI.

A request clamps one variable of a resident session and re-runs from the
session's stored messages.  Its result must be the same in the mix (many
sessions, requests overlapping on the device, fewer slots than sessions) as
alone (a server holding only that session), and the same as the plain path
(fbp_set_evidence then fbp_run on a graph that saw the same requests); the
bound is the parity tolerance, 1e-5, and bit-identical results are expected.
Static-strategy sessions are also compared with the FP64 oracle.
"""
import re

import numpy as np
import pytest

from oracle import oracle as O
from paper_2509_22337_gb300 import gen

pytestmark = pytest.mark.gpu
TOL_P = 1e-5
MAX_IT = {"PARALL": 30, "TOPO_FB": 40}
TOL = 1e-6


def sessions():
    gs = [gen.bingo(n_tuples=1500 + 700 * i, seed=700 + i) for i in range(4)]
    gs += [gen.smartfl(n_layers=10, width=60, seed=710 + i, planted=True) for i in range(2)]
    return gs, ["PARALL"] * 4 + ["TOPO_FB"] * 2


def request_lists(gs, n_per, seed):
    rng = np.random.default_rng(seed)
    out = []
    for g in gs:
        free = np.flatnonzero(np.asarray(g.evidence) < 0)
        vars_ = rng.choice(free, size=n_per, replace=False)
        out.append([(int(v), int(rng.integers(0, 2))) for v in vars_])
    return out


def serve(S, gs, strats, reqs, which, max_inflight=4, iters_per_tick=8):
    srv = S.Server(max_inflight=max_inflight, iters_per_tick=iters_per_tick)
    sid = {i: srv.open(gs[i], strats[i], MAX_IT[strats[i]], TOL) for i in which}
    tickets = []
    for k in range(max(len(reqs[i]) for i in which)):  # interleaved across sessions
        for i in which:
            if k < len(reqs[i]):
                v, x = reqs[i][k]
                tickets.append((i, k, srv.submit(sid[i], v, x)))
    out = {}
    for i, k, t in tickets:
        info, p = srv.wait(t)
        assert info["state"] == S.FBP_REQ_DONE, info
        out[(i, k)] = (info, p.copy())
    st = srv.stats()
    srv.close()
    return out, st


def plain(fbp, g, strategy, reqs, max_iters=None):
    max_iters = MAX_IT[strategy] if max_iters is None else max_iters
    G = fbp.Graph(g, strategy)
    G.run(max_iters, TOL)
    out = []
    for v, x in reqs:
        G.set_evidence(v, x)
        status, it, res = G.run(max_iters, TOL)
        out.append((status, it, G.marginals().copy()))
    G.close()
    return out


def test_same_alone_in_the_mix_and_on_the_plain_path(fbp):
    from paper_2509_22337_gb300 import fbp_serve as S
    gs, strats = sessions()
    reqs = request_lists(gs, 5, seed=720)
    mix, st = serve(S, gs, strats, reqs, range(len(gs)))
    assert st["completed"] == sum(len(r) for r in reqs) and st["failed"] == 0
    assert st["peak_inflight"] > 1  # requests of several sessions ran at once
    worst_alone = worst_plain = 0.0
    for i in range(len(gs)):
        alone, _ = serve(S, gs, strats, reqs, [i])
        ref = plain(fbp, gs[i], strats[i], reqs[i])
        for k in range(len(reqs[i])):
            info, p = mix[(i, k)]
            ai, ap = alone[(i, k)]
            assert info["iters"] == ai["iters"] == ref[k][1], (i, k)
            assert info["status"] == ai["status"] == ref[k][0], (i, k)
            worst_alone = max(worst_alone, float(np.abs(p - ap).max()))
            worst_plain = max(worst_plain, float(np.abs(p - ref[k][2]).max()))
    print(f"max |mix - alone| = {worst_alone:.3e}, max |mix - plain| = {worst_plain:.3e}")
    assert worst_alone <= TOL_P and worst_plain <= TOL_P


def test_static_sessions_match_oracle(fbp):
    from paper_2509_22337_gb300 import fbp_serve as S
    gs, strats = sessions()
    idx = [i for i, s in enumerate(strats) if s != "PARALL"]
    reqs = request_lists(gs, 4, seed=721)
    mix, _ = serve(S, gs, strats, reqs, idx, max_inflight=2)
    for i in idx:
        o = O.Oracle(gs[i])
        r = o.run(strats[i], MAX_IT[strats[i]], TOL)
        for k, (v, x) in enumerate(reqs[i]):
            o.set_evidence(v, x)
            r = o.run(strats[i], MAX_IT[strats[i]], TOL, a2v=r["a2v"], history=True)
            if r["min_pos"] < 1e-36:
                print(f"session {i} request {k}: FP64 run leaves FP32 range, not compared")
                continue
            info, p = mix[(i, k)]
            err = np.abs(p - o.marginals(r["a2v"])).max()
            assert err <= TOL_P, (i, k, err)
            assert abs(info["iters"] - r["iters"]) <= 1, (i, k, info["iters"], r["iters"])


def _estimate(S, g, strategy):
    """The server's size estimate for g, read from its refusal with a 1-byte budget."""
    srv = S.Server(hbm_budget_bytes=1)
    with pytest.raises(Exception) as e:
        srv.open(g, strategy, 10, TOL)
    srv.close()
    return int(re.search(r"needs about (\d+) bytes", str(e.value)).group(1))


def test_admission_under_hbm_budget(fbp):
    from paper_2509_22337_gb300 import fbp_serve as S
    gs = [gen.bingo(n_tuples=2000, seed=730 + i) for i in range(3)]
    probe = S.Server()
    probe.open(gs[0], "PARALL", 20, TOL)
    probe.open(gs[1], "PARALL", 20, TOL)
    two = probe.stats()["resident_bytes"]  # actual device bytes of the first two sessions
    probe.close()
    budget = two + _estimate(S, gs[2], "PARALL") - 1  # the third fits only once one of them closes
    srv = S.Server(hbm_budget_bytes=budget, max_inflight=8, iters_per_tick=8)
    s0 = srv.open(gs[0], "PARALL", 20, TOL)
    s1 = srv.open(gs[1], "PARALL", 20, TOL)
    s2 = srv.open(gs[2], "PARALL", 20, TOL)  # returns at once: waits for memory
    st = srv.stats()
    assert st["sessions_resident"] == 2 and st["sessions_waiting"] == 1
    free2 = int(np.flatnonzero(np.asarray(gs[2].evidence) < 0)[0])
    t2 = srv.submit(s2, free2, 1)
    t0 = srv.submit(s0, int(np.flatnonzero(np.asarray(gs[0].evidence) < 0)[0]), 0)
    srv.wait(t0)
    assert srv.poll(t2)["state"] == S.FBP_REQ_QUEUED  # its session is not loaded yet
    srv.close_session(s0)  # frees memory: session 2 loads and its request runs
    info, p = srv.wait(t2)
    assert info["state"] == S.FBP_REQ_DONE
    st = srv.stats()
    assert st["peak_resident_bytes"] <= budget and st["sessions_resident"] == 2
    ref = plain(fbp, gs[2], "PARALL", [(free2, 1)], max_iters=20)
    assert info["iters"] == ref[0][1] and np.abs(p - ref[0][2]).max() <= TOL_P
    srv.close_session(s1)
    srv.close()


def test_device_result_and_bad_requests(fbp):
    import torch
    from paper_2509_22337_gb300 import fbp_serve as S
    g = gen.bingo(n_tuples=1200, seed=740)
    srv = S.Server()
    sid = srv.open(g, "PARALL", MAX_IT["PARALL"], TOL)
    v = int(np.flatnonzero(np.asarray(g.evidence) < 0)[3])
    out = torch.full((g.n_vars,), -1.0, device="cuda")
    info, _ = srv.wait(srv.submit(sid, v, 1, result=out))
    ref = plain(fbp, g, "PARALL", [(v, 1)])
    assert info["iters"] == ref[0][1]
    assert np.abs(out.cpu().numpy() - ref[0][2]).max() <= TOL_P
    for bad in [(sid + 5, v, 1), (sid, g.n_vars, 1), (sid, -1, 1), (sid, v, 2)]:
        with pytest.raises(fbp.FbpError) as e:
            srv.submit(*bad)
        assert e.value.code == fbp.FBP_ERR_INVALID_ARG
    with pytest.raises(fbp.FbpError):
        srv.open(g, "RESIDUAL", 10, TOL)
    srv.close()


def test_destroy_with_queued_requests_returns(fbp):
    from paper_2509_22337_gb300 import fbp_serve as S
    g = gen.bingo(n_tuples=3000, seed=750)
    srv = S.Server(max_inflight=1)
    sid = srv.open(g, "PARALL", 200, TOL)
    free = np.flatnonzero(np.asarray(g.evidence) < 0)
    for k in range(20):
        srv.submit(sid, int(free[k]), k & 1)
    srv.close()  # running request finishes, queued ones fail, nothing hangs
