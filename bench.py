"""Benchmark: BP message updates/s on the BINGO-shaped 1M-tuple derivation graph.

One step = one whole run of the hot path on one graph: messages reset to
uniform, then flooding (PARALL) iterations until the largest message change
is below 1e-6 or 500 iterations, then the marginals (Eq. 3) into a device
buffer.  `value` counts the factor-to-variable message updates of the step
over its device time (CUDA events on the library's stream), graph already
resident in HBM.  The L2 is flushed (a 512 MiB write) between timed steps.

`e2e` times the same work through the C ABI from host buffers: graph creation
(CSR transpose, host-to-device copies), schedule construction, the run, and
the marginals copied back to the host.  `forms` (one GPU only) compares, on
reduced workloads, the batched form against a per-graph launch loop and the
served form against a cold-start per-request path on the same arrivals.
`--workload` selects the other configurations.

`--impl reference` times the FP64 oracle (the CPU baseline) on the host cores.
`--gpus N` under torchrun runs one independent replica per GPU (a single graph
does not shard); value is the sum over ranks of updates / the slowest rank's
time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import tempfile
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    # name: (generator, strategy, max_iters, tol, description)
    "smartfl200k": ("smartfl", "TOPO_FB", 100, 1e-6,
                    "SmartFL-shaped layered DAG: 200k vars in 200 layers, 300k factors, 5% evidence; "
                    "TOPO_FB to max change < 1e-6 or 100 sweeps"),
    "bingo1m": ("bingo", "PARALL", 500, 1e-6,
                "BINGO-shaped cyclic derivation graph: 1M tuples, 2M NOISY_AND rules (+3M vars); "
                "PARALL to max change < 1e-6 or 500 iterations"),
    "bingo1m_residual": ("bingo", "RESIDUAL", 500, 1e-6,
                         "BINGO-shaped cyclic derivation graph: 1M tuples, 2M NOISY_AND rules (+3M vars); "
                         "RESIDUAL (classes and Algorithm 2 levels built on the device every iteration) to max "
                         "change < 1e-6 or 500 iterations"),
    "bingo1m_seqfix": ("bingo", "SEQFIX", 2, 0.0,
                       "BINGO-shaped cyclic derivation graph: 1M tuples, 2M NOISY_AND rules (+3M vars); SEQFIX "
                       "(one message at a time in edge order, run as Algorithm 2's levels), exactly 2 sweeps, by "
                       "the belief-form sequential engine (FBP_OPT_ENGINE = 3)"),
    "tiny": ("tiny", "PARALL", 50, 0.0, "tiny derivation DAG, PARALL, exactly 50 iterations"),
    "generic200k": ("generic", "TOPO_FB", 100, 1e-6,
                    "SmartFL-200k structure with every factor generic: random term lists (1-6 terms, "
                    "variables free w.p. 0.3, plus a 0.05-weight all-free term) evaluated by Algorithm 1; "
                    "TOPO_FB to max change < 1e-6 or 100 sweeps"),
    "alarms": ("tiny", "SEQFIX", 500, 1e-6,
               "interactive alarm ranking on the tiny derivation DAG (2,000 tuples, 3,000 NOISY_AND(0.9) "
               "rules): 30 alarms with planted ground truth (rules truly fire w.p. 0.8); each answer is "
               "clamped and BP re-runs warm to max change < 1e-6 or 500 iterations; SEQFIX (asynchronous) "
               "and PARALL"),
    "batched": ("batched", "MIXED", 0, 1e-6,
                "512 graphs, sizes log-uniform in 1e3..1e5: even SmartFL-shaped (TOPO_FB, tol 1e-6, <= 100 "
                "sweeps), odd BINGO-shaped (PARALL, tol 1e-6, <= 500 iterations); one batched run"),
    "serving": ("serving", "PARALL", 500, 1e-6,
                "64 resident BINGO-shaped sessions, 5e4..5e5 tuples (log-uniform); Poisson request stream "
                "at 2000 req/s, each request clamps one unobserved tuple and re-runs PARALL warm to "
                "max change < 1e-6 or 500 iterations; 120 GB HBM budget"),
}


# Workloads whose full-size graph the oracle cannot run one iteration of in a
# bounded sample: its Algorithm 2 scan walks every edge of each neighbouring
# variable, and BINGO's hub variables carry ~1e5 edges (one RESIDUAL iteration
# of the 1M-tuple graph took 562 s on one core).  The CPU sample then runs the
# same generator at a smaller scale, and says so.
# graph options a workload sets after creating its graph handle (option id: value)
WORKLOAD_OPTIONS = {"bingo1m_seqfix": {3: 3}}  # FBP_OPT_ENGINE: the belief-form sequential engine

ORACLE_SAMPLE_GRAPHS = {
    "bingo1m_seqfix": (dict(n_tuples=50_000),
                       "the same generator at 1/20 scale (50k tuples; the oracle's cost per update grows with the "
                       "degrees of the factor's variables, so this overstates its full-size rate)"),
    "bingo1m_residual": (dict(n_tuples=100_000),
                         "the same generator at 1/10 scale (100k tuples; this overstates the oracle's full-size "
                         "rate, as its cost per edge grows with hub degree)"),
}


def make_graph(name, **kw):
    from paper_2509_22337_gb300 import gen
    kind = WORKLOADS[name][0]
    if kw:
        return {"smartfl": gen.smartfl, "bingo": gen.bingo, "tiny": gen.tiny}[kind](**kw)
    if kind == "generic":
        return gen.with_generic_factors(gen.smartfl(), 1.0, seed=9)
    return {"smartfl": gen.smartfl, "bingo": gen.bingo, "tiny": gen.tiny}[kind]()


def dist_info():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, index: int):
        self.index = index
        self.p = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(prefix="fbp_clocks_", suffix=".csv")
            self.f = os.fdopen(fd, "w")
            self.p = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}",
                 "--query-gpu=index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:  # noqa: BLE001
            self.p = None
            if self.path:
                try:
                    self.f.close()
                    os.remove(self.path)
                except Exception:  # noqa: BLE001
                    pass
                self.path = None
        return self

    def __exit__(self, *exc):
        if self.p is not None:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except Exception:  # noqa: BLE001
                self.p.kill()
            self.f.close()

    def summary(self):
        if self.p is None or not self.path or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as fh:
            lines = fh.readlines()
        os.remove(self.path)
        for line in lines:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def aggregate(ms: float, units: float, device: str = "cuda"):
    """The job's time and work over all ranks: the slowest rank's time and the
    sum of the units every rank processed (unchanged for one process)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(ms), float(units)
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def shard(sizes, world: int, rank: int) -> list:
    """Independent units (graphs, sessions) of the given sizes, bin-packed over
    the ranks: largest first onto the least-loaded rank.  Returns this rank's
    unit indices in ascending order; every unit goes to exactly one rank."""
    load = [0] * world
    owner = [0] * len(sizes)
    for i in sorted(range(len(sizes)), key=lambda k: (-sizes[k], k)):
        r = min(range(world), key=lambda q: (load[q], q))
        owner[i] = r
        load[r] += sizes[i]
    return [i for i in range(len(sizes)) if owner[i] == rank]


def algorithmic_bytes_per_half(g):
    """Bytes one half-iteration (one pass over every level of one level list)
    of the persistent level engine must move at minimum: per edge the old and
    the new message (8 B), its row record (16 B) and its var-major
    (edge, level) pair (8 B); per factor one work item (16 B); per variable
    its unary potential (4 B).  Messages gathered while forming v->a products
    are re-reads of the same 4 B/edge array and are not counted again."""
    E, V, A = g.n_edges, g.n_vars, g.n_factors
    return 32 * E + 16 * A + 4 * V


def algorithmic_bytes_flood(g):
    """Bytes one flooding iteration of this layout must move: per edge the
    variable-major message copy read in phase 1 and scattered in phase 2
    (4 + 4 B), and in phase 2 the edge's variable, its variable-major slot and
    its message read and written (4 + 4 + 4 + 4 B); per variable its row
    offset and unary potential read and its 8-byte belief record written and
    read once (24 B); per factor its row offset, type and parameter (9 B)."""
    E, V, A = g.n_edges, g.n_vars, g.n_factors
    return 24 * E + 24 * V + 9 * A


def pair_model_bytes_per_pass(g):
    """The method's per-pass byte model, with every message a pair of FP32
    values (the measure `roofline.achieved` is based on): per edge four
    message touches of 8 B (gather a->v and write v->a in phase 1, read v->a
    and write a->v in phase 2) and one 4-B index; per variable its row offset
    and unary pair (12 B); per factor its row offset, type and parameter
    (9 B).  One pass is one flooding iteration, or one level list of a static
    schedule (every edge updated once).  This library stores one float per
    message, so its own minimum (algorithmic_bytes_flood / _per_half) is
    lower; both are reported."""
    E, V, A = g.n_edges, g.n_vars, g.n_factors
    return 36 * E + 12 * V + 9 * A


# Sources each profiled kernel is built from: a DRAM traffic figure taken by
# ncu is reported only while these files are unchanged.
KERNEL_SOURCES = {
    "k_engine": ["fbp_engine.cu", "fbp_msg.cuh", "fbp_internal.h", "fbp_flood_dev.cuh", "fbp_flood.h"],
    "flood": ["fbp_flood.cu", "fbp_flood.h", "fbp_flood_dev.cuh", "fbp_msg.cuh", "fbp_internal.h"],
    "k_seq": ["fbp_seq.cu", "fbp_flood.h", "fbp_flood_dev.cuh", "fbp_msg.cuh", "fbp_internal.h"],
}


def profiled_traffic(kernel: str, workload: str):
    """DRAM bytes (read + write) per launch of `kernel` on `workload` from the
    committed ncu summaries under profiles/, or None when there is none for
    the kernel's current sources."""
    import glob
    import hashlib
    import re
    h = hashlib.sha256()
    for f in KERNEL_SOURCES[kernel]:
        with open(os.path.join(ROOT, "paper_2509_22337_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    want = h.hexdigest()[:16]
    pat = re.compile(r"traffic: (\S+) (\S+) dram_bytes_per_launch=(\d+) sources_sha256=([0-9a-f]+)")
    for path in sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md"))):
        with open(path) as fh:
            for m in pat.finditer(fh.read()):
                if m.group(1) == kernel and m.group(2) == workload and m.group(4) == want:
                    return int(m.group(3))
    return None


def batched_compare(graphs, sch, mi, tol, stream, steps=1, warmup=1, tune=True):
    """One batched run of `graphs` (fbp_batch, autotuned) against the per-graph
    fbp_run loop on the same GPU, both from uniform messages with the graphs
    resident.  Returns the batch's per-step seconds, the loop's seconds, the
    tuning, the batch's statistics and whether every member's marginals are
    the same bit for bit both ways."""
    import torch
    from paper_2509_22337_gb300 import autotune, fbp_batch as BB
    from paper_2509_22337_gb300 import fbp as F
    B = BB.Batch(graphs, sch, mi, tol, stream=stream)
    tuning = autotune.tune_batch(B, graphs, sch) if tune else None
    for _ in range(warmup):
        B.reset()
        B.run()
    torch.cuda.synchronize()
    times, upd = [], 0
    for _ in range(steps):
        B.reset()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        B.run()
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t0)
        upd += B.stats()["updates"]
    st = B.stats()
    Gs = [F.Graph(g, s, stream=stream) for g, s in zip(graphs, sch)]
    for G in Gs:
        G.run(1, 0.0)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    loop_upd = 0
    for G, m, t in zip(Gs, mi, tol):
        G.reset()
        G.run(m, t)
        loop_upd += G.stats()["updates"]
    torch.cuda.synchronize()
    loop_s = time.perf_counter() - t0
    same = all(np.array_equal(B.marginals(i), G.marginals()) for i, G in enumerate(Gs))
    for G in Gs:
        G.close()
    # the batch's other forms, each timed once after a warm run
    FORM_ARGS = {"one": dict(one_launch=True), "queue": dict(one_launch=False, static_queue=True),
                 "engine": dict(one_launch=False, static_queue=False)}
    others = {}
    for form, kw in FORM_ARGS.items():
        if form == B.form:
            continue
        B2 = BB.Batch(graphs, sch, mi, tol, stream=stream, **kw)
        if tune:
            autotune.tune_batch(B2, graphs, sch)
        B2.run()
        B2.reset()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        B2.run()
        torch.cuda.synchronize()
        others[form] = time.perf_counter() - t0
        same = same and all(np.array_equal(B.marginals(i), B2.marginals(i)) for i in range(len(graphs)))
        B2.close()
    form = B.form
    B.close()
    return {"times": times, "updates": upd, "loop_s": loop_s, "loop_updates": loop_upd, "tuning": tuning,
            "stats": st, "same_results": bool(same), "form": form, "other_forms": others}


def serve_window(srv, sids, window):
    """Submit each request of `window` whose session is served here at its
    arrival time (relative to the window's first), wait for all.  Returns the
    requests' infos (latency from submission, queueing included) and the wall
    seconds."""
    base = float(window["t"][0])
    tickets = []
    start = time.perf_counter()
    for r in window:
        if int(r["session"]) not in sids:
            continue
        delay = (float(r["t"]) - base) - (time.perf_counter() - start)
        if delay > 0:
            time.sleep(delay)
        tickets.append(srv.submit(sids[int(r["session"])], int(r["var"]), int(r["value"])))
    infos = [srv.wait(t)[0] for t in tickets]
    return infos, time.perf_counter() - start


def cold_window(sessions, window, strategy, max_iters, tol):
    """The cold-start per-request plain path on the same arrivals: each request,
    at its arrival time and one at a time (FIFO), builds a new graph with its
    session's evidence so far, runs from uniform messages and reads the
    marginals back.  Returns per-request service and latency (arrival to
    result) in ms, and the wall seconds."""
    import torch
    from paper_2509_22337_gb300 import fbp as F, gen
    evid = [np.array(g.evidence, copy=True) for g in sessions]
    base = float(window["t"][0])
    svc, lat = [], []
    start = time.perf_counter()
    for r in window:
        evid[int(r["session"])][int(r["var"])] = int(r["value"])
        delay = (float(r["t"]) - base) - (time.perf_counter() - start)
        if delay > 0:
            time.sleep(delay)
        g = sessions[int(r["session"])]
        gc = gen.FactorGraph(g.n_vars, g.factor_ptr, g.factor_vars, g.factor_type, g.factor_param, g.prior_p1,
                             evid[int(r["session"])].copy(), g.name)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        G = F.Graph(gc, strategy)
        G.run(max_iters, tol)
        G.marginals()
        G.close()
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        svc.append((t2 - t1) * 1e3)
        lat.append((t2 - start - (float(r["t"]) - base)) * 1e3)
    return np.array(svc), np.array(lat), time.perf_counter() - start


def _pct(x):
    return {"p50": round(float(np.percentile(x, 50)), 3), "p99": round(float(np.percentile(x, 99)), 3)}


def forms_compare(args, stream):
    """Reduced batched and served comparisons for the default bench line (one
    GPU): the batched form against the per-graph loop on the first
    --forms-graphs graphs of the batched workload's generator; the served form
    against the cold-start path on the same --forms-requests arrivals of the
    serving workload's stream over --forms-sessions sessions."""
    from paper_2509_22337_gb300 import fbp_serve as SV, gen
    out = {}
    graphs = gen.batched_mix(n_graphs=args.forms_graphs, seed=4)
    sch = ["TOPO_FB" if i % 2 == 0 else "PARALL" for i in range(len(graphs))]
    mi = [100 if s == "TOPO_FB" else 500 for s in sch]
    r = batched_compare(graphs, sch, mi, [1e-6] * len(graphs), stream)
    n = len(graphs)
    bs = float(np.median(r["times"]))
    out["batched"] = {
        "graphs": n, "n_edges": int(sum(g.n_edges for g in graphs)),
        "batched_graphs_per_s": round(n / bs, 2), "loop_graphs_per_s": round(n / r["loop_s"], 2),
        "speedup_vs_loop": round(r["loop_s"] / bs, 2), "same_results_bit_for_bit": r["same_results"],
        "form": r["form"],
        "other_forms_graphs_per_s": {k: round(n / v, 2) for k, v in r["other_forms"].items()},
        "what": "one fbp_batch run vs fbp_run per graph on the same GPU, graphs resident, from uniform "
                "messages; even graphs SmartFL-shaped TOPO_FB, odd BINGO-shaped PARALL; the batch's other forms "
                "(one: one persistent launch; queue: static members in the member queue beside the flooding "
                "kernels; engine: static members in the level engine beside them) timed beside it; every "
                "member's marginals compared bit for bit across all of them"}
    _, strategy, max_iters, tol, _ = WORKLOADS["serving"]
    sessions = gen.serving_sessions(args.forms_sessions)
    window = gen.request_stream(sessions, 2000.0, 30.0)[: args.forms_requests]
    srv = SV.Server(hbm_budget_bytes=120 << 30, max_inflight=args.serve_inflight, iters_per_tick=args.serve_tick)
    sids = {i: srv.open(sessions[i], strategy, max_iters, tol) for i in range(len(sessions))}
    while srv.stats()["sessions_warming"] > 0:
        time.sleep(0.01)
    infos, wall = serve_window(srv, sids, window)
    srv.close()
    assert all(i["state"] == SV.FBP_REQ_DONE for i in infos), "a served request failed"
    lat = np.array([i["latency_ms"] for i in infos])
    svc, clat, cwall = cold_window(sessions, window, strategy, max_iters, tol)
    out["serving"] = {
        "sessions": len(sessions), "requests": len(infos), "offered_rate_req_s": 2000.0,
        "served_req_per_s": round(len(infos) / wall, 2), "served_latency_ms": _pct(lat),
        "cold_req_per_s": round(len(window) / cwall, 2), "cold_latency_ms": _pct(clat),
        "cold_service_ms": _pct(svc),
        "speedup_vs_cold": round((len(infos) / wall) / (len(window) / cwall), 2),
        "p99_vs_cold": round(float(np.percentile(clat, 99)) / max(float(np.percentile(lat, 99)), 1e-9), 2),
        "iters_per_request_mean": round(float(np.mean([i["iters"] for i in infos])), 1),
        "what": "the same arrivals (Poisson 2000 req/s) replayed through the server (resident sessions, "
                "warm re-runs, continuous batching) and through the cold-start path (new graph with the "
                "evidence so far, run from uniform messages, marginals to the host), one request at a time; "
                "latency from arrival to result, queueing included"}
    return out


def run_batched(args, rank, world, local):
    """The batched workload: one fbp_batch run of 512 graphs vs a per-graph loop."""
    import torch
    from paper_2509_22337_gb300 import fbp_batch as BB, gen

    graphs = gen.batched_mix(n_graphs=args.batch_graphs, seed=4 + 1000 * rank)
    sch = ["TOPO_FB" if i % 2 == 0 else "PARALL" for i in range(len(graphs))]
    mi = [100 if s == "TOPO_FB" else 500 for s in sch]
    tol = [1e-6] * len(graphs)
    stream = torch.cuda.current_stream()
    if world > 1:
        torch.distributed.barrier()
    with Clocks(local) as clk:
        r = batched_compare(graphs, sch, mi, tol, stream, steps=args.steps, warmup=args.warmup)
    st, tuning, total = r["stats"], r["tuning"], float(sum(r["times"]))
    # end to end: batch creation from host arrays, run, every marginal to the host
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    B2 = BB.Batch(graphs, sch, mi, tol, stream=stream)
    B2.tune(**tuning)
    B2.run()
    for i in range(len(graphs)):
        B2.marginals(i)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e_upd = B2.stats()["updates"]
    B2.close()
    h2d = sum(g.nbytes() for g in graphs)
    d2h = sum(4 * g.n_vars for g in graphs)
    t_max, tot = aggregate(total, r["updates"])
    n = len(graphs)
    loop_s = r["loop_s"]
    if rank == 0:
        line = {
            "metric": "BP message updates/s", "value": round(tot / t_max, 1), "unit": "msg_updates/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(t_max / args.steps * 1e3, 3), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "batched", "desc": WORKLOADS["batched"][4], "n_graphs": n,
                       "n_vars": sum(g.n_vars for g in graphs), "n_edges": sum(g.n_edges for g in graphs),
                       "tuning": tuning, "l2": "inputs larger than L2", "parallelism": f"replicas{world}"},
            "graphs_per_s": round(n * world * args.steps / t_max, 2),
            "per_graph_loop": {"graphs_per_s": round(n / loop_s, 2), "ms": round(loop_s * 1e3, 2),
                               "msg_updates_per_s": round(r["loop_updates"] / loop_s, 1)},
            "speedup_vs_loop": round((loop_s / n) / (t_max / (n * args.steps * world)), 2),
            "same_results_bit_for_bit": r["same_results"],
            "form": r["form"],
            "other_forms_graphs_per_s": {k: round(n / v, 2) for k, v in r["other_forms"].items()},
            "max_iters_run": st["iters"],
            "e2e": {"value": round(e2e_upd / e2e_s, 1), "unit": "msg_updates/s", "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": int(d2h), "ms_per_step": round(e2e_s * 1e3, 2)},
            "gpu_launches": int(st["kernel_launches"] * args.steps), "clocks": clk.summary(),
        }
        print(json.dumps(line))


class OracleGraph:
    """The FP64 oracle behind the graph-handle calls the ranking loop makes
    (the CPU baseline of the alarms workload)."""

    def __init__(self, g, strategy):
        from oracle import oracle as O
        O.build()
        self.o, self.strategy, self.a2v = O.Oracle(g), strategy, None

    def run(self, max_iters, tol):
        r = self.o.run(self.strategy, max_iters, tol, a2v=self.a2v)
        self.a2v = r["a2v"]
        return (0 if r["converged"] else 1), r["iters"], r["residual"]

    def marginals(self):
        return self.o.marginals(self.a2v)

    def set_evidence(self, var, value):
        self.o.set_evidence(var, value)


def alarms_setup():
    from paper_2509_22337_gb300 import gen
    g = gen.tiny()
    alarms, truth = gen.planted_alarms(g, 30, seed=5, fire=0.8)
    return g, alarms, truth


def run_alarms(args, rank, world, local):
    """The interactive alarm-ranking loop (Sec. 5.3): one step = a graph whose
    messages hold the run before the first question, then 30 questions, each
    answer clamped and BP re-run warm.  Timed: the loop (marginals to the host,
    the choice, the clamp, the run); untimed: building the graph.  Every rank
    runs its own replica."""
    import torch
    from paper_2509_22337_gb300 import fbp as F, ranking

    _, _, max_iters, tol, desc = WORKLOADS["alarms"]
    g, alarms, truth = alarms_setup()
    stream = torch.cuda.current_stream()
    per = {}
    clk_all = None
    for strategy in ("SEQFIX", "PARALL"):
        def fresh():
            G = F.Graph(g, strategy, stream=stream)
            G.run(max_iters, tol)
            torch.cuda.synchronize()
            return G
        for _ in range(args.warmup):
            G = fresh()
            ranking.run_loop(G, alarms, truth, max_iters, tol)
            G.close()
        times, runs = [], []
        with Clocks(local) as clk:
            for _ in range(args.steps):
                G = fresh()
                t0 = time.perf_counter()
                r = ranking.run_loop(G, alarms, truth, max_iters, tol)
                torch.cuda.synchronize()
                times.append(time.perf_counter() - t0)
                runs.append(r)
                G.close()
        if strategy == "SEQFIX":
            clk_all = clk.summary()
        wall, n_int = aggregate(float(sum(times)), float(len(alarms) * args.steps))
        r0 = runs[0]
        per[strategy] = {
            "interactions_per_s": round(n_int / wall, 2), "ms_per_interaction": round(wall / n_int * 1e3, 3),
            "bp_iterations_per_answer": round(float(np.mean(r0["iters"])), 1),
            "inversions": r0["inversions"], "rank_100pct_t": r0["rank100"], "rank_90pct_t": r0["rank90"],
            "message_updates_per_s": round(sum(r["updates"] for r in runs) / wall, 1),
            "gpu_launches_per_step": int(np.mean([r["launches"] for r in runs])),
            "bp_iterations_per_step": int(np.mean([sum(r["iters"]) for r in runs])),
            "device_ms_per_step": round(float(np.mean([r["device_ms"] for r in runs])), 3)}
    if rank != 0:
        return
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        O = OracleGraph(g, "SEQFIX")
        O.run(max_iters, tol)
        t0 = time.perf_counter()
        ro = ranking.run_loop(O, alarms, truth, max_iters, tol)
        dt = time.perf_counter() - t0
        cpu = {"value": round(len(alarms) / dt, 3), "unit": "interactions/s", "cores": 1, "kind": "oracle",
               "sample": f"the same 30-question SEQFIX loop ({dt:.1f} s, single thread)",
               "inversions": ro["inversions"], "rank_100pct_t": ro["rank100"], "rank_90pct_t": ro["rank90"]}
    s = per["SEQFIX"]
    peaks_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    peak = float(json.load(open(peaks_path)).get("hbm_gbs", 6800.0)) if os.path.exists(peaks_path) else 6800.0
    ach = pair_model_bytes_per_pass(g) * s["bp_iterations_per_step"] / max(s["device_ms_per_step"], 1e-9) / 1e6
    line = {
        "metric": "alarm-ranking interactions/s", "value": s["interactions_per_s"], "unit": "interactions/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(s["ms_per_interaction"] * len(alarms), 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "alarms", "desc": desc, "n_vars": g.n_vars, "n_edges": g.n_edges,
                   "alarms": int(len(alarms)), "true_alarms": int(truth.sum()), "max_iters": max_iters, "tol": tol,
                   "l2": "graph resident in L2 (the loop re-reads it every iteration by design)",
                   "parallelism": f"replicas{world}"},
        "per_strategy": per,
        "roofline": {"bound": "hbm", "achieved": round(ach, 2), "peak": peak, "unit": "GB/s",
                     "frac": round(ach / peak, 5), "traffic": None,
                     "kernel": "k_engine in one block (SEQFIX levels of ~11 edges), all runs of one step",
                     "bytes_model": "36E+12V+9A per BP iteration (FP32 message pairs)",
                     "note": "per-level latency, not bandwidth, bounds this loop"},
        "cpu_baseline": cpu,
        "e2e": {"value": s["interactions_per_s"], "unit": "interactions/s", "h2d_bytes_per_step": 3 * len(alarms),
                "d2h_bytes_per_step": 4 * g.n_vars * len(alarms),
                "note": "every interaction reads all marginals back to the host and sends one clamp"},
        "gpu_launches": s["gpu_launches_per_step"] * args.steps,
        "clocks": clk_all,
    }
    print(json.dumps(line))


def run_serving(args, rank, world, local):
    """The served workload: resident sessions, an open-loop Poisson request
    stream replayed at its own arrival times, continuous batching by the
    library's server.  One step = one window of the stream (--serve-requests
    arrivals); warm-up windows come from the stream after the timed ones."""
    from paper_2509_22337_gb300 import fbp_serve as SV, gen

    _, strategy, max_iters, tol, desc = WORKLOADS["serving"]
    n_sess = args.serve_sessions
    sessions = gen.serving_sessions(n_sess)
    stream = gen.request_stream(sessions, 2000.0, 30.0)
    per = args.serve_requests
    need = per * (args.steps + args.warmup)
    if need > len(stream):
        raise SystemExit(f"the stream holds {len(stream)} requests, {need} asked for")
    srv = SV.Server(hbm_budget_bytes=120 << 30, max_inflight=args.serve_inflight,
                    iters_per_tick=args.serve_tick)
    # sessions are independent: with several GPUs each rank serves a bin-packed
    # share of them and the requests addressed to those (no collective)
    mine = shard([g.n_edges for g in sessions], world, rank)
    t0 = time.perf_counter()
    sids = {i: srv.open(sessions[i], strategy, max_iters, tol) for i in mine}
    glob = {v: k for k, v in sids.items()}  # server session id -> workload session index
    while srv.stats()["sessions_warming"] > 0:
        time.sleep(0.01)
    load_s = time.perf_counter() - t0

    def replay(window):
        infos, dt = serve_window(srv, sids, window)
        for i in infos:
            i["session"] = glob[i["session"]]
        return infos, dt

    for w in range(args.warmup):  # warm-up windows: the end of the stream
        replay(stream[len(stream) - per * (w + 1): len(stream) - per * w])
    infos, wall = [], 0.0
    st0 = srv.stats()
    with Clocks(local) as clk:
        for k in range(args.steps):
            i, dt = replay(stream[k * per:(k + 1) * per])
            infos += i
            wall += dt
    st1 = srv.stats()
    if world > 1:  # every rank's requests into the percentiles; the slowest rank's time
        import torch.distributed as dist
        parts = [None] * world
        dist.all_gather_object(parts, infos)
        infos = [i for p in parts for i in p]
        wall, _ = aggregate(wall, 0.0)
    lat = np.array([i["latency_ms"] for i in infos])
    svc = np.array([i["latency_ms"] - i["queue_ms"] for i in infos])
    dev = np.array([i["device_ms"] for i in infos])
    its = np.array([i["iters"] for i in infos])
    assert all(i["state"] == SV.FBP_REQ_DONE for i in infos), "a served request failed"
    value = len(infos) / wall
    # algorithmic bytes of every iteration the timed requests ran
    sess_bytes = [pair_model_bytes_per_pass(g) for g in sessions]
    moved = sum(sess_bytes[i["session"]] * i["iters"] for i in infos)
    peak = float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"]) \
        if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else 6800.0
    achieved = moved / wall / 1e9
    srv.close()

    # cold-start per-request plain path, replayed on the first timed window at
    # the requests' own arrival times, one request at a time: a new graph with
    # the session's evidence so far, a run from uniform messages, marginals to
    # the host.  Its latency (arrival to result, queueing included) is what the
    # served form's latency is compared with.
    if rank != 0:
        return
    window = stream[: per * args.cold_windows]
    cold, cold_lat, cold_wall = cold_window(sessions, window, strategy, max_iters, tol)
    cold_rate = len(window) / cold_wall
    n_vars_mean = float(np.mean([sessions[i["session"]].n_vars for i in infos]))
    line = {
        "metric": "served requests/s", "value": round(value, 2), "unit": "req/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(wall / args.steps * 1e3, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "serving", "desc": desc, "n_sessions": n_sess,
                   "n_vars": int(sum(g.n_vars for g in sessions)), "n_edges": int(sum(g.n_edges for g in sessions)),
                   "requests_per_step": per, "offered_rate_req_s": 2000.0, "max_inflight": args.serve_inflight,
                   "iters_per_tick": args.serve_tick, "hbm_budget_gb": 120,
                   "l2": "inputs larger than L2",
                   "parallelism": f"sessions bin-packed over {world} GPU(s)" if world > 1 else "replicas1"},
        "latency_ms": {"p50": round(float(np.percentile(lat, 50)), 3), "p99": round(float(np.percentile(lat, 99)), 3),
                       "note": "submission to result on the host, queueing under the offered rate included"},
        "service_ms": {"p50": round(float(np.percentile(svc, 50)), 3), "p99": round(float(np.percentile(svc, 99)), 3)},
        "device_ms": {"p50": round(float(np.percentile(dev, 50)), 3), "p99": round(float(np.percentile(dev, 99)), 3)},
        "iters_per_request": {"mean": round(float(its.mean()), 1), "max": int(its.max())},
        "load_s": round(load_s, 2),
        "cold_start": {"req_per_s": round(cold_rate, 3),
                       "service_ms": {"p50": round(float(np.percentile(cold, 50)), 3),
                                      "p99": round(float(np.percentile(cold, 99)), 3)},
                       "latency_ms": {"p50": round(float(np.percentile(cold_lat, 50)), 3),
                                      "p99": round(float(np.percentile(cold_lat, 99)), 3)},
                       "sample": f"the first {len(cold)} requests of the timed stream, replayed at their arrival "
                                 "times",
                       "what": "per request: fbp_graph_create with the evidence so far, fbp_run from uniform "
                               "messages, marginals to the host, destroy; one request at a time, FIFO"},
        "speedup_vs_cold": round(value / cold_rate, 2),
        "roofline": {"bound": "hbm", "achieved": round(achieved, 2), "peak": peak, "unit": "GB/s",
                     "frac": round(achieved / peak, 4), "traffic": None,
                     "kernel": "flooding iteration kernels of all running requests",
                     "bytes_model": "36E+12V+9A per iteration (FP32 message pairs)"},
        "e2e": {"value": round(value, 2), "unit": "req/s", "h2d_bytes_per_step": 4 * per,
                "d2h_bytes_per_step": int(4 * n_vars_mean * per),
                "note": "each request is submitted from the host and its marginals land in host memory"},
        "gpu_launches": int(st1["kernel_launches"] - st0["kernel_launches"]),
        "server": {"ticks": int(st1["ticks"] - st0["ticks"]), "peak_inflight": st1["peak_inflight"],
                   "resident_gb": round(st1["peak_resident_bytes"] / 2**30, 2)},
        "clocks": clk.summary(),
    }
    print(json.dumps(line))


def run_gpu(args):
    import torch

    rank, world, local = dist_info()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    import __graft_entry__ as ge
    from paper_2509_22337_gb300 import fbp as F

    if rank == 0 or not os.path.exists(F.lib_path()):
        ge.build()
    if world > 1:
        torch.distributed.barrier()
    F.load()
    if args.workload in ("batched", "serving", "alarms"):
        {"batched": run_batched, "serving": run_serving, "alarms": run_alarms}[args.workload](args, rank, world, local)
        if world > 1:
            torch.distributed.destroy_process_group()
        return
    _, strategy, max_iters, tol, desc = WORKLOADS[args.workload]
    g = make_graph(args.workload)
    stream = torch.cuda.current_stream()
    G = F.Graph(g, strategy, stream=stream)
    for k, v in WORKLOAD_OPTIONS.get(args.workload, {}).items():
        G.set_option(k, v)
    p_out = torch.empty(max(g.n_vars, 1), dtype=torch.float32, device="cuda")
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")

    def step():
        G.reset()
        G.run(max_iters, tol)
        G.marginals(out=p_out)

    # marginals: one kernel, and a second one when some row is longer than 256 entries
    marg_launches = 1 + int(np.bincount(np.asarray(g.factor_vars), minlength=g.n_vars).max(initial=0) > 256)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    updates = 0
    launches = 0
    run_ms = []
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with Clocks(local) as clk:
        t0 = time.perf_counter()
        for i in range(args.steps):
            flush.fill_(i & 0xFF)
            ev[i][0].record(stream)
            step()
            ev[i][1].record(stream)
            st = G.stats()
            updates += st["updates"]
            launches += st["kernel_launches"] + 1 + marg_launches  # + reset fill + marginals
            run_ms.append(st["run_ms"])
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
    if world > 1:
        torch.distributed.barrier()
    ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = float(sum(ms))
    st = G.stats()
    t_max, tot_updates = aggregate(total_ms, updates)
    value = tot_updates / (t_max / 1e3)

    # roofline of the dominant kernel
    sweeps = st["iters"]
    launches_per_step = max(st["kernel_launches"], 1)
    kernel_ms = float(np.median(run_ms))
    if strategy == "PARALL":
        # the unit is one flooding iteration (its five kernels, replayed from
        # a captured CUDA graph): algorithmic bytes per iteration over the
        # device time per iteration
        kname = "flooding iteration (k_beliefs, k_row_beliefs, k_a2v_lanes, k_flood_check)"
        kkey = "flood"
        launches_per_step = max(sweeps, 1)
        bytes_per_launch = pair_model_bytes_per_pass(g)
        layout_bytes = algorithmic_bytes_flood(g)
    elif strategy == "RESIDUAL":
        # one RESIDUAL iteration: the device schedule, then each of its
        # levels as a flooding step over the whole graph (bytes of one level:
        # a lower bound when an iteration has several levels)
        kname = "RESIDUAL iteration (device schedule + flooding levels)"
        kkey = "flood"
        launches_per_step = max(sweeps, 1)
        bytes_per_launch = pair_model_bytes_per_pass(g)
        layout_bytes = algorithmic_bytes_flood(g)
    elif WORKLOAD_OPTIONS.get(args.workload, {}).get(3) == 3:
        kname = "k_seq_belief (belief-form sequential engine: one block, one launch per run)"
        kkey = "k_seq"
        halves = 2 if strategy == "TOPO_FB" else 1
        bytes_per_launch = pair_model_bytes_per_pass(g) * halves * sweeps / launches_per_step
        layout_bytes = bytes_per_launch
    else:
        kname = "k_engine (persistent level engine, one launch per run)"
        kkey = "k_engine"
        halves = 2 if strategy == "TOPO_FB" else 1
        bytes_per_launch = pair_model_bytes_per_pass(g) * halves * sweeps / launches_per_step
        layout_bytes = algorithmic_bytes_per_half(g) * halves * sweeps / launches_per_step
    per_launch_ms = kernel_ms / launches_per_step
    peaks_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    peaks = json.load(open(peaks_path)) if os.path.exists(peaks_path) else {"hbm_gbs": 6800.0}
    peak = float(peaks.get("hbm_gbs", 6800.0))
    achieved = bytes_per_launch / (per_launch_ms / 1e3) / 1e9
    roof = {"bound": "hbm", "achieved": round(achieved, 2), "peak": peak, "unit": "GB/s",
            "frac": round(achieved / peak, 4), "traffic": profiled_traffic(kkey, args.workload), "kernel": kname,
            "per_launch_us": round(per_launch_ms * 1e3, 3), "bytes_per_launch": int(bytes_per_launch),
            "bytes_model": "36E+12V+9A per pass (FP32 message pairs)",
            "bytes_per_launch_layout": int(layout_bytes),
            "achieved_layout": round(layout_bytes / (per_launch_ms / 1e3) / 1e9, 2),
            "peak_source": "measured" if os.path.exists(peaks_path) else "fallback"}
    levels_per_step = st["levels"] * sweeps
    level_stats = {"levels_per_sweep": st["levels"],
                   "us_per_level": round(kernel_ms * 1e3 / max(levels_per_step, 1), 3)}

    # end to end through the C ABI from host buffers
    e2e = None
    if rank == 0 or True:
        fp = np.ascontiguousarray(g.factor_ptr, np.int64)
        host_p = np.empty(g.n_vars, np.float32)
        e2e_t = []
        h2d = d2h = 0
        for i in range(max(2, min(args.steps, 5))):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            H = F.Graph(g, strategy, stream=stream)
            for k, v in WORKLOAD_OPTIONS.get(args.workload, {}).items():
                H.set_option(k, v)
            H.run(max_iters, tol)
            host_p[:] = H.marginals()
            sth = H.stats()
            H.close()
            torch.cuda.synchronize()
            e2e_t.append(time.perf_counter() - t0)
        E, V, A = g.n_edges, g.n_vars, g.n_factors
        halves = 2 if strategy == "TOPO_FB" else 1
        h2d = 4 * (A + 1) + A + 4 * A + 4 * E * 3 + 4 * (V + 1) + 4 * V + (8 * E * halves if strategy != "PARALL" else 0)
        d2h = 4 * V + 4 * 64 * sth["iters"] + 8
        e2e = {"value": round(sth["updates"] / float(np.median(e2e_t)), 1), "unit": "msg_updates/s",
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
               "ms_per_step": round(float(np.median(e2e_t)) * 1e3, 3)}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(args.workload, budget_s=args.cpu_seconds)
    forms = None
    if world == 1 and not args.no_forms:
        forms = forms_compare(args, stream)

    if rank == 0:
        line = {
            "metric": "BP message updates/s", "value": round(value, 1), "unit": "msg_updates/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(t_max / args.steps, 4), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": args.workload, "desc": desc, "n_vars": g.n_vars, "n_factors": g.n_factors,
                       "n_edges": g.n_edges, "strategy": strategy, "max_iters": max_iters, "tol": tol,
                       "sweeps_per_step": st["iters"], "levels_per_sweep": st["levels"],
                       "l2": "flushed between steps (512 MiB write)",
                       "parallelism": f"replicas{world}"},
            "time_to_converge_ms": round(total_ms / args.steps, 4),
            "roofline": roof, "level_latency": level_stats, "cpu_baseline": cpu, "e2e": e2e, "forms": forms,
            "gpu_launches": int(launches),
            "clocks": clk.summary(),
        }
        print(json.dumps(line))
    G.close()
    if world > 1:
        torch.distributed.destroy_process_group()


def cpu_baseline(workload, budget_s=15.0):
    """The FP64 oracle on the host cores, on a bounded sample of the workload:
    the first few sweeps/iterations of the same graph and schedule, once on
    one thread (the paper's single-threaded baseline form) and once with each
    level's independent updates spread over every host core (same results)."""
    from oracle import oracle as O
    O.build()
    _, strategy, max_iters, tol, _ = WORKLOADS[workload]
    kw, note = ORACLE_SAMPLE_GRAPHS.get(workload, ({}, ""))
    g = make_graph(workload, **kw)
    o = O.Oracle(g)
    host = os.cpu_count() or 1
    # calibrate: one iteration on one thread
    t0 = time.perf_counter()
    o.run(strategy, 1, 0.0)
    t1 = time.perf_counter() - t0
    iters = int(max(1, min(max_iters, budget_s / max(t1, 1e-6))))
    unit = "sweeps" if strategy == "TOPO_FB" else "iterations"
    where = f"{note}, {g.n_edges} edges," if note else f"the full {workload} graph"
    t0 = time.perf_counter()
    r = o.run(strategy, iters, 0.0)
    dt = time.perf_counter() - t0
    t0 = time.perf_counter()
    rp = o.run(strategy, iters, 0.0, threads=host)
    dtp = time.perf_counter() - t0
    return {"value": round(r["updates"] / dt, 1), "unit": "msg_updates/s", "cores": 1, "kind": "oracle",
            "host_cores": host,
            "sample": f"{iters} {unit} of {strategy} on {where} from uniform messages ({dt:.1f} s, single thread)",
            "parallel": {"value": round(rp["updates"] / dtp, 1), "unit": "msg_updates/s", "cores": rp["threads"],
                         "kind": "oracle",
                         "sample": f"the same {iters} {unit}, each level's updates over {rp['threads']} host "
                                   f"threads ({dtp:.1f} s)"}}


def run_reference_alarms(args, world):
    """The alarms workload's reference arm: the same loop on the FP64 oracle."""
    from paper_2509_22337_gb300 import ranking
    _, strategy, max_iters, tol, desc = WORKLOADS["alarms"]
    g, alarms, truth = alarms_setup()
    times = []
    for k in range(args.warmup + args.steps):
        G = OracleGraph(g, strategy)
        G.run(max_iters, tol)
        t0 = time.perf_counter()
        r = ranking.run_loop(G, alarms, truth, max_iters, tol)
        if k >= args.warmup:
            times.append(time.perf_counter() - t0)
    tot = float(sum(times))
    value = len(alarms) * args.steps / tot
    line = {"impl": "reference", "metric": "alarm-ranking interactions/s", "value": round(value, 3),
            "unit": "interactions/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(tot / args.steps * 1e3, 3), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "alarms", "desc": desc, "strategy": strategy},
            "cpu_baseline": {"value": round(value, 3), "unit": "interactions/s", "cores": 1, "kind": "oracle",
                             "sample": "the whole 30-question loop per step",
                             "inversions": r["inversions"], "rank_100pct_t": r["rank100"],
                             "rank_90pct_t": r["rank90"]},
            "e2e": {"value": round(value, 3), "unit": "interactions/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def run_reference(args):
    rank, world, local = dist_info()
    if rank != 0:
        return
    if args.workload == "alarms":
        run_reference_alarms(args, world)
        return
    from oracle import oracle as O
    O.build()
    _, strategy, max_iters, tol, desc = WORKLOADS[args.workload]
    kw, note = ORACLE_SAMPLE_GRAPHS.get(args.workload, ({}, ""))
    g = make_graph(args.workload, **kw)
    o = O.Oracle(g)
    sample_iters = {"smartfl200k": 4, "bingo1m": 2, "bingo1m_residual": 1, "tiny": 50,
                    "generic200k": 2}[args.workload]
    where = f"{note}, {g.n_edges} edges," if note else "the full graph"
    host = os.cpu_count() or 1
    for _ in range(args.warmup):
        o.run(strategy, 1, 0.0, threads=host)
    times, upd, used = [], 0, 1
    for _ in range(args.steps):
        t0 = time.perf_counter()
        r = o.run(strategy, sample_iters, 0.0, threads=host)
        times.append(time.perf_counter() - t0)
        upd += r["updates"]
        used = r["threads"]
    tot = float(sum(times))
    value = upd / tot
    line = {
        "impl": "reference", "metric": "BP message updates/s", "value": round(value, 1),
        "unit": "msg_updates/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(tot / args.steps * 1e3, 3), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "desc": desc, "strategy": strategy,
                   "sample": f"{sample_iters} {'sweeps' if strategy == 'TOPO_FB' else 'iterations'} of {where} per step",
                   "sample_n_vars": g.n_vars, "sample_n_edges": g.n_edges},
        "cpu_baseline": {"value": round(value, 1), "unit": "msg_updates/s", "cores": used, "kind": "oracle",
                         "host_cores": host,
                         "sample": f"{sample_iters} {strategy} {'sweeps' if strategy == 'TOPO_FB' else 'iterations'} of {where} per step, each level's "
                                   f"updates over {used} host threads"},
        "e2e": {"value": round(value, 1), "unit": "msg_updates/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--workload", default="bingo1m", choices=sorted(WORKLOADS))
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-forms", action="store_true",
                    help="single-graph workloads: skip the reduced batched and served comparisons")
    ap.add_argument("--forms-graphs", type=int, default=128, help="graphs of the reduced batched comparison")
    ap.add_argument("--forms-sessions", type=int, default=16, help="sessions of the reduced served comparison")
    ap.add_argument("--forms-requests", type=int, default=64, help="requests of the reduced served comparison")
    ap.add_argument("--batch-graphs", type=int, default=512)
    ap.add_argument("--serve-sessions", type=int, default=64)
    ap.add_argument("--serve-requests", type=int, default=128)
    ap.add_argument("--serve-inflight", type=int, default=64)
    ap.add_argument("--serve-tick", type=int, default=16)
    ap.add_argument("--cold-windows", type=int, default=1,
                    help="serving: windows of the stream replayed through the cold-start path")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
