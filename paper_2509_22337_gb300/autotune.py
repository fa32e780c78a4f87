"""Autotuner for the launch shapes of the CUDA path.

It times candidate launch shapes on the caller's own graph (or batch) and
keeps the fastest.  No knob changes the arithmetic: the engine's shapes and
the flooding split (a long row's product is always grouped in 256-entry
sub-chunks, whichever kernel carries it) leave every message bit-identical,
which the tests check, so the timing-dependent pick never changes a result:

* static strategies (persistent level engine): grid mode with 1, 1/2 or 2
  blocks per SM, a single block (block barriers between levels: for narrow
  levels), one 16-block cluster, or one launch per level (the paper's
  execution); the level-fusion threshold (runs of consecutive levels of at
  most that many lanes go to one block between grid barriers) and the
  one-block threshold (the whole run in one block when the levels average at
  most that many lanes);
* flooding: how long a variable row may get before its sub-chunk products
  are combined by a warp instead of one thread, and the block size of the
  sub-chunk pass (the threads-per-message split of long rows).

Choices are cached in a JSON file keyed by a signature of the graph
(strategy, size and level-shape buckets), so a second graph of the same shape
skips the search.  Set FBP_TUNE_CACHE to choose the file.
"""
from __future__ import annotations

import json
import math
import os
import time

from . import fbp as F

CACHE = os.environ.get("FBP_TUNE_CACHE", os.path.join(os.path.expanduser("~"), ".cache", "fbp_gb300_tune.json"))


def _bucket(x: float) -> int:
    return int(round(math.log2(max(x, 1.0))))


def _load():
    try:
        with open(CACHE) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(cache):
    try:
        os.makedirs(os.path.dirname(CACHE), exist_ok=True)
        tmp = CACHE + f".tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(cache, f, indent=1, sort_keys=True)
        os.replace(tmp, CACHE)
    except OSError:
        pass


def graph_signature(fg, strategy: str, levels: int = 0) -> str:
    return f"graph/{strategy}/v{_bucket(fg.n_vars)}/e{_bucket(fg.n_edges)}/l{_bucket(levels + 1)}"


def batch_signature(graphs, schedules) -> str:
    n_static = sum(s != "PARALL" for s in schedules)
    e = sum(g.n_edges for g in graphs)
    return f"batch/n{_bucket(len(graphs))}/s{_bucket(n_static + 1)}/e{_bucket(e)}"


def _sms() -> int:
    import torch
    return torch.cuda.get_device_properties(0).multi_processor_count


def _time(fn, reps: int = 2) -> float:
    import torch
    best = float("inf")
    for _ in range(reps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        fn()
        torch.cuda.synchronize()
        best = min(best, time.perf_counter() - t0)
    return best


def graph_candidates(strategy: str):
    sms = _sms()
    if strategy == "PARALL":
        for hub in (64, 128, 256):
            for chunk in (512, 1024, 2048):
                yield {F.FBP_OPT_FLOOD_HUB_MIN: hub, F.FBP_OPT_FLOOD_CHUNK: chunk}
        return
    base = {F.FBP_OPT_ENGINE: 1, F.FBP_OPT_ENGINE_CLUSTER: 1, F.FBP_OPT_ENGINE_GRID: 0,
            F.FBP_OPT_ENGINE_FUSE_LANES: 0, F.FBP_OPT_ENGINE_SOLO_LANES: 128}
    yield dict(base)
    for grid in (1, sms // 2, sms, 2 * sms):
        yield {**base, F.FBP_OPT_ENGINE_GRID: grid}
    for solo in (0, 32, 512):
        yield {**base, F.FBP_OPT_ENGINE_SOLO_LANES: solo}
    for fuse in (32, 64, 128, 256):  # level fusion inside the grid run (one-block switch off)
        yield {**base, F.FBP_OPT_ENGINE_FUSE_LANES: fuse, F.FBP_OPT_ENGINE_SOLO_LANES: 0}
    yield {**base, F.FBP_OPT_ENGINE_CLUSTER: 16}
    yield {**base, F.FBP_OPT_ENGINE: 0}


def _apply(G, opts):
    for k, v in opts.items():
        G.set_option(int(k), int(v))


def tune_graph(G, fg, strategy: str, sample_iters: int = 5, use_cache: bool = True) -> dict:
    """Pick the fastest launch shape for graph handle G (a fbp.Graph built from
    FactorGraph fg with `strategy`), apply it and return it.  The messages are
    reset afterwards."""
    levels = G.stats()["levels"] if strategy != "PARALL" else 1
    sig = graph_signature(fg, strategy, levels)
    cache = _load() if use_cache else {}
    if sig in cache:
        opts = {int(k): v for k, v in cache[sig]["opts"].items()}
        _apply(G, opts)
        return opts
    results = []
    for opts in graph_candidates(strategy):
        try:
            _apply(G, opts)
        except F.FbpError:
            continue
        def run():
            G.reset()
            G.run(sample_iters, 0.0)
        run()  # warm-up (first use builds plans)
        results.append((_time(run), opts))
    results.sort(key=lambda r: r[0])
    best = results[0][1]
    _apply(G, best)
    G.reset()
    if use_cache:
        cache[sig] = {"opts": {str(k): v for k, v in best.items()},
                      "seconds": results[0][0], "tried": len(results)}
        _store(cache)
    return best


def batch_candidates(form: str = "engine"):
    """Launch shapes tried for a batch of the given form ("engine": static
    members in the level engine; "queue": static members in the member queue;
    "one": every member in the member queue)."""
    if form == "one":
        yield from batch_candidates_one()
        return
    sms = _sms()
    if form == "queue":
        # how many member-queue clusters leave room for the flooding kernels
        # beside them (0: half of the resident ones; a large value: all)
        for cluster in (8, 16):
            for qc in (0, sms // 4, 1 << 20):
                yield dict(engine_grid=0, engine_cluster=cluster, flood_hub_min=256, flood_chunk=8192,
                           engine_fuse_lanes=0, engine_solo_lanes=128, queue_clusters=qc)
        yield dict(engine_grid=0, engine_cluster=8, flood_hub_min=128, flood_chunk=8192,
                   engine_fuse_lanes=0, engine_solo_lanes=128, queue_clusters=0)
        return
    for cluster in (1, 16):
        for grid in ((0, sms, 2 * sms) if cluster == 1 else (0,)):
            for hub in (128, 256):
                yield dict(engine_grid=grid, engine_cluster=cluster, flood_hub_min=hub, flood_chunk=8192,
                           engine_fuse_lanes=0, engine_solo_lanes=128, queue_clusters=0)
    for fuse in (64, 256):
        yield dict(engine_grid=0, engine_cluster=1, flood_hub_min=256, flood_chunk=8192, engine_fuse_lanes=fuse,
                   engine_solo_lanes=0, queue_clusters=0)


def batch_candidates_one():
    """The one-launch form's knob: blocks per cluster of the member queue."""
    for cluster in (16, 8):
        yield dict(engine_grid=0, engine_cluster=cluster, flood_hub_min=256, flood_chunk=8192,
                   engine_fuse_lanes=0, engine_solo_lanes=128, queue_clusters=0)


def tune_batch(B, graphs, schedules, use_cache: bool = True) -> dict:
    """Pick the fastest launch shapes for a fbp_batch.Batch by timing whole
    batch runs from uniform messages; apply and return them."""
    form = getattr(B, "form", "one" if getattr(B, "one_launch", False) else "engine")
    sig = batch_signature(graphs, schedules) + ("" if form == "engine" else "/" + form)
    cache = _load() if use_cache else {}
    if sig in cache:
        best = cache[sig]["tuning"]
        B.tune(**best)
        return best
    results = []
    for t in batch_candidates(form):
        B.tune(**t)
        def run():
            B.reset()
            B.run()
        run()
        results.append((_time(run, reps=1), t))
    results.sort(key=lambda r: r[0])
    best = results[0][1]
    B.tune(**best)
    B.reset()
    if use_cache:
        cache[sig] = {"tuning": best, "seconds": results[0][0], "tried": len(results)}
        _store(cache)
    return best
