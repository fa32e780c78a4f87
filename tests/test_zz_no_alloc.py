"""fbp_run_fixed_scratch (include/fbp_fixed.h) against fbp_run, through the C ABI.

Some callers cannot allocate device memory once they are running: a server
that hands all of its device memory to resident graphs before the first
request, or a latency-bound caller that cannot take an allocation (and the
synchronisation it may bring) inside a request.  fbp_run may grow a graph's
per-iteration residual words through the graph's allocator;
fbp_run_fixed_scratch takes that scratch from a static device array instead.
It runs the same persistent level engine as fbp_run, so its results must equal
fbp_run's bit for bit (well inside the 1e-5 marginal tolerance of the parity
tests).  The file name puts it last in collection: it must pass in a fresh
process and after every other GPU test of the session.
"""
import numpy as np
import pytest

from paper_2509_22337_gb300 import gen

pytestmark = pytest.mark.gpu


def _same(a, b, ra, rb, what):
    assert ra[0] == rb[0], f"{what}: status {ra[0]} vs {rb[0]}"
    assert ra[1] == rb[1], f"{what}: iterations {ra[1]} vs {rb[1]}"
    assert np.float32(ra[2]).tobytes() == np.float32(rb[2]).tobytes(), f"{what}: residual {ra[2]} vs {rb[2]}"
    assert np.array_equal(a.marginals(), b.marginals()), what
    assert np.array_equal(a.messages(), b.messages()), what
    sa, sb = a.stats(), b.stats()
    for k in ("updates", "guards", "iters", "levels"):
        assert sa[k] == sb[k], f"{what}: stats[{k}] {sa[k]} vs {sb[k]}"


@pytest.mark.parametrize("strategy", ["TOPO_FB", "SEQFIX", "TOPO"])
def test_two_calls_in_a_row_match_fbp_run(fbp, strategy):
    fg = gen.smartfl(n_layers=24, width=120, seed=61, planted=True)
    a, b = fbp.Graph(fg, strategy), fbp.Graph(fg, strategy)
    for call in (1, 2):  # the second call continues from the first one's messages
        ra = a.run(40, 1e-6)
        rb = b.run_fixed_scratch(40, 1e-6)
        _same(a, b, ra, rb, f"{strategy} call {call}")
    a.close()
    b.close()


@pytest.mark.parametrize("alloc", ["torch", None])
def test_allocates_nothing_where_fbp_run_would(fbp, alloc):
    """A fresh graph's residual words cover 64 iterations; fbp_run grows them
    through the graph's allocator (PyTorch's caching allocator, or cudaMalloc
    when the graph has no allocator) for a longer run.  The fixed-scratch call
    must touch neither: PyTorch's counters and the device's free bytes stay
    as they were across two warmed calls."""
    import gc
    import torch
    fg = gen.smartfl(n_layers=16, width=80, seed=62, planted=True)
    a, b = fbp.Graph(fg, "TOPO_FB", alloc=alloc), fbp.Graph(fg, "TOPO_FB", alloc=alloc)
    b.run_fixed_scratch(5, 0.0)  # first call on the device: symbol lookup, module load
    b.reset()
    # graphs left by earlier tests free their memory when collected: collect
    # them now and keep the collector off while the allocator is watched
    gc.collect()
    gc.disable()
    try:
        torch.cuda.synchronize()
        before = (torch.cuda.memory_allocated(), torch.cuda.memory_reserved())
        free_before = torch.cuda.mem_get_info()[0]
        rb = b.run_fixed_scratch(3000, 0.0)
        rb2 = b.run_fixed_scratch(3000, 0.0)
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free_before
        assert (torch.cuda.memory_allocated(), torch.cuda.memory_reserved()) == before
        ra = a.run(3000, 0.0)
        torch.cuda.synchronize()
        if alloc == "torch":
            assert torch.cuda.memory_allocated() > before[0]  # fbp_run did grow its residual words
    finally:
        gc.enable()
    ra2 = a.run(3000, 0.0)
    _same(a, b, ra2, rb2, "second 3000-iteration call")
    assert ra[1] == rb[1] == 3000
    a.close()
    b.close()


def test_iteration_limit(fbp):
    """FBP_FIXED_SCRATCH_MAX_ITERS iterations run; one more is rejected before
    any work and leaves the graph as it was."""
    limit = fbp.FBP_FIXED_SCRATCH_MAX_ITERS
    fg = gen.random_tree(10, seed=63)
    a, b = fbp.Graph(fg, "TOPO_FB"), fbp.Graph(fg, "TOPO_FB")
    m0 = b.messages().copy()
    with pytest.raises(fbp.FbpError) as e:
        b.run_fixed_scratch(limit + 1, 0.0)
    assert e.value.code == fbp.FBP_ERR_INVALID_ARG and str(limit) in str(e.value)
    assert np.array_equal(b.messages(), m0)
    ra = a.run(limit, 0.0)
    rb = b.run_fixed_scratch(limit, 0.0)
    assert rb[1] == limit
    _same(a, b, ra, rb, "limit")
    a.close()
    b.close()


def test_rejects_strategies_that_need_run_buffers(fbp):
    fg = gen.tiny()
    for strategy in ("PARALL", "RESIDUAL"):
        g = fbp.Graph(fg, strategy)
        with pytest.raises(fbp.FbpError) as e:
            g.run_fixed_scratch(5, 0.0)
        assert e.value.code == fbp.FBP_ERR_INVALID_ARG
        g.close()


def test_zero_iterations_and_empty_graph(fbp):
    fg = gen.smartfl(n_layers=6, width=20, seed=64)
    a, b = fbp.Graph(fg, "TOPO"), fbp.Graph(fg, "TOPO")
    _same(a, b, a.run(0, 1e-6), b.run_fixed_scratch(0, 1e-6), "zero iterations")
    empty = gen.FactorGraph(3, np.zeros(1, np.int64), np.zeros(0, np.int32), np.zeros(0, np.uint8),
                            np.zeros(0, np.float32), np.array([0.3, np.nan, 0.9], np.float32),
                            np.full(3, -1, np.int8), "empty")
    e1, e2 = fbp.Graph(empty, "SEQFIX"), fbp.Graph(empty, "SEQFIX")
    _same(e1, e2, e1.run(10, 1e-6), e2.run_fixed_scratch(10, 1e-6), "empty graph")
    for g in (a, b, e1, e2):
        g.close()
