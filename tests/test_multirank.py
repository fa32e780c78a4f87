"""The multi-GPU host logic of bench.py on CPU: two gloo ranks on 127.0.0.1.

A single graph does not shard (replicas only); independent units (batched
graphs, served sessions) are bin-packed over the ranks with no collective on
the data path, and the job's time and work are the slowest rank's time and
the sum over ranks.  These tests run that logic with the gloo backend."""
import multiprocessing as mp
import os
import socket

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import sys
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t, u = bench.aggregate(10.0 * (rank + 1), 100 + rank, device="cpu")
    sizes = [5, 1, 9, 3, 3, 7, 2, 8]
    mine = bench.shard(sizes, world, rank)
    parts = [None] * world
    dist.all_gather_object(parts, mine)
    dist.destroy_process_group()
    q.put((rank, t, u, parts))


def _run(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in ps:
        p.start()
    out = [q.get(timeout=120) for _ in ps]
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    return sorted(out)


def test_two_ranks_aggregate_and_shard():
    pytest.importorskip("torch.distributed")
    out = _run(2)
    for rank, t, u, parts in out:
        assert t == 20.0 and u == 201.0  # slowest rank's time, summed work
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(8))  # every unit on exactly one rank
        sizes = [5, 1, 9, 3, 3, 7, 2, 8]
        loads = [sum(sizes[i] for i in p) for p in parts]
        assert max(loads) - min(loads) <= max(sizes)
    assert out[0][3] == out[1][3]  # both ranks computed the same assignment


def test_single_process_is_unchanged():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate(3.5, 7, device="cpu") == (3.5, 7.0)
    assert bench.shard([4, 2, 1], 1, 0) == [0, 1, 2]
