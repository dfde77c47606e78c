"""Replica aggregation of bench.py across ranks (world size 2, gloo on CPU):
value = all ranks' work / the slowest rank's time."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t = bench.reduce_max_over_ranks(10.0 + 5.0 * rank, world)
        w = bench.reduce_sum_over_ranks(100.0 * (rank + 1), world)
        bench._barrier(world)
        out.put((rank, t, w))
    finally:
        dist.destroy_process_group()


def test_replica_reductions_gloo_world2():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # every rank sees the slowest time and the summed work
    assert res == [(0, 15.0, 300.0), (1, 15.0, 300.0)]


def test_single_rank_reductions_are_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_max_over_ranks(3.5, 1) == 3.5
    assert bench.reduce_sum_over_ranks(2.0, 1) == 2.0
