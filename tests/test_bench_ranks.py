"""The benchmark's multi-rank path (replicas, max of the times and sum of the
work over ranks) on two gloo ranks on the CPU."""

import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    import torch.distributed as dist

    import bench

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mx, sm = bench.reduce_over_ranks([1.5 + rank, 7.0 - rank], [10.0 * (rank + 1)], "cpu")
        out.put((rank, mx, sm))
    finally:
        dist.destroy_process_group()


def test_reduce_over_two_gloo_ranks():
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    results = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for _, mx, sm in results:
        assert mx == [2.5, 7.0] and sm == [30.0]


def test_single_rank_is_identity():
    import bench

    assert bench.reduce_over_ranks([3.0], [4.0], "cpu") == ([3.0], [4.0])
