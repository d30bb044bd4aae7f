"""The replica path of bench.py on two CPU ranks (gloo): the job time is the slowest rank's,
the work the sum of the ranks' (weak scaling, no collective on the data path)."""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    ms, cells = bench.reduce_over_ranks(10.0 * (rank + 1), 1000 * (rank + 1), world, "cpu")
    out.put((rank, ms, cells))
    dist.barrier()
    dist.destroy_process_group()


def test_reduce_over_two_gloo_ranks():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res == [(0, 20.0, 3000.0), (1, 20.0, 3000.0)]


def test_single_rank_is_identity():
    import bench

    assert bench.reduce_over_ranks(12.5, 777, 1, "cpu") == (12.5, 777)
