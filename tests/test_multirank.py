"""The multi-rank (weak scaling) host logic of bench.py with two gloo ranks
on CPU: ranks get distinct points, and the report combines the units of all
ranks with the slowest rank's time."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import workloads as W


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, q):
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    units, ms = bench.combine_ranks(1000, 10.0 + rank, dist, "cpu")
    pts = W.points_f64(1, 16, bench.points_seed(rank))
    q.put((rank, units, ms, pts))
    dist.destroy_process_group()


def test_two_gloo_ranks_combine_weak_scaling():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort(key=lambda x: x[0])
    for _, units, ms, _ in res:
        assert units == 2000 and ms == 11.0
    assert not np.array_equal(res[0][3], res[1][3])


def test_single_rank_passthrough():
    import bench
    assert bench.combine_ranks(5, 3.0) == (5, 3.0)
