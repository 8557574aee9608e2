"""The N > 1 bench path (one replica per GPU, weak scaling): the whole-job step
time is the slowest rank's and the work is the sum of every rank's cells.
Exercised with a world-size-2 gloo process group on the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import sys

    import torch
    import torch.distributed as dist

    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms, cells = bench.reduce_over_ranks(10.0 + 5.0 * rank, 1e9 * (rank + 1), dist, torch.device("cpu"))
    out[rank] = (ms, cells)
    dist.barrier()
    dist.destroy_process_group()


def test_reduce_over_two_ranks():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for r in range(2):
        assert out[r] == (15.0, 3e9)


def test_single_process_passthrough():
    import bench

    assert bench.reduce_over_ranks(3.0, 7.0, None, None) == (3.0, 7.0)
