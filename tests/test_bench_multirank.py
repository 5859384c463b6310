"""bench.py's multi-rank aggregation (slowest rank's time, summed units) on
world_size 2 with the gloo backend, CPU only."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t, u = bench.aggregate(100.0 + 50.0 * rank, 3 + rank, dist, "cpu")
    out[rank] = (t, u)
    w, r, loc = bench.dist_setup()
    assert (w, r) == (world, rank)
    dist.barrier()
    dist.destroy_process_group()


def test_aggregate_two_ranks():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    assert out[0] == (150.0, 7) and out[1] == (150.0, 7)


def test_aggregate_single_process():
    import bench
    assert bench.aggregate(12.5, 4) == (12.5, 4)
