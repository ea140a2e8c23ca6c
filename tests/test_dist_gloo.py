"""Replica aggregation of bench.py across ranks (world_size 2, gloo, CPU):
pairs are summed over ranks and the slowest rank's span is the job's span."""
import os
import socket

import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    pairs = 1.0e9 * (rank + 1)
    seconds = 0.5 + rank
    ms = 10.0 * (rank + 1)
    v, m = bench.aggregate(pairs, seconds, ms)
    out[rank] = (v, m)
    dist.barrier()
    dist.destroy_process_group()


def test_replica_aggregation_two_ranks():
    port = _free_port()
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    total = 1.0e9 + 2.0e9
    for r in range(2):
        v, m = out[r]
        assert abs(v - total / 1.5) < 1e-3 * total
        assert m == 20.0
