"""Replica aggregation of bench.py across ranks (gloo, world size 2, CPU): the slowest rank's time
is reported and the throughput counts every rank's units."""
import os
import socket

import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    r, local, w = bench.dist_init("gloo")
    assert (r, w) == (rank, world)
    bench.barrier()
    value, t = bench.aggregate(units_per_rank=1000, times_ms_rank=100.0 * (rank + 1), world=w)
    out[rank] = (value, t)
    import torch.distributed as dist
    dist.destroy_process_group()


def test_two_rank_aggregate():
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
    # slowest rank: 200 ms; 2 ranks x 1000 units / 0.2 s = 10000 units/s on both ranks
    assert out[0] == out[1] == (10000.0, 200.0)
