"""Multi-rank timing aggregation of bench.py, world size 2 over gloo on CPU.

Each rank runs its own independent session (replicas, no data-path
collective); the whole-job figures are the max elapsed time over ranks and the
sum of the units all ranks processed.
"""

import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, results):
    import torch.distributed as dist

    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    elapsed = 1.0 + rank  # rank 1 is the slower one
    units = 100.0 * (rank + 1)
    t, u = bench.aggregate(elapsed, units, dist)
    results[rank] = (t, u, bench.env_rank())
    dist.barrier()
    dist.destroy_process_group()


def test_aggregate_max_time_sum_units_world2():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    results = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, results)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    for r in range(2):
        t, u, (rank, _, world) = results[r]
        assert t == pytest.approx(2.0)  # max over ranks
        assert u == pytest.approx(300.0)  # sum over ranks
        assert rank == r and world == 2


def test_aggregate_single_process_is_identity():
    import bench

    assert bench.aggregate(1.5, 42.0, None) == (1.5, 42.0)
