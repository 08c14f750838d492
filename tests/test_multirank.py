"""The N > 1 path of bench.py on CPU: two gloo ranks run as replicas (each its
own seeded batch, no data exchange), the step time is the maximum over
ranks and the throughput counts the units of every rank."""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from workloads import c4_batch
    local = [120.0, 95.0][rank]
    ms, value = bench.aggregate(local, 4096, dist, "cpu")
    mu, sizes = c4_batch(16, seed=bench.rank_seed(4, rank))
    q.put((rank, ms, value, mu[0].tolist()))
    dist.destroy_process_group()


def test_two_rank_replicas_aggregate():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (_, ms0, v0, mu0), (_, ms1, v1, mu1) = res
    assert ms0 == ms1 == 120.0                      # the slowest rank sets the step time
    assert abs(v0 - 2 * 4096 / 0.120) < 1e-6 and v0 == v1
    assert mu0 != mu1                               # each replica has its own batch


def test_single_rank_aggregate():
    import bench
    ms, value = bench.aggregate(50.0, 4096, None)
    assert ms == 50.0 and abs(value - 4096 / 0.05) < 1e-9
