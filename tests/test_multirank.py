"""Multi-rank bench logic on CPU (gloo, world_size 2): the single-mesh path
runs independent replicas per rank with no data-path collective; the job
time is the max over ranks and the rate counts the units of all ranks."""
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


def _worker(rank, world, port, q):
    import torch.distributed as dist
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = 10.0 + 5.0 * rank           # rank 1 is the slow one
    ms_max = bench.reduce_over_ranks(ms, dist, "cpu")
    rate = bench.aggregate_rate(1000.0, ms_max, world)
    q.put((rank, ms_max, rate))
    dist.barrier()
    dist.destroy_process_group()


def test_replicas_max_time_and_aggregate_rate():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for rank, ms_max, rate in res:
        assert ms_max == 15.0
        assert abs(rate - 2 * 1000.0 / 15e-3) < 1e-6


def test_single_rank_identity():
    import bench
    assert bench.reduce_over_ranks(7.0, None) == 7.0
    assert bench.aggregate_rate(100.0, 10.0, 1) == 100.0 / 10e-3
