"""The multi-rank timing path of bench.py (replicas, no data-path collective) with
world_size 2 on CPU (gloo): the job time is the slowest rank's and the units are
summed over ranks."""
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


def _worker(rank, world, port, out):
    import torch
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local_ms = 100.0 + 50.0 * rank          # rank 1 is the slow one
    local_units = 1000 + rank
    ms, units = bench.aggregate(dist, torch.device("cpu"), local_ms, local_units)
    out[rank] = (ms, units)
    dist.barrier()
    dist.destroy_process_group()


def test_aggregate_max_time_sum_units_two_ranks():
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
    assert out[0] == out[1] == (150.0, 2001)


def test_aggregate_single_process_is_identity():
    import bench
    assert bench.aggregate(None, None, 12.5, 7) == (12.5, 7)
