"""Replica aggregation of bench.py (N > 1 runs N independent workloads, one per
rank): the timed region is the maximum over ranks and the whole-job rate
counts every rank's steps.  World size 2 on the gloo backend, CPU only."""
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
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    elapsed = [100.0, 250.0][rank]
    t, value = bench.aggregate_over_ranks(elapsed, steps=10, world=world, dist=dist, device="cpu")
    results[rank] = (t, value)
    dist.destroy_process_group()


def test_max_over_ranks_and_whole_job_rate():
    ctx = mp.get_context("spawn")
    manager = ctx.Manager()
    results = manager.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, results)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    for r in range(2):
        t, value = results[r]
        assert t == pytest.approx(250.0)
        assert value == pytest.approx(2 * 10 / 0.25)
