"""The replica path of bench.py on two CPU ranks (gloo): each rank runs an
independent replica, the job's time is the slowest rank's, and the value is
the points of all ranks over that time.  No GPU is involved."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = [120.0, 150.0][rank]
    total, value = bench.combine_ranks(local_ms, units_per_rank=1000, steps=10, world=world)
    q.put((rank, total, value))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_replicas():
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
    for rank, total, value in res:
        assert total == 150.0
        assert value == pytest.approx(2 * 1000 * 10 / 0.150)


def test_single_rank_needs_no_process_group():
    import bench
    total, value = bench.combine_ranks(50.0, 100, 5, 1)
    assert total == 50.0 and value == pytest.approx(100 * 5 / 0.05)
