"""The multi-rank bookkeeping of bench.py on CPU: two gloo ranks, each with its
own (independent-instance) timing; the job value takes the slowest rank's
time and counts the solves of all ranks (weak scaling, replicas only)."""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    local_ms = [400.0, 500.0][rank]  # rank 1 is the slower one
    max_ms, value = bench.job_value(local_ms, 5, world, "cpu")
    dist.barrier()
    q.put((rank, max_ms, value))
    dist.destroy_process_group()


def test_job_value_two_gloo_ranks():
    import multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, max_ms, value in res:
        assert max_ms == 500.0
        assert value == pytest.approx(2 * 5 / 0.5)


def test_job_value_single_rank():
    import bench

    assert bench.job_value(250.0, 5, 1, "cpu") == (250.0, pytest.approx(20.0))
