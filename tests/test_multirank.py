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


def test_balanced_partition_properties():
    """The greedy cost balance assigns every unit exactly once, keeps each
    rank's list ascending, is deterministic, and meets the list-scheduling
    bound (largest load <= average load + largest unit) and Graham's 4/3
    bound against brute force on small cases."""
    import itertools

    import numpy as np

    from paper_1607_00315_gb300 import shard, synth

    rng = np.random.default_rng(7)
    for world in (1, 2, 3, 8):
        costs = [shard.unit_cost(int(n), 4) for n in rng.integers(32, 513, size=200)]
        parts = shard.balanced_partition(costs, world)
        assert len(parts) == world
        assert sorted(k for p in parts for k in p) == list(range(len(costs)))
        assert all(p == sorted(p) for p in parts)
        assert parts == shard.balanced_partition(costs, world)
        loads = [sum(costs[k] for k in p) for p in parts]
        assert max(loads) <= sum(costs) / world + max(costs) + 1e-9
    for trial in range(20):
        costs = list(rng.uniform(0.1, 5.0, size=7))
        world = 2 + trial % 2
        loads = [sum(costs[k] for k in p) for p in shard.balanced_partition(costs, world)]
        best = min(max(sum(c for c, a in zip(costs, asg) if a == r) for r in range(world))
                   for asg in itertools.product(range(world), repeat=len(costs)))
        assert max(loads) <= 4.0 / 3.0 * best + 1e-12
    # the batched workload's 512 instances over 8 ranks stay within 2% of even
    probs = synth.batch_problems(512)
    costs = [shard.unit_cost(p.n, len(synth.LAMBDA_PATH)) for p in probs]
    loads = [sum(costs[k] for k in p) for p in shard.balanced_partition(costs, 8)]
    assert max(loads) <= 1.02 * sum(costs) / 8
    assert shard.balanced_partition([], 3) == [[], [], []]
    with pytest.raises(ValueError):
        shard.balanced_partition([1.0], 0)


def _batched_worker(rank, world, port, q):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    local_s, local_solves = [(2.0, 300), (2.5, 212)][rank]
    res = bench.batched_job_value(local_s, local_solves, world, "cpu")
    dist.barrier()
    q.put((rank,) + res)
    dist.destroy_process_group()


def test_batched_job_value_two_gloo_ranks():
    """Sharded batches: the job's time is the slowest rank's and the solves
    of all ranks are counted once."""
    import multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_batched_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, max_s, total, value in res:
        assert max_s == 2.5 and total == 512
        assert value == pytest.approx(512 / 2.5)


def test_route_stream_properties():
    """Online routing of a serving stream: deterministic, covers every
    request, sends each request to a rank whose assigned work before it was
    the least, and keeps the final loads within one request's cost of each
    other."""
    import numpy as np

    from paper_1607_00315_gb300 import shard, synth

    trace = synth.serving_trace(300)
    costs = [shard.unit_cost(r[1]) for r in trace]
    for world in (1, 2, 4, 8):
        own = shard.route_stream(costs, world)
        assert own == shard.route_stream(costs, world)
        assert len(own) == len(costs) and set(own) <= set(range(world))
        load = np.zeros(world)
        for c, r in zip(costs, own):
            assert load[r] == load.min()
            load[r] += c
        assert load.max() - load.min() <= max(costs) + 1e-9
    assert shard.route_stream([], 2) == []
