"""Multi-rank host logic on CPU: two gloo ranks shard a heterogeneous batch of
independent reconstructions and agree on the timed maximum."""
import os
import socket

import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2011_00162_gb300 import multi, synth


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    probs = synth.batched_problems(16, seed=3)
    costs = [len(p.offsets()) * p.m * p.m for p in probs]
    mine = multi.shard(costs, rank, world)
    got = [None] * world
    dist.all_gather_object(got, mine)
    t = multi.max_over_ranks(1.5 + rank)
    if rank == 0:
        out.put((got, t, costs))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_partition_the_batch():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got, t, costs = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    flat = sorted(i for part in got for i in part)
    assert flat == list(range(len(costs)))          # every reconstruction exactly once
    loads = [sum(costs[i] for i in part) for part in got]
    assert max(loads) <= 0.5 * sum(costs) + max(costs)  # greedy balance bound
    assert t == 2.5                                   # max over ranks


def test_shard_single_rank_and_errors():
    assert multi.shard([3.0, 1.0, 2.0], 0, 1) == [0, 1, 2]
    assert multi.max_over_ranks(4.0) == 4.0
    import pytest
    with pytest.raises(ValueError):
        multi.shard([1.0], 2, 2)
