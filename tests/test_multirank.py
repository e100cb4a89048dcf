"""The multi-rank host logic on CPU: two processes over gloo (no GPU).

Every rank must get its own right-hand side, the batched workload's problems
must be partitioned exactly once across ranks with balanced loads, and the
timing reduction must return the slowest rank's time on every rank.
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2402_12833_gb300 import multi
from paper_2402_12833_gb300 import problems as pb


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, lr = multi.rank_env()
        sizes = pb.batch_sizes(256, seed=4)
        costs = [s * s for s in sizes]
        mine = multi.shard_batch(costs, r, w)
        # the slowest rank's time, as bench.py takes it
        t = multi.max_over_ranks(1.5 + r)
        total = multi.sum_over_ranks(sum(costs[i] for i in mine))
        shards = [None] * w
        dist.all_gather_object(shards, mine)
        seeds = [None] * w
        dist.all_gather_object(seeds, multi.problem_seed(2, r))
        q.put((r, w, lr, t, total, shards, seeds))
    finally:
        dist.destroy_process_group()


def test_two_ranks_over_gloo():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    results = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    sizes = pb.batch_sizes(256, seed=4)
    costs = [s * s for s in sizes]
    for r, w, lr, t, total, shards, seeds in results:
        assert w == world and lr == r
        assert t == 1.5 + (world - 1)                      # max over ranks
        assert total == sum(costs)                         # every problem counted once
        flat = sorted(i for sh in shards for i in sh)
        assert flat == list(range(256))                    # an exact partition
        loads = [sum(costs[i] for i in sh) for sh in shards]
        assert max(loads) - min(loads) <= max(costs)       # balanced to one problem
        assert len(set(seeds)) == world                    # distinct right-hand sides


def test_shard_batch_single_rank_and_degenerate():
    assert multi.shard_batch([5, 1, 3], 0, 1) == [0, 1, 2]
    assert multi.shard_batch([], 0, 2) == []
    # more ranks than problems: some ranks get none, none gets two
    shards = [multi.shard_batch([4, 4], r, 3) for r in range(3)]
    assert sorted(i for s in shards for i in s) == [0, 1]
    assert max(len(s) for s in shards) == 1
    assert multi.max_over_ranks(3.25) == 3.25               # no process group: identity
