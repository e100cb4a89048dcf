"""Host-side helpers for runs over several GPUs (one process per GPU).

The solver itself runs on one GPU; what shards across ranks are independent
problems: every rank solves its own right-hand side (weak scaling), and the
batched workload's problems are partitioned between ranks with no
communication on the data path.  Only the timing uses a collective (the
slowest rank's time).  Works with the ``nccl`` backend on GPUs and ``gloo``
on CPUs.
"""
from __future__ import annotations

import os


def rank_env():
    """(rank, world size, local rank) from the launcher's environment."""
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def problem_seed(base: int, rank: int) -> int:
    """Seed of rank ``rank``'s right-hand side (distinct per rank)."""
    return base + rank


def shard_batch(costs, rank: int, world: int):
    """Indices of the problems rank ``rank`` solves: the problems are dealt
    largest first to the rank with the least total cost so far (ties: lowest
    rank), so that every problem goes to exactly one rank and the ranks'
    loads differ by at most one problem's cost."""
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    load = [0.0] * world
    mine = []
    for i in order:
        r = min(range(world), key=lambda k: (load[k], k))
        load[r] += costs[i]
        if r == rank:
            mine.append(i)
    return sorted(mine)


def max_over_ranks(value: float, device=None) -> float:
    """The largest value over all ranks (identity without a process group)."""
    import torch
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value: float, device=None) -> float:
    """The sum of a value over all ranks (identity without a process group)."""
    import torch
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())
