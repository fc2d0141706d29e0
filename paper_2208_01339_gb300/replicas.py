"""Running the solver on N GPUs of one node: replicas, no collectives.

The method's data path on one GPU has no exchange step, and independent
instances (the batched workload) are partitioned across ranks, so N > 1 runs
N independent solvers.  torch.distributed is used only for the timing
barrier and to take the slowest rank's time.
"""
from __future__ import annotations

import os


def rank_env():
    """(rank, world size, local rank) from the launcher's environment."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def shard(n_items: int, rank: int, world: int) -> range:
    """Contiguous block of item indices owned by `rank` (sizes differ by at most one)."""
    q, r = divmod(n_items, world)
    start = rank * q + min(rank, r)
    return range(start, start + q + (1 if rank < r else 0))


def shard_balanced(weights, rank: int, world: int) -> list:
    """Indices owned by `rank` when items of the given work weights are
    dealt, heaviest first, to the least-loaded rank (ties: lowest rank);
    every rank computes the same assignment.  Returned in index order."""
    load = [0.0] * world
    own = [[] for _ in range(world)]
    for i in sorted(range(len(weights)), key=lambda j: (-float(weights[j]), j)):
        r = min(range(world), key=lambda q: (load[q], q))
        load[r] += float(weights[i])
        own[r].append(i)
    return sorted(own[rank])


def max_over_ranks(value: float, device=None) -> float:
    """The largest `value` over all ranks (the value itself without a process group)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(device=None):
    import torch
    import torch.distributed as dist

    if dist.is_available() and dist.is_initialized():
        dist.barrier()
    if device is not None and torch.cuda.is_available():
        torch.cuda.synchronize(device)
