"""Multi-process plumbing: one process per GPU under torchrun.

Independent simulations (ensemble instances, serving requests) shard across
ranks with no collective on the data path: each rank runs its own set with
its own seeds, and only the timing is reduced (maximum over ranks).
"""
from __future__ import annotations

import os


def env():
    """(rank, world_size, local_rank) from the torchrun environment."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def rank_seed(seed: int, rank: int) -> int:
    """Seed of a simulation's replica on `rank` (rank 0 keeps the seed)."""
    return int(seed) + 1_000_003 * int(rank)


def shard(n: int, rank: int, world: int) -> range:
    """Items of `n` owned by `rank` (round robin)."""
    return range(rank, n, world)


def max_over_ranks(x: float, device=None) -> float:
    """Maximum of a per-rank scalar over all ranks (identity without a
    process group)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
