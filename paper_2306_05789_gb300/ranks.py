"""Process-per-GPU helpers for the benchmark and other multi-rank drivers.

The method shards without any data exchange: independent problems (batches,
served requests) are split across ranks, and a single problem runs as one
replica per GPU.  The only collectives are outside the data path: a barrier
around timed regions and the maximum of the ranks' times.
"""
from __future__ import annotations

import os


def rank_env():
    """(rank, world, local_rank) from the torchrun environment (1 process: 0, 1, 0)."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def shard_range(count: int, rank: int, world: int):
    """Contiguous share [lo, hi) of `count` units for `rank`; shares differ by at most one."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("need 0 <= rank < world")
    base, extra = divmod(count, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def instance_seed(seed: int, rank: int) -> int:
    """Seed of rank `rank`'s own draw of instances (weak scaling: every rank a full set)."""
    return seed + 1000003 * rank


def max_over_ranks(value: float, device=None) -> float:
    """Maximum of `value` over the default process group (the value itself without one)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.barrier()
