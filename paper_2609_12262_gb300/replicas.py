"""Multi-GPU replicas: shots are independent, so N ranks (one per GPU) each decode
their own shard and meet only to time the job (barrier, maximum over ranks).
There is no collective on the data path."""

from __future__ import annotations

import os


def world() -> tuple[int, int, int]:
    """(world_size, rank, local_rank) from the torchrun environment."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def shard(num_units: int, world_size: int, rank: int) -> tuple[int, int]:
    """Contiguous [begin, end) of `num_units` owned by `rank` (sizes differ by at most 1)."""
    base, extra = divmod(num_units, world_size)
    begin = rank * base + min(rank, extra)
    return begin, begin + base + (1 if rank < extra else 0)


def shard_seed(seed: int, rank: int) -> int:
    """Seed of rank `rank`'s own generated input batch (weak scaling)."""
    return seed + 1000 * rank


def max_over_ranks(value: float, device=None) -> float:
    """Maximum of a per-rank number over all ranks (identity without a process group)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
