"""Weak scaling over independent signals.

The hot path partitions into independent signals, so ranks never exchange data:
each rank recovers its own signals (seed offsets disjoint across ranks) and the
ranks share only a barrier and the max / sum of a few timing scalars.
"""
from __future__ import annotations

import os

SEED_STRIDE = 1000   # signals per rank stay below this, so rank offsets never overlap


def world_info():
    """(world_size, rank, local_rank) from the torchrun environment (1, 0, 0 when absent)."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def rank_seed_offsets(rank: int, per_rank: int) -> list:
    """Seed offsets of the signals rank `rank` recovers."""
    if per_rank > SEED_STRIDE:
        raise ValueError("at most %d signals per rank" % SEED_STRIDE)
    return [SEED_STRIDE * rank + b for b in range(per_rank)]


def _reduce(value: float, op: str, device: str) -> float:
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())


def max_over_ranks(value: float, device: str = "cuda") -> float:
    return _reduce(value, "max", device)


def sum_over_ranks(value: float, device: str = "cuda") -> float:
    return _reduce(value, "sum", device)


def barrier():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.barrier()
