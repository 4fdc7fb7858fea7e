"""Pair sharding across ranks (one process per GPU).

Circuit pairs are independent and pair p is a function of (seed, p) only, so
ranks share nothing on the data path: step s of rank r contracts the pair range
[(s * world + r) * per_rank, +per_rank).  The only collective is the
max-over-ranks of the step time (and, for a global estimate, a sum of the FP64
moments).
"""
from __future__ import annotations


def pair_range(step: int, rank: int, world: int, per_rank: int):
    """First pair index and count of a rank's share of one step."""
    return (step * world + rank) * per_rank, per_rank


def max_over_ranks(value: float, dist=None, device=None) -> float:
    """Maximum of a per-rank scalar over all ranks (identity without a process group)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(values, dist=None, device=None):
    """Element-wise sum of per-rank FP64 moment vectors (identity without a process group)."""
    import torch
    t = torch.as_tensor(values, dtype=torch.float64, device=device).clone()
    if dist is not None and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return t
