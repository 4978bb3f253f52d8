"""Multi-rank helpers for H v over shots (one process per GPU).

Shots are independent: H_d v = sum over shots of each shot's contribution
(paper section 3: "two wave equations per source").  A rank applies H to v
for its block of shots and the blocks are summed.  The sum is taken in a
fixed rank order on every rank (gather, then add rank 0, 1, ...), so the
result is bitwise the same on all ranks and does not depend on message
arrival order.  On one GPU the world is a single rank and no collective runs.
"""
from __future__ import annotations

import torch
import torch.distributed as dist

__all__ = ["shard_shots", "fixed_order_allreduce", "max_over_ranks"]


def shard_shots(ns: int, rank: int, world: int) -> range:
    """Contiguous block of shots for `rank`: the first ns % world ranks get one more."""
    base, extra = divmod(ns, world)
    start = rank * base + min(rank, extra)
    return range(start, start + base + (1 if rank < extra else 0))


def fixed_order_allreduce(t: torch.Tensor, group=None) -> torch.Tensor:
    """Sum of `t` over ranks, added in rank order 0, 1, ..., world-1 on every rank."""
    if not dist.is_available() or not dist.is_initialized() or dist.get_world_size(group) == 1:
        return t.clone()
    parts = [torch.empty_like(t) for _ in range(dist.get_world_size(group))]
    dist.all_gather(parts, t.contiguous(), group=group)
    out = parts[0].clone()
    for p in parts[1:]:
        out += p
    return out


def max_over_ranks(x: float, device=None, group=None) -> float:
    """Largest value of a host scalar over ranks (timings: the slowest rank sets the time)."""
    if not dist.is_available() or not dist.is_initialized() or dist.get_world_size(group) == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())
