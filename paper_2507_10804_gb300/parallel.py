"""Multi-rank H v over shots (one process per GPU).

Shots are independent: H_d v = E^T sum over shots of each shot's extended
image (paper section 3: two wave equations per source; eq. (grad) sums the
imaging over sources).  A rank owns a contiguous block of shots
(``shard_shots``), computes the extended image of its block in FP64 on the
padded grid (``Problem.hessian_apply_partial``), the images are summed in a
fixed rank order on every rank (gather, then add rank 0, 1, ...: bitwise the
same on all ranks, independent of message arrival order), and the sum is
folded onto the interior once (``Problem.fold``).  That sum is the one
exchange step of the split.  On one GPU the world is a single rank and no
collective runs.
"""
from __future__ import annotations

import torch
import torch.distributed as dist

__all__ = ["shard_shots", "fixed_order_allreduce", "max_over_ranks", "sharded_hessian_apply", "shard_problem"]


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


def sharded_hessian_apply(partial, fold, group=None):
    """H_d v over every rank's shot block: ``partial()`` returns this rank's extended image (FP64),
    the images are summed in rank order on every rank, ``fold(ext)`` maps the sum onto the interior."""
    return fold(fixed_order_allreduce(partial(), group))


def shard_problem(problem_cls, w, rank: int, world: int, device=None):
    """The Problem of workload ``w`` restricted to this rank's block of shots (``shard_shots``)."""
    idx = list(shard_shots(w.ns, rank, world))
    a = w.acq
    return problem_cls(w.nz, w.nx, w.nb, w.h, w.nt, w.dt, w.f0, w.t0, w.vmax, a.src_iz[idx], a.src_ix[idx],
                       a.rec_iz[idx], a.rec_ix[idx], R=w.R, sigma=w.sigma, device=device)
