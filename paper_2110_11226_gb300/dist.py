"""Multi-GPU generation step: the population is sharded by programs.

Rank r holds programs [r*P_local, (r+1)*P_local) of a global population of
world*P_local programs and evaluates them on the full dataset (rows are not
split, so no partial sums cross GPUs).  Selection needs every fitness value
(Sec. III-C1: tournaments draw from the whole population), so the one
exchange is an all-gather of the per-rank fitness vectors; every rank then
runs the same tournaments over the gathered vector and gets the same
winners.  Timing helpers take the maximum over ranks.
"""
from __future__ import annotations

import torch
import torch.distributed as dist


def shard_bounds(n_total: int, world: int, rank: int):
    """Contiguous, balanced program shard [start, end) of rank `rank`."""
    base, extra = divmod(n_total, world)
    start = rank * base + min(rank, extra)
    return start, start + base + (1 if rank < extra else 0)


def gather_fitness(fit_local: torch.Tensor, group=None) -> torch.Tensor:
    """All-gather equal-sized fitness shards into the global vector (rank order)."""
    world = dist.get_world_size(group)
    if world == 1:
        return fit_local
    parts = [torch.empty_like(fit_local) for _ in range(world)]
    dist.all_gather(parts, fit_local.contiguous(), group=group)
    return torch.cat(parts)


def max_over_ranks(x: float, device=None) -> float:
    if not dist.is_initialized() or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
