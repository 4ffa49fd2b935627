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


def gather_fitness(fit_local: torch.Tensor, group=None, n_total=None) -> torch.Tensor:
    """All-gather the fitness shards into the global vector (rank order).

    Shards from shard_bounds differ by at most one program when the world
    size does not divide the population; all_gather needs equal sizes, so
    every shard is padded to the largest (ceil(n_total / world)) and each
    rank's part is trimmed back to its own length afterwards.  n_total
    defaults to world * len(fit_local) (equal shards)."""
    world = dist.get_world_size(group)
    if world == 1:
        return fit_local
    if n_total is None:
        n_total = world * fit_local.numel()
    cap = -(-n_total // world)
    sizes = [shard_bounds(n_total, world, r) for r in range(world)]
    sizes = [b - a for a, b in sizes]
    rank = dist.get_rank(group)
    if fit_local.numel() != sizes[rank]:
        raise ValueError(f"rank {rank} holds {fit_local.numel()} fitness values, "
                         f"its shard of {n_total} has {sizes[rank]}")
    padded = torch.full((cap,), float("nan"), dtype=fit_local.dtype, device=fit_local.device)
    padded[:fit_local.numel()] = fit_local
    parts = [torch.empty_like(padded) for _ in range(world)]
    dist.all_gather(parts, padded, group=group)
    return torch.cat([part[:n] for part, n in zip(parts, sizes)])


def max_over_ranks(x: float, device=None) -> float:
    if not dist.is_initialized() or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
