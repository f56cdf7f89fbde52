"""Multi-process helpers: the systems of a batch are independent, so a batch is
sharded across ranks with no collective on the data path (weak scaling).  The
one exchange is the gradient with respect to the shared matrix's coefficient,
a sum over every system of the batch: it is combined across ranks in rank
order, so the result does not depend on the reduction order of the backend.

All functions take an optional ``group`` and work with any torch.distributed
backend (NCCL between GPUs, gloo on CPUs).
"""
from __future__ import annotations

import torch
import torch.distributed as dist


def shard(M_total: int, rank: int, world: int):
    """(start, count) of the systems owned by ``rank``: contiguous, balanced to
    within one system, in rank order."""
    if world < 1 or not 0 <= rank < world or M_total < 0:
        raise ValueError("bad shard request")
    base, extra = divmod(M_total, world)
    count = base + (1 if rank < extra else 0)
    start = rank * base + min(rank, extra)
    return start, count


def sum_in_rank_order(value: torch.Tensor, group=None) -> torch.Tensor:
    """Sum of ``value`` (same shape on every rank) over the ranks, added in rank
    order 0, 1, ... so every rank gets the same bits on every run."""
    if not dist.is_available() or not dist.is_initialized():
        return value.clone()
    world = dist.get_world_size(group)
    parts = [torch.empty_like(value) for _ in range(world)]
    dist.all_gather(parts, value.contiguous(), group=group)
    total = parts[0].clone()
    for p in parts[1:]:
        total += p
    return total


def max_over_ranks(x: float, device=None, group=None) -> float:
    """The largest of a scalar over the ranks (the slowest rank's time)."""
    if not dist.is_available() or not dist.is_initialized():
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())


def batch_mean_in_rank_order(local_mean: torch.Tensor, local_count: int, total_count: int,
                             group=None) -> torch.Tensor:
    """The mean over every system of the batch of a per-step statistic that each rank
    has averaged over its own ``local_count`` systems (the coarsening length of
    section 5.3, one value per step): sum_r count_r * mean_r / total, combined in
    rank order so every rank gets the same bits."""
    if total_count < 1:
        raise ValueError("the batch is empty")
    weighted = local_mean.to(torch.float64) * float(local_count)
    return sum_in_rank_order(weighted, group) / float(total_count)
