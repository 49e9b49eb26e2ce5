"""Multi-GPU form of the hot path: one process per GPU.

Views are independent problems, so each rank renders its own views with its
own copy of the octree and the grid (weak scaling, no collective on the data
path).  The exchange a training loop would add after the backward is the
sum of the FP32 table gradients over ranks; ``sum_table_grad`` is that step.
"""
from __future__ import annotations

import torch
import torch.distributed as dist


def _world() -> int:
    return dist.get_world_size() if dist.is_available() and dist.is_initialized() else 1


def view_ids(rank: int, world: int, step: int, views_per_rank: int = 1) -> list:
    """View ids rendered by ``rank`` at ``step``: disjoint across ranks and
    steps, and the same set of views for every world size at a given total
    view count."""
    if not 0 <= rank < world:
        raise ValueError("rank %d outside a world of %d" % (rank, world))
    base = (step * world + rank) * views_per_rank
    return list(range(base, base + views_per_rank))


def max_over_ranks(x: float, device=None) -> float:
    """Largest value of ``x`` over all ranks (the job's time is its slowest rank's)."""
    if _world() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_table_grad(grad: torch.Tensor) -> torch.Tensor:
    """In-place sum of every rank's FP32 table gradient."""
    if grad.dtype != torch.float32:
        raise TypeError("the table gradient is FP32")
    if _world() > 1:
        dist.all_reduce(grad, op=dist.ReduceOp.SUM)
    return grad
