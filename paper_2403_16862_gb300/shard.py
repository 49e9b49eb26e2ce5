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


class GradExchange:
    """The table-gradient exchange of a multi-GPU step, overlapped with the
    next view's forward.

    Two FP32 gradient tables alternate between steps.  Step k's backward
    accumulates into table k % 2 (``begin``); ``launch`` then starts the sum
    over ranks of that table as an asynchronous collective (NCCL runs it on
    its own stream after the backward's kernels, gloo on a host thread), and
    the caller goes on with step k + 1's forward.  Before step k + 2 clears
    the same table, ``begin`` waits for step k's collective, so a gradient is
    always summed before the next backward writes that table.  ``result(k)``
    waits for step k's sum and returns it (valid until step k + 2 begins);
    ``finish`` waits for every collective in flight.  With one rank the
    collective is skipped and each table holds the rank's own gradient."""

    def __init__(self, shape, device=None):
        self.bufs = [torch.zeros(shape, dtype=torch.float32, device=device) for _ in range(2)]
        self.work = [None, None]
        self.step = -1

    def _wait(self, i):
        if self.work[i] is not None:
            self.work[i].wait()
            self.work[i] = None

    def begin(self) -> torch.Tensor:
        self.step += 1
        i = self.step % 2
        self._wait(i)  # step - 2's sum of this table is complete
        self.bufs[i].zero_()
        return self.bufs[i]

    def launch(self):
        i = self.step % 2
        if _world() > 1:
            self.work[i] = dist.all_reduce(self.bufs[i], op=dist.ReduceOp.SUM, async_op=True)

    def result(self, step: int) -> torch.Tensor:
        if not 0 <= self.step - step <= 1:
            raise ValueError("step %d's table has been reused (current step %d)" % (step, self.step))
        self._wait(step % 2)
        return self.bufs[step % 2]

    def finish(self):
        for i in range(2):
            self._wait(i)
