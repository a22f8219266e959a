"""Shot parallelism across ranks (Sec. 2.3: shots are independent).

Each rank models a contiguous block of shots; the only exchange is the sum
over shots of the velocity gradient and of the misfit, one all-reduce per
gradient evaluation.  Pure host logic over ``torch.distributed``; the solver
itself runs per rank.
"""
from __future__ import annotations

import torch
import torch.distributed as dist


def shard(nshot: int, rank: int, world: int) -> slice:
    """Contiguous block of shots of `rank` (sizes differ by at most one)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank/world")
    base, extra = divmod(nshot, world)
    start = rank * base + min(rank, extra)
    return slice(start, start + base + (1 if rank < extra else 0))


def reduce_gradient(grad: torch.Tensor, misfit: torch.Tensor, group=None) -> None:
    """Sum the per-rank gradients and misfits in place over the group."""
    if dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1:
        dist.all_reduce(grad, op=dist.ReduceOp.SUM, group=group)
        dist.all_reduce(misfit, op=dist.ReduceOp.SUM, group=group)
