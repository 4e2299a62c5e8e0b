"""Agent-parallel sharding across ranks (one process per GPU).

Agents are independent within a step, so the forward rollout needs no
communication: each rank owns a contiguous range of agents cut at group
boundaries where possible.  The adjoint has one exchange: the per-group
parameter gradients (n_groups x 16 floats) and the scalar loss are summed
over ranks after the backward pass.
"""
from __future__ import annotations

import numpy as np
import torch
import torch.distributed as dist


def shard_range(n: int, rank: int, world: int) -> tuple[int, int]:
    """Contiguous [lo, hi) of n agents for this rank, sizes differing by at most one."""
    base, extra = divmod(n, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def shard_by_groups(gid: np.ndarray, world: int) -> list[tuple[int, int]]:
    """Contiguous ranges for sorted group ids, cut at group boundaries when every rank still gets work."""
    n = int(gid.size)
    cuts = [shard_range(n, r, world) for r in range(world)]
    if n == 0 or np.any(np.diff(gid.astype(np.int64)) < 0):
        return cuts
    starts = np.flatnonzero(np.diff(gid.astype(np.int64))) + 1
    bounds = [0]
    for r in range(1, world):
        target = cuts[r][0]
        cand = starts[np.argmin(np.abs(starts - target))] if starts.size else target
        b = int(cand) if abs(int(cand) - target) <= n // (4 * world) else target
        bounds.append(max(b, bounds[-1]))
    bounds.append(n)
    return [(bounds[r], bounds[r + 1]) for r in range(world)]


def allreduce_grads(dtheta: torch.Tensor, loss: torch.Tensor | None = None):
    """Sum per-group parameter gradients (and the loss) over ranks, in place."""
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(dtheta, op=dist.ReduceOp.SUM)
        if loss is not None:
            dist.all_reduce(loss, op=dist.ReduceOp.SUM)
    return dtheta, loss
