"""Replica sharding of shots across ranks (host side).

Shots are independent and every random draw is keyed by (seed, global shot
index), so a run sharded over N ranks decodes exactly the shots of a one-rank
run: rank r of N takes the contiguous range returned by `shot_range`, and the
only exchange is a sum of integer counters (shots, nonconverged, logical,
failures) and a max of the timed seconds.
"""
from __future__ import annotations


def shot_range(rank: int, world: int, steps: int, batch: int, step: int) -> tuple[int, int]:
    """(first global shot index, count) of `step` on `rank`.

    Each rank owns the block [rank * steps * batch, (rank + 1) * steps * batch)
    and walks it in `steps` batches of `batch` shots.
    """
    if not (0 <= rank < world) or not (0 <= step < steps) or batch < 0:
        raise ValueError("rank/step out of range")
    return rank * steps * batch + step * batch, batch


def reduce_counters(counters, seconds: float, group=None):
    """Sum integer counters and take the max of `seconds` over all ranks.

    `counters` is a 1-D torch int64 tensor on the device the process group
    uses (CPU for gloo); returns (summed counters, max seconds).
    """
    import torch
    import torch.distributed as dist
    c = counters.clone()
    t = torch.tensor([seconds], dtype=torch.float64, device=c.device)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1:
        dist.all_reduce(c, op=dist.ReduceOp.SUM, group=group)
        dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return c, float(t.item())
