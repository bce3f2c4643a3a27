"""Sharding of Monte-Carlo shots over ranks (one process per GPU).

Shots are independent and the sampler is counter-based (shot k's errors
depend only on the seed and k), so ranks take disjoint shot ranges and the
only exchange is a sum of failure / work counters and the max of the timed
region over ranks, once after timing.  The functions take the
``torch.distributed`` module so the same code runs on NCCL (GPUs) and gloo
(CPU tests).
"""
from __future__ import annotations


def first_shot(step: int, rank: int, world: int, ip: int, n_p: int, shots: int) -> int:
    """First shot index of rank `rank` for error rate number `ip` (of `n_p`)
    in step `step`: ranges of `shots` shots, step-major, then rank, then p,
    so every (step, rank, p) range is disjoint from every other."""
    return ((step * world + rank) * n_p + ip) * shots


def reduce_counters(dist, *tensors) -> None:
    """Sum counter tensors over ranks in place (no-op on one rank)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return
    for t in tensors:
        dist.all_reduce(t)


def max_over_ranks(dist, value: float, device) -> float:
    """The largest `value` over ranks (the timed region's max)."""
    import torch
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
