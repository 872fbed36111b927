"""Replica (data-parallel) bookkeeping for several GPUs.

Rendering: rays and views are independent and the table is read-only, so each
rank renders its own frames from its own copy of the table; no data-path
collective exists, only the reductions of the per-rank timing (the slowest rank
bounds the job) and ray counts.

Fitting: each rank renders its shard of the target views and accumulates its
part of the gradient table; one all-reduce (sum) of that table per step makes
every replica take the same optimiser step (the exchange step of a
data-parallel fit).
"""
from __future__ import annotations

from typing import List


def frames_for_rank(rank: int, world: int, count: int, total_frames: int) -> List[int]:
    """`count` consecutive orbit frames for `rank`; ranks take disjoint blocks
    (modulo the orbit length)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank/world")
    return [(rank * count + k) % total_frames for k in range(count)]


def reduce_max(value: float) -> float:
    """Max over ranks (identity without an initialised process group)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def reduce_sum(value: float) -> float:
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def shard(items, rank: int, world: int):
    """The contiguous block of `items` of `rank` (sizes differ by at most one)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank/world")
    n = len(items)
    lo = rank * n // world
    hi = (rank + 1) * n // world
    return items[lo:hi]


def allreduce_sum_(t):
    """In-place sum over ranks of a tensor (identity without a process group)."""
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return t
