"""Replica (data-parallel) bookkeeping for several GPUs.

Rays and views are independent and the table is read-only, so each rank
renders its own frames from its own copy of the table; no data-path
collective exists. The only collective is the reduction of the per-rank timing
(the slowest rank bounds the job) and of the per-rank ray counts.
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
