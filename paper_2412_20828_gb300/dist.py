"""Frame sharding across ranks (one process per GPU).

Frames are independent, so the decoder shards by frame index with no data-path
collective: rank r decodes its own frames, numbered from ``frame_base(r)`` so the
synthetic frames and automorphism draws of every rank are disjoint and identical to a
single-process run over the same indices.  Only bookkeeping crosses ranks: the
slowest rank's time (max) and the error counters (sum).
"""
from __future__ import annotations

import os

FRAMES_PER_RANK_SPAN = 1_000_000_000  # frame-index span reserved per rank


def env_ranks():
    """(rank, world_size, local_rank) from the torchrun environment (1 process: 0, 1, 0)."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def frame_base(rank: int) -> int:
    return rank * FRAMES_PER_RANK_SPAN


def max_over_ranks(value: float, device=None) -> float:
    """The largest value over all ranks (the job's wall time is the slowest rank's)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(tensor):
    """In-place sum of integer counters over ranks; returns the tensor."""
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(tensor, op=dist.ReduceOp.SUM)
    return tensor


def job_throughput(units_per_rank: int, world: int, slowest_seconds: float) -> float:
    """Whole-job throughput: all ranks' units over the slowest rank's time."""
    return units_per_rank * world / slowest_seconds
