"""Host-side logic for running on several GPUs of one node.

The ChFSI path shards by independent problems (whole sequences, or the
k-point-style problems of a batch): each rank solves its own share with no
data-path collective.  The only collectives are the timing reduction (max
over ranks) and a barrier; they run on whatever backend the process group
uses (NCCL on GPUs, gloo on the CPU).
"""
from __future__ import annotations

import os


def env():
    """(world_size, rank, local_rank) from the torchrun environment."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def shard(num_items: int, rank: int, world: int) -> list:
    """Round-robin share of items 0..num_items-1 for `rank`."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank/world")
    return list(range(rank, num_items, world))


def max_over_ranks(value: float, device=None) -> float:
    """Maximum of a per-rank scalar (a no-op without a process group)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value: float, device=None) -> float:
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def whole_job_seconds_per_unit(units_this_rank: int, seconds_this_rank: float, device=None):
    """Seconds per unit of the whole job: all ranks' units over the slowest
    rank's time (weak scaling: every rank brings its own units)."""
    total = sum_over_ranks(units_this_rank, device)
    t = max_over_ranks(seconds_this_rank, device)
    return t / max(total, 1.0), t, total
