"""Replica bookkeeping for running independent analyses on several GPUs.

Every analysis is independent (each rank solves its own problems; no data is
exchanged), so N GPUs run N replicas and the only collectives are the timing
barrier and the max-over-ranks reduction of the elapsed time.
"""
from __future__ import annotations

import os
from typing import Tuple

import torch


def rank_info() -> Tuple[int, int, int]:
    """(world size, rank, local rank) from the torchrun environment."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def max_over_ranks(x: float, device=None) -> float:
    """The maximum of x over all ranks (x itself without a process group)."""
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier() -> None:
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.barrier()


def whole_job_rate(units_per_rank: int, world: int, slowest_ms: float) -> float:
    """Units per second of the whole job: all ranks' units over the slowest rank's time."""
    if slowest_ms <= 0:
        raise ValueError("elapsed time must be positive")
    return world * units_per_rank / (slowest_ms * 1e-3)
