"""Replicas across GPUs: each rank computes its own clouds, no collective on
the data path.  One cloud is never split across GPUs; a step's time is the
maximum over ranks and the job's throughput is every rank's units over that
time (weak scaling)."""
from __future__ import annotations

import os


def rank_world():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def replica_seed(base: int, rank: int) -> int:
    """Seed of rank `rank`'s cloud: distinct, reproducible replicas."""
    return base + rank


def max_over_ranks(value: float, device=None) -> float:
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank: int, world: int, step_ms_max: float) -> float:
    """Units of all ranks per second of the slowest rank."""
    return world * units_per_rank / (step_ms_max * 1e-3)
