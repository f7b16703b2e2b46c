"""Replica bookkeeping for runs on several GPUs of one node.

Every solve here is independent (one system or batch per GPU, no data-path collective), so a
multi-GPU run is N replicas: each rank times its own work, the job's time is the maximum over
ranks, and throughput counts the work of all ranks. Only host-side control collectives are used
(a barrier and a max-reduction of one number).
"""
from __future__ import annotations

import os


def world() -> tuple[int, int, int]:
    """(rank, local_rank, world_size) from the torchrun environment (1 process by default)."""
    return int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0")), int(os.environ.get("WORLD_SIZE", "1"))


def barrier(dist) -> None:
    if dist is not None and dist.is_available() and dist.is_initialized():
        dist.barrier()


def max_over_ranks(dist, value: float, device=None) -> float:
    """Maximum of `value` over all ranks (identity without an initialised process group)."""
    if dist is None or not dist.is_available() or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_throughput(dist, units_per_rank: int, seconds: float, device=None) -> tuple[float, float]:
    """Whole-job throughput: (units of all ranks) / (max time over ranks). Returns (value, max_time)."""
    tmax = max_over_ranks(dist, seconds, device)
    n = dist.get_world_size() if (dist is not None and dist.is_available() and dist.is_initialized()) else 1
    return n * units_per_rank / tmax, tmax
