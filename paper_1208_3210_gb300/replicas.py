"""Host-side logic of running one benchmark replica per GPU.

Instances of the susceptibility are independent (one band, grid and filling
each), so several GPUs run replicas with no exchange on the data path: each
rank computes its own copy of the workload (weak scaling), and the ranks
meet only to time the run, which is as slow as its slowest rank.  The
rendezvous follows torchrun's environment (RANK, LOCAL_RANK, WORLD_SIZE,
MASTER_ADDR, MASTER_PORT); the collective backend is NCCL on GPUs, gloo for
host-only checks.
"""
from __future__ import annotations

import os


def rank_info():
    """(rank, local_rank, world_size) from the torchrun environment."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0")),
            int(os.environ.get("WORLD_SIZE", "1")))


def max_over_ranks(x: float, world: int, device: str = "cuda") -> float:
    """The largest value of x over all ranks (x itself for one rank); the
    tensor lives on `device` (the backend's device: cuda for NCCL, cpu for
    gloo)."""
    if world == 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank_step: int, world: int, steps: int, max_rank_seconds: float) -> float:
    """Units of all ranks per second when every rank did `steps` steps of
    `units_per_rank_step` units and the slowest took `max_rank_seconds`."""
    return units_per_rank_step * world * steps / max_rank_seconds
