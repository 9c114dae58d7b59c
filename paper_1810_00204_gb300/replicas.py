"""Host-side logic for running independent plan replicas on several GPUs.

Planning requests are independent (Alg. 1 plans each executed step on its
own), so N GPUs run N disjoint sets of episodes with no data exchange; the
only collective is the timing reduction (max over ranks of the timed region).
"""
from __future__ import annotations

import os
from typing import Tuple

import torch
import torch.distributed as dist


def world() -> Tuple[int, int, int]:
    """(rank, local_rank, world_size) from the launcher's environment."""
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)),
            int(os.environ.get("WORLD_SIZE", 1)))


def episode_range(rank: int, world_size: int, per_rank: int) -> range:
    """Disjoint episode ids of one rank (weak scaling: per_rank fixed)."""
    if not (0 <= rank < world_size) or per_rank < 0:
        raise ValueError("bad rank / world size / per_rank")
    return range(rank * per_rank, (rank + 1) * per_rank)


def reduce_max(x: float, device=None) -> float:
    """Max of a host scalar over all ranks (identity without a process group)."""
    if not (dist.is_available() and dist.is_initialized()):
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def reduce_sum(x: float, device=None) -> float:
    if not (dist.is_available() and dist.is_initialized()):
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def barrier(device=None):
    if dist.is_available() and dist.is_initialized():
        if device is not None and torch.device(device).type == "cuda":
            dist.barrier(device_ids=[torch.device(device).index])
        else:
            dist.barrier()
