"""Multi-process bookkeeping for independent renders on several GPUs.

Each rank solves its own image (a different seed): there is no data-path
collective. Only the timing is combined: the job's time is the maximum over
ranks and its work the sum over ranks.
"""
from __future__ import annotations

import torch
import torch.distributed as dist


def combine_throughput(local_seconds: float, local_units: float, device=None):
    """(max seconds over ranks, total units over ranks); identity on 1 rank."""
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(local_seconds), float(local_units)
    t = torch.tensor([float(local_seconds)], dtype=torch.float64, device=device)
    u = torch.tensor([float(local_units)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def rank_seed(base_seed: int, rank: int) -> int:
    """Seed of rank's independent render."""
    return int(base_seed) + 1000003 * int(rank)
