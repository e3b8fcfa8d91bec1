"""Whole-job throughput of independent replicas, one per GPU (one process
per GPU; the systems never exchange data, so no collective runs on the data
path).  Each rank times its own replica; the job's time is the slowest
rank's, and its work is the sum over ranks (weak scaling)."""
from __future__ import annotations


def aggregate(units: float, ms: float, device=None):
    """(units of all ranks / max-over-ranks time in seconds, max ms).

    Without an initialised process group this is the single-process value.
    `device` is where the two reduction scalars live: the rank's GPU under
    NCCL, the CPU under gloo."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return units / (ms / 1000.0), ms
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    u = torch.tensor([units], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(u.item()) / (float(t.item()) / 1000.0), float(t.item())


def replica_seed(rank: int, base: int = 0) -> int:
    """Seed of rank's replica: every rank simulates a different system."""
    return base + rank
