"""Timing bookkeeping for independent replicas on several GPUs.

Replicas exchange no data (each rank integrates its own system); only the
benchmark's bookkeeping crosses ranks: the slowest rank's time and the sum
of the interactions.  Works with
any torch.distributed backend (NCCL on GPUs, gloo on CPU).
"""
from __future__ import annotations


def combine_timing(ms: float, interactions: float, device=None) -> tuple[float, float]:
    """(max over ranks of ms, sum over ranks of interactions); identity when
    torch.distributed is not initialised."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(ms), float(interactions)
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    i = torch.tensor([float(interactions)], dtype=torch.float64, device=device)
    dist.all_reduce(i, op=dist.ReduceOp.SUM)
    return float(t.item()), float(i.item())
