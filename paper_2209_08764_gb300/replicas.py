"""Multi-GPU runs of the level step: independent replicas, one per GPU.

A traversal does not shard across GPUs in this library (one GPU holds the
whole graph; there is no exchange step), so N GPUs run N independent
replicas, each on its own sources (weak scaling).  The only collective is on
the timing: the slowest rank's time and the total work of all ranks.
"""
from __future__ import annotations


def aggregate(dist, local_ms: float, local_units: float, device=None) -> tuple[float, float]:
    """(max of local_ms over ranks, sum of local_units over ranks).

    ``dist`` is ``torch.distributed`` (initialised) or None for one process;
    ``device`` the tensor device of the process group's backend (a CUDA
    device for NCCL, None for gloo on the CPU).
    """
    if dist is None:
        return float(local_ms), float(local_units)
    import torch
    t = torch.tensor([float(local_ms)], dtype=torch.float64, device=device)
    u = torch.tensor([float(local_units)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def rank_source_seed(base_seed: int, rank: int) -> int:
    """Seed of the sources rank ``rank`` traverses: each replica draws its own
    (offset 1000 per rank), so N replicas do N times the work."""
    return int(base_seed) + 1000 * int(rank)
