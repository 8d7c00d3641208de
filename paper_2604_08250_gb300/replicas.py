"""Independent replicas across ranks (one process per GPU).

The swap-MC sweep of one lattice runs on one GPU; N GPUs run N independent
replicas (RNG replica index = rank), so there is no data-path collective.
Only the timing is combined: the job takes as long as its slowest rank, and
its throughput counts the attempts of every rank.
"""
from __future__ import annotations


def job_throughput(local_ms: float, attempts_per_rank: float, dist=None, device=None):
    """(attempts/s of the whole job, slowest rank's time in ms).  With an
    initialised torch.distributed process group the local times are reduced
    with MAX (a tensor on `device`, or CPU for gloo)."""
    world = 1
    t_ms = float(local_ms)
    if dist is not None and dist.is_available() and dist.is_initialized():
        import torch
        world = dist.get_world_size()
        t = torch.tensor([t_ms], dtype=torch.float64, device=device if device is not None else "cpu")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        t_ms = float(t.item())
    if t_ms <= 0:
        raise ValueError("elapsed time must be positive")
    return world * float(attempts_per_rank) / (t_ms * 1e-3), t_ms
