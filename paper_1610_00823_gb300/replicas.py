"""Replica-parallel runs (one independent tree per GPU, no data exchange): the host-side
cross-rank steps of a timed run, backend-agnostic (NCCL on GPUs, gloo on CPU).

A multi-GPU run of the box code here is replicas only: every rank solves its own problem, so the
only collective work is a barrier around the timed region and the maximum of the per-rank times.
"""
from __future__ import annotations

import torch


def _device(dist):
    return torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl" else torch.device("cpu")


def barrier(dist) -> None:
    """Barrier over all ranks (no-op without a process group)."""
    if dist is not None:
        dist.barrier()


def max_over_ranks(x: float, dist) -> float:
    """The largest of the ranks' values (the run's time is its slowest rank's)."""
    if dist is None:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=_device(dist))
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, ms_max: float, world: int) -> float:
    """Units per second of the whole job: every rank processes units_per_rank in ms_max ms."""
    return world * units_per_rank / (ms_max / 1e3)
