"""Multi-rank helpers for weak scaling over walkers.

Walkers are independent given the pulsar array, so ranks share nothing on the
data path: every rank holds the whole array and its own batch of walkers
(its own seed).  Only timing crosses ranks: the job time is the maximum over
ranks and the job throughput is all ranks' walkers over that time.
"""
from __future__ import annotations


def rank_seed(base_seed: int, rank: int) -> int:
    """Seed of rank `rank`'s walker batch (rank 0 keeps the base seed)."""
    return int(base_seed) + 7919 * int(rank)


def max_over_ranks(value: float, device=None) -> float:
    """Maximum of a float over all ranks of the default process group."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank: int, world: int, seconds: float) -> float:
    """Whole-job units per second under weak scaling."""
    return world * units_per_rank / seconds
