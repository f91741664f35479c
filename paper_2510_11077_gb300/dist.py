"""Multi-rank helpers for weak scaling over walkers.

Walkers are independent given the pulsar array, so ranks share nothing on the
data path: every rank holds the whole array and its own batch of walkers
(its own seed).  Only timing crosses ranks: the job time is the maximum over
ranks and the job throughput is all ranks' walkers over that time.
"""
from __future__ import annotations

import os


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


def env() -> tuple[int, int, int]:
    """(world size, rank, local rank) from the launcher's environment (1, 0, 0
    when run as a single process)."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def barrier() -> None:
    """Barrier over the default process group; a no-op for a single process."""
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.barrier()


def timed_steps(run_step, steps: int, warmup: int, sync=None, resolve=None, on_start=None,
                device=None):
    """The timing protocol of a weak-scaling run, the same on every rank:
    `warmup` untimed steps, then sync + barrier, then `steps` timed steps,
    then sync + barrier.  run_step(timed) runs one step and, when timed,
    returns its measurement; resolve(list) turns the measurements into
    seconds after the closing sync (CUDA events; identity by default);
    on_start() runs right before the timed steps (e.g. a clock sampler).
    Returns (this rank's per-step seconds, the job time = the maximum over
    ranks of each rank's total)."""
    sync = sync or (lambda: None)
    resolve = resolve or (lambda m: list(m))
    for _ in range(max(warmup, 0)):
        run_step(False)
    sync()
    if on_start:
        on_start()
    barrier()
    sync()
    meas = [run_step(True) for _ in range(steps)]
    sync()
    barrier()
    secs = [float(x) for x in resolve(meas)]
    return secs, max_over_ranks(sum(secs), device=device)
