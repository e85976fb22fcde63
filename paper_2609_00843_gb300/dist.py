"""Rank handling for runs with one process per GPU (torchrun).

The benchmark's step is a set of independent arrays, so N GPUs run N replicas:
every rank sorts arrays of its own (seeds derived from the rank) and nothing
of the sort's data crosses ranks.  The only cross-rank work is timing -- a
barrier on both sides of the timed region and the maximum of the ranks'
elapsed times, from which the whole job's throughput is the units all ranks
processed divided by that maximum.
"""
from __future__ import annotations

import os


def rank_env() -> tuple[int, int, int]:
    """(rank, world size, local rank) from the launcher's environment."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def rank_seed(seed: int, rank: int) -> int:
    """Rank 0 keeps the base seed (its arrays are the single-GPU workload);
    every other rank gets an independent stream."""
    from .gen import derive_seed
    return seed if rank == 0 else derive_seed(seed, rank)


def init(backend: str, device=None) -> None:
    import torch.distributed as dist
    if device is not None:
        dist.init_process_group(backend, device_id=device)
    else:
        dist.init_process_group(backend)


def active() -> bool:
    import torch.distributed as dist
    return dist.is_available() and dist.is_initialized()


def barrier() -> None:
    if active():
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, device=None) -> float:
    """The maximum of `x` over all ranks (x itself without a process group)."""
    if not active():
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank: float, world: int, max_ms: float) -> float:
    """Whole-job units per second: every rank's units over the slowest rank's time."""
    return units_per_rank * world / (max_ms * 1e-3)


def finish() -> None:
    if active():
        import torch.distributed as dist
        dist.destroy_process_group()
