"""Rank handling for runs with one process per GPU (torchrun).

The benchmark's step is a set of independent arrays, so N GPUs run N replicas:
every rank sorts arrays of its own (seeds derived from the rank) and nothing
of the sort's data crosses ranks.  The only cross-rank work is timing -- a
barrier on both sides of the timed region and the maximum of the ranks'
elapsed times, from which the whole job's throughput is the units all ranks
processed divided by that maximum.

One array can also be sorted across ranks (sharded).  The sorted output
depends on the global histogram alone (Section 3.1, Algorithms 4 and 7;
Section 3.2, Lemma 3), so rank r, holding the contiguous slice
[r*n/P, (r+1)*n/P) of the input, counts its slice (Algorithm 5), takes part
in one sum all-reduce of the R counts, and writes the same index window of
the sorted array.  No keys cross ranks.
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


# ---------------------------------------------------------------- sharded sort
def slice_bounds(n: int, world: int, rank: int) -> tuple[int, int]:
    """Rank `rank`'s contiguous share [lo, hi) of n items: its input slice and
    its window of the sorted output alike.  The shares tile [0, n) in rank
    order and differ in size by at most one."""
    if world < 1 or not 0 <= rank < world or n < 0:
        raise ValueError(f"bad shard: n={n} world={world} rank={rank}")
    return rank * n // world, (rank + 1) * n // world


def sharded_sort_rank(rank: int, world: int, n_total: int, slice_counts, all_reduce_sum,
                      fill_window):
    """One rank's part of a single array sorted across `world` ranks.

    slice_counts()            -> this rank's counts (R entries) of its slice
    all_reduce_sum(counts)    -> the counts summed over all ranks (the one
                                 exchange; may work in place and return its
                                 argument)
    fill_window(g, lo, hi)    -> positions [lo, hi) of the sorted array whose
                                 global counts are g
    The steps are passed in, so the same partition and exchange logic runs
    over the GPU entry points (ShardedSorter) or over CPU stand-ins in tests.
    Returns whatever fill_window returns.
    """
    lo, hi = slice_bounds(n_total, world, rank)
    counts = slice_counts()
    g = all_reduce_sum(counts)
    return fill_window(g, lo, hi)


class ShardedSorter:
    """Sharded single-array sort on this rank's GPU: rtcdf_hist_accumulate on
    the local slice, a torch.distributed sum all-reduce of the R counts (the
    process group's backend: NCCL across GPUs), rtcdf_fill_from_counts for
    the local window.  Device buffers (counts, workspace) are kept for reuse;
    all work is ordered on `stream` (the collective runs with that stream as
    the current one)."""

    def __init__(self, max_R: int, device=None, stream=None):
        import torch
        from . import rtcdf
        self.torch, self.rtcdf = torch, rtcdf
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None else device
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.max_R = int(max_R)
        self.counts = torch.zeros(self.max_R, dtype=torch.int32, device=self.device)
        self.ws_bytes = rtcdf.rtcdf_workspace_size(self.max_R)
        self.ws = torch.zeros(self.ws_bytes // 4 + 64, dtype=torch.int32, device=self.device)

    def sort(self, in_slice, n_total: int, minVal: int, maxVal: int, out_window,
             rank: int | None = None, world: int | None = None):
        """Sort the array whose slice this rank holds: `in_slice` (int32, this
        rank's share per slice_bounds) in, `out_window` (int32, the same
        length) out.  Returns out_window."""
        torch, rt = self.torch, self.rtcdf
        R = int(maxVal) - int(minVal)
        if not 1 <= R <= self.max_R:
            raise ValueError(f"R={R} outside 1..{self.max_R}")
        if rank is None or world is None:
            rank, world = 0, 1
            if active():
                import torch.distributed as dist
                rank, world = dist.get_rank(), dist.get_world_size()
        lo, hi = slice_bounds(n_total, world, rank)
        if in_slice.numel() != hi - lo or out_window.numel() != hi - lo:
            raise ValueError("slice and window must hold this rank's share of n_total")
        sh = self.stream.cuda_stream
        counts = self.counts[:R]

        def slice_counts():
            with torch.cuda.stream(self.stream):
                counts.zero_()
            rc = rt.rtcdf_hist_accumulate(in_slice.data_ptr() if in_slice.numel() else 0,
                                          in_slice.numel(), int(minVal), int(maxVal),
                                          counts.data_ptr(), sh)
            if rc != rt.OK:
                raise rt.RtcdfError(rc, "rtcdf_hist_accumulate")
            return counts

        def all_reduce_sum(c):
            if world > 1:
                import torch.distributed as dist
                with torch.cuda.stream(self.stream):
                    dist.all_reduce(c, op=dist.ReduceOp.SUM)  # int32 sums wrap like uint32
            return c

        def fill_window(g, a, b):
            rc = rt.rtcdf_fill_from_counts(g.data_ptr(), int(n_total), int(minVal), int(maxVal), a, b,
                                           out_window.data_ptr() if b > a else 0, self.ws.data_ptr(),
                                           self.ws_bytes, sh)
            if rc != rt.OK:
                raise rt.RtcdfError(rc, "rtcdf_fill_from_counts")
            return out_window

        return sharded_sort_rank(rank, world, int(n_total), slice_counts, all_reduce_sum, fill_window)

    def status(self) -> tuple[int, int]:
        """Device status of the fills so far (synchronises the stream)."""
        return self.rtcdf.rtcdf_ws_status_get(self.ws.data_ptr(), self.stream.cuda_stream)
