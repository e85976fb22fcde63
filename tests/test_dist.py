"""The multi-rank path of the benchmark on CPU: two gloo ranks (one process
each) exercise the rank helpers the GPU run uses -- per-rank seeds, the
barrier, the maximum of the ranks' times and the whole-job throughput -- and
each rank sorts its own arrays with the oracle, which must differ between
ranks (independent replicas) and be correct."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2609_00843_gb300 import dist as rdist


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import oracle
    from paper_2609_00843_gb300 import gen
    r, w, lr = rdist.rank_env()
    assert (r, w, lr) == (rank, world, rank)
    rdist.init("gloo")
    try:
        seed = rdist.rank_seed(gen.derive_seed(1, 0, 7), r)
        keys = gen.keys_host(5000, -1000, 128, gen.UNIFORM, seed)
        srt = oracle.counting_sort(keys, -1000, -1000 + 128)
        assert np.array_equal(srt, np.sort(keys))
        rdist.barrier()
        elapsed = 1.0 + 2.0 * r          # this rank's "time"
        mx = rdist.max_over_ranks(elapsed)
        out.put((r, seed, int(srt[:64].sum()), mx,
                 rdist.job_throughput(5000, w, mx * 1e3)))
    finally:
        rdist.finish()


def test_two_gloo_ranks_replicas_and_max_timing():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    res = sorted(q.get(timeout=10) for _ in range(2))
    (r0, s0, h0, m0, t0), (r1, s1, h1, m1, t1) = res
    assert (r0, r1) == (0, 1)
    assert s0 != s1                         # independent arrays per rank
    assert m0 == m1 == 3.0                  # max over ranks, same on both
    assert t0 == t1 == pytest.approx(2 * 5000 / 3.0)


def test_single_process_helpers_without_group():
    assert not rdist.active()
    assert rdist.max_over_ranks(4.5) == 4.5
    rdist.barrier()
    assert rdist.rank_seed(123, 0) == 123 and rdist.rank_seed(123, 1) != 123
    assert rdist.job_throughput(1e8 * 12, 1, 2.0) == pytest.approx(6e11)


# ---------------------------------------------------------------- sharded sort
def _shard_main(rank, world, port, n, minVal, R, dist_kind, seed, out):
    """One rank of a sharded sort on CPU: its slice of the seeded array is
    counted (the oracle's histogram stands in for the GPU count), the counts
    are summed over the gloo ranks (the real exchange), and the rank's window
    of the sorted array is produced from the global counts (the oracle's
    output rule stands in for the GPU fill)."""
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import torch
    import torch.distributed as dist
    import oracle
    from paper_2609_00843_gb300 import gen
    rdist.init("gloo")
    try:
        lo, hi = rdist.slice_bounds(n, world, rank)
        mine = gen.keys_host(hi - lo, minVal, R, dist_kind, seed, first=lo)
        seen = {}

        def slice_counts():
            c = torch.from_numpy(oracle.histogram(mine, minVal, minVal + R).astype(np.int64))
            seen["local"] = c.clone()
            return c

        def all_reduce_sum(c):
            dist.all_reduce(c, op=dist.ReduceOp.SUM)
            return c

        def fill_window(g, a, b):
            cdf = np.cumsum(g.numpy().astype(np.uint64))
            return oracle.values_at(cdf, minVal, np.arange(a, b, dtype=np.uint64))

        window = rdist.sharded_sort_rank(rank, world, n, slice_counts, all_reduce_sum, fill_window)
        out.put((rank, lo, hi, window, seen["local"].numpy()))
    finally:
        rdist.finish()


@pytest.mark.parametrize("world,n,R,kind", [(2, 200_003, 1 << 12, 1), (2, 3, 5, 0), (3, 100_000, 1, 2),
                                            (4, 50_001, 1 << 18, 0)])
def test_sharded_sort_over_gloo_ranks_matches_oracle(world, n, R, kind):
    import oracle
    from paper_2609_00843_gb300 import gen
    minVal = -777
    seed = gen.derive_seed(60, world, R, kind)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_shard_main, args=(r, world, port, n, minVal, R, kind, seed, q))
             for r in range(world)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=300) for _ in range(world)), key=lambda t: t[0])
    for p in procs:
        p.join(timeout=120)
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    full = gen.keys_host(n, minVal, R, kind, seed)
    want = oracle.counting_sort(full, minVal, minVal + R)
    # The windows tile [0, n) in rank order, each rank counted exactly its own
    # slice, and together the windows are the oracle's sorted array.
    assert [(r[1], r[2]) for r in res] == [rdist.slice_bounds(n, world, k) for k in range(world)]
    for rank, lo, hi, window, local in res:
        assert np.array_equal(local, oracle.histogram(full[lo:hi], minVal, minVal + R).astype(np.int64))
        assert np.array_equal(window, want[lo:hi]), f"rank {rank} window [{lo}, {hi}) differs"
    assert np.array_equal(np.concatenate([r[3] for r in res]), want)


def test_slice_bounds_tile_the_array():
    for n in (0, 1, 7, 100, 10**9 + 7):
        for world in (1, 2, 3, 8):
            b = [rdist.slice_bounds(n, world, r) for r in range(world)]
            assert b[0][0] == 0 and b[-1][1] == n
            assert all(b[i][1] == b[i + 1][0] for i in range(world - 1))
            assert max(h - l for l, h in b) - min(h - l for l, h in b) <= 1
    with pytest.raises(ValueError):
        rdist.slice_bounds(10, 2, 2)
