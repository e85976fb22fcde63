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
