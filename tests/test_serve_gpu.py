"""Continuous-batching server: every request's result is the same alone (served
one at a time) and in the mix (admitted while others run, batched with them),
and matches the CPU oracle -- bit-exact.  Whole traces are compared through
order-dependent digests of the sorted outputs; selected requests' outputs are
copied back from the server and compared with the oracle element by element.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_2609_00843_gb300 import _build, gen, rtcdf

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    _build.build()
    torch.cuda.init()


def trace(count, seed, n_hi=3e6, rate=20000.0, r_hi=2 ** 18):
    n, mn, R, dist, seeds = gen.serving_requests(seed, count, n_lo=1e3, n_hi=n_hi, r_hi=r_hi)
    arr = gen.poisson_arrivals(seed, count, rate)
    return n, mn, R, dist, seeds, arr


def config(budget, digests=True, streams=4, max_batch=64, single_min=1 << 21, max_large=0, prio=0):
    return rtcdf.ServerConfig(budget_bytes=budget, num_streams=streams, max_batch=max_batch,
                              single_min_keys=single_min, fill=gen.fill_function_address(),
                              digests=1 if digests else 0, max_large_inflight=max_large,
                              large_priority=prio)


def output_buffers(n, chosen):
    """Host buffers for the requests in `chosen` and the pointer array the
    server copies their sorted outputs to (NULL for the others)."""
    bufs = {int(i): np.full(int(n[i]), 0x7FFFFFFF, dtype=np.int32) for i in chosen}
    ptrs = (ctypes.c_void_p * len(n))()
    for i, b in bufs.items():
        ptrs[i] = b.ctypes.data
    return bufs, ptrs


def assert_outputs_match_oracle(bufs, n, mn, R, dist, seeds):
    for i, got in bufs.items():
        a = gen.keys_host(int(n[i]), int(mn[i]), int(R[i]), int(dist[i]), int(seeds[i]))
        want = oracle.counting_sort(a, int(mn[i]), int(mn[i]) + int(R[i]))
        bad = np.nonzero(got != want)[0]
        assert bad.size == 0, (f"request {i} (n={n[i]}, R={R[i]}): {bad.size} positions differ "
                               f"from the oracle, first {bad[:8].tolist()}")


def oracle_digest(n, mn, R, dist, seed):
    a = gen.keys_host(int(n), int(mn), int(R), int(dist), int(seed))
    return gen.digest(oracle.counting_sort(a, int(mn), int(mn) + int(R)))


def test_digest_definition_matches_device():
    """The device digest of a sorted output equals the numpy digest."""
    n, mn, R, dist, seeds, arr = trace(8, gen.derive_seed(50), n_hi=2e5)
    reqs = rtcdf.make_requests(n, mn, mn + R, dist, seeds, np.zeros(8))
    res, _ = rtcdf.rtcdf_serve_sequential(config(1 << 30), reqs, 8)
    for i in range(8):
        assert res[i].status == 0
        assert res[i].digest == oracle_digest(n[i], mn[i], R[i], dist[i], seeds[i])


def test_results_alone_equal_results_in_the_mix():
    count = 400
    n, mn, R, dist, seeds, arr = trace(count, gen.derive_seed(51))
    reqs = rtcdf.make_requests(n, mn, mn + R, dist, seeds, arr)
    mix, st = rtcdf.rtcdf_serve_trace(config(4 << 30), reqs, count)
    alone, _ = rtcdf.rtcdf_serve_sequential(config(4 << 30), reqs, count)
    assert st.launches_batched > 0 and st.batched_requests > 0
    assert st.max_inflight > 1, "launches should overlap"
    for i in range(count):
        assert mix[i].status == 0 and alone[i].status == 0
        assert mix[i].digest == alone[i].digest, f"request {i} differs alone vs in the mix"
        assert mix[i].done_s >= mix[i].launch_s >= mix[i].admit_s >= arr[i] - 1e-6
    # and against the oracle on a sample
    for i in range(0, count, 23):
        assert mix[i].digest == oracle_digest(n[i], mn[i], R[i], dist[i], seeds[i]), i


def test_served_outputs_equal_oracle_element_by_element():
    """Requests admitted while others run and batched with them: every output
    of n <= 1e6 keys, and a seeded sample of the larger ones, copied back from
    the server and compared with the oracle position by position."""
    count = 300
    n, mn, R, dist, seeds, arr = trace(count, gen.derive_seed(54), n_hi=3e6, rate=20000.0)
    reqs = rtcdf.make_requests(n, mn, mn + R, dist, seeds, arr)
    rng = np.random.default_rng(54)
    big = np.nonzero(n > 1_000_000)[0]
    chosen = list(np.nonzero(n <= 1_000_000)[0]) + list(rng.choice(big, size=min(12, big.size),
                                                                    replace=False))
    bufs, ptrs = output_buffers(n, chosen)
    cfg = config(4 << 30)
    cfg.outputs = ctypes.cast(ptrs, ctypes.c_void_p)
    res, st = rtcdf.rtcdf_serve_trace(cfg, reqs, count)
    assert st.launches_batched > 0 and st.max_inflight > 1
    for i in range(count):
        assert res[i].status == 0, i
    assert_outputs_match_oracle(bufs, n, mn, R, dist, seeds)


def test_large_requests_on_high_priority_streams_match():
    """Large requests written and sorted on high-priority streams, batches on
    default ones: every result equals the one served alone, and a sample of
    the large outputs equals the oracle element by element."""
    count = 300
    n, mn, R, dist, seeds, arr = trace(count, gen.derive_seed(55), n_hi=8e6, rate=20000.0)
    reqs = rtcdf.make_requests(n, mn, mn + R, dist, seeds, arr)
    big = np.nonzero(n >= (1 << 21))[0]
    bufs, ptrs = output_buffers(n, list(big[:10]))
    cfg = config(4 << 30, prio=1)
    cfg.outputs = ctypes.cast(ptrs, ctypes.c_void_p)
    mix, st = rtcdf.rtcdf_serve_trace(cfg, reqs, count)
    alone, _ = rtcdf.rtcdf_serve_sequential(config(4 << 30), reqs, count)
    assert st.launches_single > 0 and st.launches_batched > 0
    for i in range(count):
        assert mix[i].status == 0 and mix[i].digest == alone[i].digest, i
    assert_outputs_match_oracle(bufs, n, mn, R, dist, seeds)


def test_load_adaptive_policy_results_match():
    """Keys written on the launch stream right before the sort, one large
    launch at a time until a backlog of large requests forms: every result
    equals the one served alone, and sampled outputs equal the oracle."""
    count = 400
    n, mn, R, dist, seeds, arr = trace(count, gen.derive_seed(56), n_hi=8e6, rate=40000.0)
    reqs = rtcdf.make_requests(n, mn, mn + R, dist, seeds, arr)
    chosen = list(np.nonzero(n <= 200_000)[0][:30]) + list(np.nonzero(n >= (1 << 21))[0][:8])
    bufs, ptrs = output_buffers(n, chosen)
    cfg = config(4 << 30, max_large=1)
    cfg.fill_at_launch, cfg.large_queue_burst = 1, 3
    cfg.outputs = ctypes.cast(ptrs, ctypes.c_void_p)
    mix, st = rtcdf.rtcdf_serve_trace(cfg, reqs, count)
    alone, _ = rtcdf.rtcdf_serve_sequential(config(4 << 30), reqs, count)
    assert st.launches_single > 0 and st.launches_batched > 0
    for i in range(count):
        assert mix[i].status == 0 and mix[i].digest == alone[i].digest, i
    assert_outputs_match_oracle(bufs, n, mn, R, dist, seeds)


def test_small_budget_admission_waits_for_memory():
    count = 120
    n, mn, R, dist, seeds, arr = trace(count, gen.derive_seed(52), n_hi=4e6, rate=1e6)
    reqs = rtcdf.make_requests(n, mn, mn + R, dist, seeds, arr)
    budget = 256 << 20  # a handful of large requests at a time
    res, st = rtcdf.rtcdf_serve_trace(config(budget), reqs, count)
    alone, _ = rtcdf.rtcdf_serve_sequential(config(budget), reqs, count)
    assert st.peak_bytes <= budget
    for i in range(count):
        assert res[i].status == 0 and res[i].digest == alone[i].digest


def test_request_larger_than_budget_is_refused_others_served():
    n = np.array([1000, 50_000_000, 2000])
    mn = np.array([0, 0, -5])
    R = np.array([100, 100, 7])
    reqs = rtcdf.make_requests(n, mn, mn + R, [0, 0, 1], [1, 2, 3], [0.0, 0.0, 0.0])
    res, _ = rtcdf.rtcdf_serve_trace(config(64 << 20), reqs, 3)
    assert res[1].status == rtcdf.ERR_NO_MEMORY
    for i in (0, 2):
        assert res[i].status == 0
        assert res[i].digest == oracle_digest(n[i], mn[i], R[i], [0, 0, 1][i], [1, 2, 3][i])


def test_one_large_launch_at_a_time_still_matches():
    count = 200
    n, mn, R, dist, seeds, arr = trace(count, gen.derive_seed(53), n_hi=8e6, rate=5e4)
    reqs = rtcdf.make_requests(n, mn, mn + R, dist, seeds, arr)
    res, st = rtcdf.rtcdf_serve_trace(config(2 << 30, max_large=1), reqs, count)
    alone, _ = rtcdf.rtcdf_serve_sequential(config(2 << 30), reqs, count)
    assert st.launches_single > 0
    for i in range(count):
        assert res[i].status == 0 and res[i].digest == alone[i].digest, i


def test_benchmark_serving_trace_all_requests():
    """The benchmark's serving workload (20000 requests, n log-uniform in
    [1e4, 1e8], R log-uniform in [2^7, 2^18], 32 GB budget, Poisson arrivals):
    every request's digest served in the mix equals its digest served alone,
    and a seeded sample of requests matches the oracle."""
    count = 20000
    seed = gen.derive_seed(5)
    n, mn, R, dist, seeds = gen.serving_requests(seed, count)
    arr = gen.poisson_arrivals(seed, count, 13000.0)
    reqs = rtcdf.make_requests(n, mn, mn + R, dist, seeds, arr)
    cfg = rtcdf.ServerConfig(budget_bytes=32 << 30, num_streams=4, max_batch=256,
                             single_min_keys=1 << 22, fill=gen.fill_function_address(), digests=1)
    mix, st = rtcdf.rtcdf_serve_trace(cfg, reqs, count)
    alone, _ = rtcdf.rtcdf_serve_sequential(cfg, reqs, count)
    assert st.launches_batched > 0 and st.launches_single > 0
    bad = [i for i in range(count) if mix[i].status != 0 or mix[i].digest != alone[i].digest]
    assert not bad, f"{len(bad)} requests differ, first {bad[:5]}"
    rng = np.random.default_rng(7)
    small = np.nonzero(n <= 2_000_000)[0]
    for i in rng.choice(small, size=min(40, small.size), replace=False):
        assert mix[i].digest == oracle_digest(n[i], mn[i], R[i], dist[i], seeds[i]), i


def test_benchmark_serving_trace_outputs_element_by_element():
    """The benchmark's serving trace again, with the outputs of every request
    of n <= 1e6 keys (about half of the 20000) and of a seeded sample of the
    larger ones copied back and compared with the oracle position by
    position."""
    count = 20000
    seed = gen.derive_seed(5)
    n, mn, R, dist, seeds = gen.serving_requests(seed, count)
    arr = gen.poisson_arrivals(seed, count, 13000.0)
    reqs = rtcdf.make_requests(n, mn, mn + R, dist, seeds, arr)
    rng = np.random.default_rng(8)
    big = np.nonzero(n > 1_000_000)[0]
    chosen = list(np.nonzero(n <= 1_000_000)[0]) + list(rng.choice(big, size=min(16, big.size),
                                                                    replace=False))
    bufs, ptrs = output_buffers(n, chosen)
    cfg = rtcdf.ServerConfig(budget_bytes=32 << 30, num_streams=4, max_batch=256,
                             single_min_keys=1 << 22, fill=gen.fill_function_address(), digests=0,
                             outputs=ctypes.cast(ptrs, ctypes.c_void_p))
    res, st = rtcdf.rtcdf_serve_trace(cfg, reqs, count)
    assert st.launches_batched > 0 and st.launches_single > 0
    assert all(res[i].status == 0 for i in range(count))
    assert_outputs_match_oracle(bufs, n, mn, R, dist, seeds)
