"""Segmented (batched) sort: every segment against the CPU oracle, bit-exact."""
import numpy as np
import pytest
import torch

import oracle
from paper_2609_00843_gb300 import _build, gen, rtcdf
from gpu_util import stream_handle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    _build.build()
    torch.cuda.init()


def make_segments(lengths, Rs, mins, dists, seeds, pad_front=0):
    offs = np.zeros(len(lengths) + 1, dtype=np.int64)
    offs[1:] = np.cumsum(lengths)
    offs += pad_front
    total = int(offs[-1])
    x = torch.empty(max(1, total), dtype=torch.int32, device="cuda")
    s = stream_handle()
    for i, n in enumerate(lengths):
        if n:
            gen.keys_device(x.data_ptr() + 4 * int(offs[i]), int(n), int(mins[i]), int(Rs[i]),
                            int(dists[i]), int(seeds[i]), stream=s)
    torch.cuda.synchronize()
    return x, offs, np.asarray(mins, np.int64), np.asarray(mins, np.int64) + np.asarray(Rs, np.int64)


def check_segments(x, out, offs, mins, maxs):
    a = x.cpu().numpy()
    b = out.cpu().numpy()
    for s in range(len(mins)):
        lo, hi = int(offs[s]), int(offs[s + 1])
        want = oracle.counting_sort(a[lo:hi], int(mins[s]), int(maxs[s]))
        got = b[lo:hi]
        if not np.array_equal(got, want):
            bad = np.nonzero(got != want)[0]
            raise AssertionError(f"segment {s} (n={hi - lo}, R={maxs[s] - mins[s]}): {bad.size} "
                                 f"positions differ, first {bad[:5].tolist()}")


def run_plan(x, out, offs, mins, maxs, params=None):
    plan = rtcdf.BatchPlan(offs, mins, maxs, params)
    wsb = max(256, plan.workspace_size())
    ws = torch.zeros(wsb // 4 + 64, dtype=torch.int32, device="cuda")
    s = stream_handle()
    rc = plan.run(x.data_ptr(), out.data_ptr(), ws.data_ptr(), wsb, s)
    assert rc == rtcdf.OK, rtcdf.rtcdf_status_str(rc)
    rc, bits = rtcdf.rtcdf_batch_status_get(ws.data_ptr(), s)
    return plan, ws, wsb, rc, bits


def test_mixed_small_and_large_segments():
    lengths = [0, 1, 5, 1000, 65535, 65536, 200_001, 1_000_000, 3, 70_000, 50_000, 131_073]
    Rs = [5, 1, 128, 4097, 65536, 128, 1 << 16, 1 << 14, 7, 70_000, 100_000, 1 << 20]
    mins = [0, -5, 1000, -(1 << 20), 17, -(1 << 31), 0, -3, 5, 100, -100_000, -(1 << 19)]
    dists = [i % 3 for i in range(len(lengths))]
    seeds = [gen.derive_seed(30, i) for i in range(len(lengths))]
    x, offs, mn, mx = make_segments(lengths, Rs, mins, dists, seeds)
    out = torch.full_like(x, 0x7FFFFFFF)
    plan, ws, wsb, rc, bits = run_plan(x, out, offs, mn, mx)
    assert (rc, bits) == (rtcdf.OK, 0)
    info = plan.info()
    assert info["small_segments"] >= 4 and info["large_segments"] >= 4
    check_segments(x, out, offs, mn, mx)


@pytest.mark.parametrize("by_time", [1, -1])
def test_long_in_cta_sorts_split_when_they_would_outlast_the_scan_launch(by_time):
    """A few large segments (so the plan has scan chunks) and narrow-range
    segments of 65535 keys: with the time rule on, those whose estimated
    in-CTA sort would outlast the scan launch are split into work items (fewer
    in-CTA segments), with it off the limits alone keep them in one CTA; the
    output is the same, every segment against the oracle."""
    lengths = [300_000, 150_000] + [65_535] * 6 + [2_000] * 20
    Rs = [5_000, 40_000] + [9_000, 16_000, 300, 12_000, 1, 16_000] + [700] * 20
    mins = [(-1) ** i * 3_001 * i for i in range(len(lengths))]
    x, offs, mn, mx = make_segments(lengths, Rs, mins, [i % 3 for i in range(len(lengths))],
                                    [gen.derive_seed(35, i) for i in range(len(lengths))])
    out = torch.full_like(x, 0x7FFFFFFF)
    plan, ws, wsb, rc, bits = run_plan(x, out, offs, mn, mx, rtcdf.BatchParams(small_by_time=by_time))
    assert (rc, bits) == (rtcdf.OK, 0)
    small = plan.info()["small_segments"]
    if by_time < 0:
        assert small == 26
    else:
        assert 20 <= small < 26
    check_segments(x, out, offs, mn, mx)


def test_batched_workload_shapes_sample():
    """512 segments with the batched workload's shapes (lengths log-uniform in
    [1e3, 1e6], R log-uniform in [2^7, 2^16], minVal in [-2^20, 2^20], mixed
    shapes), unaligned start, run twice on the same workspace."""
    L, mn, R, dist, seeds = gen.batched_segments(gen.derive_seed(31), 512)
    x, offs, mns, mxs = make_segments(L, R, mn, dist, seeds, pad_front=3)
    out = torch.empty_like(x)
    plan, ws, wsb, rc, bits = run_plan(x, out, offs, mns, mxs)
    assert (rc, bits) == (rtcdf.OK, 0)
    check_segments(x, out, offs, mns, mxs)
    out.fill_(0)
    s = stream_handle()
    assert plan.run(x.data_ptr(), out.data_ptr(), ws.data_ptr(), wsb, s) == rtcdf.OK
    assert rtcdf.rtcdf_batch_status_get(ws.data_ptr(), s) == (rtcdf.OK, 0)
    check_segments(x, out, offs, mns, mxs)


def test_graph_capture_and_replay_with_new_keys():
    L, mn, R, dist, seeds = gen.batched_segments(gen.derive_seed(32), 200)
    x, offs, mns, mxs = make_segments(L, R, mn, dist, seeds)
    out = torch.empty_like(x)
    plan = rtcdf.BatchPlan(offs, mns, mxs)
    wsb = plan.workspace_size()
    ws = torch.zeros(wsb // 4 + 64, dtype=torch.int32, device="cuda")
    st = torch.cuda.Stream()
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=st):
        assert plan.run(x.data_ptr(), out.data_ptr(), ws.data_ptr(), wsb, st.cuda_stream) == 0
    for rep in range(3):
        seeds2 = [gen.derive_seed(33, rep, i) for i in range(len(L))]
        x2, _, _, _ = make_segments(L, R, mn, dist, seeds2)
        x.copy_(x2)
        out.fill_(-1)
        torch.cuda.synchronize()
        g.replay()
        torch.cuda.synchronize()
        assert rtcdf.rtcdf_batch_status_get(ws.data_ptr(), st.cuda_stream) == (rtcdf.OK, 0)
        check_segments(x, out, offs, mns, mxs)


def test_one_shot_entry_point_and_in_place():
    lengths = [10, 100_000, 70_000, 1]
    Rs = [3, 1 << 12, 1 << 17, 1]
    mins = [0, -10, 7, 4]
    x, offs, mn, mx = make_segments(lengths, Rs, mins, [0, 1, 0, 2], [1, 2, 3, 4])
    a = x.cpu().numpy().copy()
    rc = rtcdf.rtcdf_sort_batched_host(x.data_ptr(), x.data_ptr(), offs, mn, mx, stream_handle())
    assert rc == rtcdf.OK
    b = x.cpu().numpy()
    for s in range(len(lengths)):
        lo, hi = offs[s], offs[s + 1]
        np.testing.assert_array_equal(b[lo:hi], oracle.counting_sort(a[lo:hi], mn[s], mx[s]))


def test_out_of_range_key_in_one_segment_reports_status():
    lengths = [1000, 300_000]
    for bad_seg in (0, 1):
        x, offs, mn, mx = make_segments(lengths, [100, 1000], [0, 0], [0, 0], [5, 6])
        x[int(offs[bad_seg]) + 17] = 100_000
        out = torch.empty_like(x)
        _, _, _, rc, bits = run_plan(x, out, offs, mn, mx)
        assert rc == rtcdf.ERR_KEY_OUT_OF_RANGE and bits & rtcdf.DEV_KEY_OUT_OF_RANGE


@pytest.mark.parametrize("hist_chunk,fill_chunk,small_max_n", [
    (4096, 4096, 1),            # every segment large, many tiny items
    (4100, 65536, 20000),       # chunk boundaries off the 16-byte grid
    (1 << 20, 1 << 18, 65535),  # few large items
])
def test_work_item_sizes_change_nothing_but_the_schedule(hist_chunk, fill_chunk, small_max_n):
    L, mn, R, dist, seeds = gen.batched_segments(gen.derive_seed(70), 48, n_lo=1, n_hi=3e5,
                                                 r_hi=2 ** 17)
    x, offs, mins, maxs = make_segments(L, R, mn, dist, seeds, pad_front=3)
    out = torch.full_like(x, 12345)
    p = rtcdf.BatchParams(hist_chunk=hist_chunk, fill_chunk=fill_chunk, small_max_n=small_max_n)
    plan, ws, wsb, rc, bits = run_plan(x, out, offs, mins, maxs, p)
    assert rc == rtcdf.OK and bits == 0
    info = plan.info()
    if small_max_n == 1:
        assert info["small_segments"] <= sum(1 for n in L if n <= 1)
    check_segments(x, out, offs, mins, maxs)


def test_profiled_launch_counts_every_item_and_sorts_the_same():
    L, mn, R, dist, seeds = gen.batched_segments(gen.derive_seed(71), 300, n_lo=10, n_hi=4e5)
    x, offs, mins, maxs = make_segments(L, R, mn, dist, seeds)
    out = torch.empty_like(x)
    plan = rtcdf.BatchPlan(offs, mins, maxs)
    wsb = max(256, plan.workspace_size())
    ws = torch.zeros(wsb // 4 + 64, dtype=torch.int32, device="cuda")
    prof = torch.zeros(rtcdf.BATCH_PROFILE_WORDS, dtype=torch.int64, device="cuda")
    prof[8:12] = -1
    s = stream_handle()
    assert plan.run_profiled(x.data_ptr(), out.data_ptr(), ws.data_ptr(), wsb, prof.data_ptr(), s) == rtcdf.OK
    rc, bits = rtcdf.rtcdf_batch_status_get(ws.data_ptr(), s)
    assert rc == rtcdf.OK and bits == 0
    w = [int(v) & ((1 << 64) - 1) for v in prof.cpu().tolist()]
    info = plan.info()
    assert sum(w[4:8]) == info["work_items"]
    assert w[5] == info["small_segments"]
    for k in range(4):
        if w[4 + k]:
            assert w[k] > 0 and w[8 + k] <= w[12 + k] and w[16 + k] <= w[k]
    summ = rtcdf.batch_profile_summary(w, info["workers"])
    assert set(summ) <= set(rtcdf.BATCH_ITEM_KINDS)
    check_segments(x, out, offs, mins, maxs)
    # and the same plan, unprofiled, replays with the counters reset
    out2 = torch.empty_like(x)
    assert plan.run(x.data_ptr(), out2.data_ptr(), ws.data_ptr(), wsb, s) == rtcdf.OK
    torch.cuda.synchronize()
    assert torch.equal(out, out2)


def test_benchmark_batched_workload_every_segment():
    """The benchmark's segmented workload itself (4096 segments, 5.8e8 keys,
    the seed bench.py uses), replayed from a CUDA graph as the benchmark does:
    every segment against the oracle."""
    L, mn, R, dist, seeds = gen.batched_segments(gen.derive_seed(4), 4096)
    x, offs, mns, mxs = make_segments(L, R, mn, dist, seeds)
    out = torch.empty_like(x)
    plan = rtcdf.BatchPlan(offs, mns, mxs)
    wsb = plan.workspace_size()
    ws = torch.zeros(wsb // 4 + 64, dtype=torch.int32, device="cuda")
    st = torch.cuda.Stream()
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=st):
        assert plan.run(x.data_ptr(), out.data_ptr(), ws.data_ptr(), wsb, st.cuda_stream) == 0
    for _ in range(2):
        out.fill_(-1)
        torch.cuda.synchronize()
        g.replay()
        torch.cuda.synchronize()
    assert rtcdf.rtcdf_batch_status_get(ws.data_ptr(), st.cuda_stream) == (rtcdf.OK, 0)
    check_segments(x, out, offs, mns, mxs)


def test_plans_chained_on_one_stream_read_each_others_output():
    """A plan whose only launch is the first one (wide-range in-CTA segments)
    followed on the same stream by a plan whose only launch is the scan
    launch (narrow-range in-CTA segments, which wait for nothing inside their
    own plan) that reads the first plan's output: the second plan's first
    launch must still wait for all earlier work in the stream."""
    S, n, r_keys = 64, 60_000, 10_000
    lengths, mins = [n] * S, [(-1) ** i * 1000 * i for i in range(S)]
    x, offs, mn, _ = make_segments(lengths, [r_keys] * S, mins, [i % 3 for i in range(S)],
                                   [gen.derive_seed(81, i) for i in range(S)])
    wide = rtcdf.BatchPlan(offs, mn, mn + 30_000)     # R > 16000: first launch only
    narrow = rtcdf.BatchPlan(offs, mn, mn + r_keys)   # R <= 16000: scan launch only
    assert wide.info()["small_segments"] == S and narrow.info()["small_segments"] == S
    ws_w = torch.zeros(max(256, wide.workspace_size()) // 4 + 64, dtype=torch.int32, device="cuda")
    ws_n = torch.zeros(max(256, narrow.workspace_size()) // 4 + 64, dtype=torch.int32, device="cuda")
    mid = torch.empty_like(x)
    out = torch.empty_like(x)
    s = stream_handle()
    for _ in range(5):
        mid.fill_(1 << 30)  # outside every range: a read before the first plan wrote it is an error
        assert wide.run(x.data_ptr(), mid.data_ptr(), ws_w.data_ptr(), ws_w.numel() * 4, s) == rtcdf.OK
        assert narrow.run(mid.data_ptr(), out.data_ptr(), ws_n.data_ptr(), ws_n.numel() * 4, s) == rtcdf.OK
        assert rtcdf.rtcdf_batch_status_get(ws_w.data_ptr(), s) == (rtcdf.OK, 0)
        assert rtcdf.rtcdf_batch_status_get(ws_n.data_ptr(), s) == (rtcdf.OK, 0)
    check_segments(x, out, offs, mn, mn + r_keys)
    wide.close()
    narrow.close()


@pytest.mark.parametrize("scan_max_R", [0, 16768])
def test_in_cta_counter_layouts_at_their_capacity(scan_max_R):
    """In-CTA segments at every counter-layout boundary: 32-bit counters up to
    8384 values in a scan-launch CTA and 27648 in a first-launch CTA, 16-bit
    split counters above that, up to 16768 values in a scan-launch CTA (its
    whole shared memory, with the plan parameter at its maximum) and 55296 in
    a first-launch CTA; each range with 65535 keys of every shape and a short
    segment whose keys leave most values empty."""
    Rs = [8384, 8385, 16000, 16768, 27648, 27649, 55296]
    lengths, ranges, mins, dists = [], [], [], []
    for i, R in enumerate(Rs):
        for d in (gen.UNIFORM, gen.NORMAL, gen.ALL_EQUAL):
            lengths.append(65535); ranges.append(R); mins.append(-(1 << 20) + 977 * i); dists.append(d)
        lengths.append(777); ranges.append(R); mins.append(5000 * i); dists.append(gen.UNIFORM)
    seeds = [gen.derive_seed(82, i) for i in range(len(lengths))]
    x, offs, mn, mx = make_segments(lengths, ranges, mins, dists, seeds, pad_front=1)
    out = torch.full_like(x, 0x7FFFFFFF)
    p = rtcdf.BatchParams(small_scan_max_R=scan_max_R)
    plan, ws, wsb, rc, bits = run_plan(x, out, offs, mn, mx, p)
    assert (rc, bits) == (rtcdf.OK, 0)
    assert plan.info()["small_segments"] == len(lengths)
    check_segments(x, out, offs, mn, mx)
    plan.close()
