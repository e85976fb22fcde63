"""Segmented sort with the segment metadata in device memory, planned on the
device (rtcdf_sort_batched, rtcdf_sort_batched_device_ws): every segment
against the CPU oracle, bit-exact; CUDA-graph replay with new keys AND new
segment layouts; metadata that breaks its bounds; and the GPU planner's
work lists compared with the host emulation of the same rules."""
import os
import shutil
import subprocess

import numpy as np
import pytest
import torch

import oracle
from paper_2609_00843_gb300 import _build, gen, rtcdf
from gpu_util import stream_handle

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


@pytest.fixture(scope="module", autouse=True)
def built():
    _build.build()
    torch.cuda.init()


def layout_keys(x, offs, lengths, mins, Rs, dists, seeds):
    s = stream_handle()
    for i, n in enumerate(lengths):
        if n:
            gen.keys_device(x.data_ptr() + 4 * int(offs[i]), int(n), int(mins[i]), int(Rs[i]), int(dists[i]),
                            int(seeds[i]), stream=s)


def make_layout(lengths, Rs, mins, dists, seeds, cap=None, pad_front=0):
    offs = np.zeros(len(lengths) + 1, dtype=np.int64)
    offs[1:] = np.cumsum(lengths)
    offs += pad_front
    total = int(offs[-1]) if cap is None else cap
    x = torch.empty(max(1, total), dtype=torch.int32, device="cuda")
    layout_keys(x, offs, lengths, mins, Rs, dists, seeds)
    mn = np.asarray(mins, np.int64)
    return x, offs, mn, mn + np.asarray(Rs, np.int64)


def to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.int64)).cuda()


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


MIXED = dict(lengths=[0, 1, 5, 1000, 65535, 65536, 200_001, 1_000_000, 3, 70_000, 50_000, 131_073],
             Rs=[5, 1, 128, 4097, 65536, 128, 1 << 16, 1 << 14, 7, 70_000, 100_000, 1 << 20],
             mins=[0, -3, 7, -(1 << 31), 100, 1 << 30, -5, 0, 2, -70_000, 12, -(1 << 19)],
             dists=[0, 1, 2, 0, 1, 2, 0, 1, 2, 0, 1, 2])


def test_library_workspace_every_segment_and_status():
    m = MIXED
    x, offs, mn, mx = make_layout(m["lengths"], m["Rs"], m["mins"], m["dists"], range(1, 13))
    out = torch.full_like(x, 0x7FFFFFFF)
    s = stream_handle()
    d_o, d_mn, d_mx = to_dev(offs), to_dev(mn), to_dev(mx)
    rc = rtcdf.rtcdf_sort_batched(x.data_ptr(), out.data_ptr(), d_o.data_ptr(), d_mn.data_ptr(), d_mx.data_ptr(),
                                  len(mn), x.numel(), 1 << 20, s)
    assert rc == rtcdf.OK, rtcdf.rtcdf_status_str(rc)
    assert rtcdf.rtcdf_status_get(s) == (rtcdf.OK, 0)
    check_segments(x, out, offs, mn, mx)
    # in place, same library workspace (left ready by the previous call)
    a = x.clone()
    rc = rtcdf.rtcdf_sort_batched(x.data_ptr(), x.data_ptr(), d_o.data_ptr(), d_mn.data_ptr(), d_mx.data_ptr(),
                                  len(mn), x.numel(), 1 << 20, s)
    assert rc == rtcdf.OK
    assert rtcdf.rtcdf_status_get(s) == (rtcdf.OK, 0)
    check_segments(a, x, offs, mn, mx)


def test_graph_replay_with_new_keys_and_new_segment_layouts():
    """One capture, replayed for three layouts of the same bounds (S segments,
    at most N keys, R <= max_R): the metadata and keys are rewritten in the
    captured device buffers between replays, and no host work happens."""
    S, N, max_R = 40, 3_000_000, 1 << 17
    wsb = rtcdf.rtcdf_batch_device_workspace_size(S, N, max_R)
    ws = torch.zeros(wsb // 4 + 64, dtype=torch.int32, device="cuda")
    x = torch.empty(N, dtype=torch.int32, device="cuda")
    out = torch.empty(N, dtype=torch.int32, device="cuda")
    d_o = torch.zeros(S + 1, dtype=torch.int64, device="cuda")
    d_mn = torch.zeros(S, dtype=torch.int64, device="cuda")
    d_mx = torch.ones(S, dtype=torch.int64, device="cuda")
    st = torch.cuda.Stream()
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=st):
        rc = rtcdf.rtcdf_sort_batched_device_ws(x.data_ptr(), out.data_ptr(), d_o.data_ptr(), d_mn.data_ptr(),
                                                d_mx.data_ptr(), S, N, max_R, ws.data_ptr(), wsb, st.cuda_stream)
        assert rc == rtcdf.OK
    rng = np.random.default_rng(30)
    for layout in range(3):
        lengths = rng.integers(0, N // S, S)
        lengths[rng.integers(0, S)] = 0
        if layout == 1:
            lengths[:5] = [70_000, 65_535, 1, 2, 65_536]
        Rs = np.exp(rng.uniform(0, np.log(max_R), S)).astype(np.int64).clip(1, max_R)
        mins = rng.integers(-(1 << 30), 1 << 30, S)
        dists = rng.integers(0, 3, S)
        offs = np.zeros(S + 1, dtype=np.int64)
        offs[1:] = np.cumsum(lengths)
        offs += layout  # segments need not start at 0
        assert offs[-1] <= N
        layout_keys(x, offs, lengths, mins, Rs, dists, [gen.derive_seed(31, layout, i) for i in range(S)])
        d_o.copy_(torch.from_numpy(offs))
        d_mn.copy_(torch.from_numpy(mins.astype(np.int64)))
        d_mx.copy_(torch.from_numpy((mins + Rs).astype(np.int64)))
        out.fill_(-1)
        torch.cuda.synchronize()
        g.replay()
        torch.cuda.synchronize()
        assert rtcdf.rtcdf_batch_status_get(ws.data_ptr(), st.cuda_stream) == (rtcdf.OK, 0), layout
        check_segments(x, out, offs, mins, mins + Rs)


@pytest.mark.parametrize("case", ["R above max_R", "offsets above max_total_keys", "offsets decrease",
                                  "minVal below int32", "empty range"])
def test_metadata_breaking_the_bounds_writes_nothing(case):
    S, N, max_R = 4, 400_000, 1 << 12
    lengths, Rs, mins = [1000, 100_000, 0, 50_000], [100, 4096, 3, 1 << 12], [0, -9, 5, 1 << 20]
    x, offs, mn, mx = make_layout(lengths, Rs, mins, [0, 1, 2, 0], [1, 2, 3, 4], cap=N)
    if case == "R above max_R":
        mx[1] = mn[1] + max_R + 1
    elif case == "offsets above max_total_keys":
        offs[-1] = N + 1
    elif case == "offsets decrease":
        offs[2] = offs[1] - 1
    elif case == "minVal below int32":
        mn[0] = -(1 << 31) - 1
    else:
        mx[3] = mn[3]
    wsb = rtcdf.rtcdf_batch_device_workspace_size(S, N, max_R)
    ws = torch.zeros(wsb // 4 + 64, dtype=torch.int32, device="cuda")
    out = torch.full_like(x, -77)
    s = stream_handle()
    d_o, d_mn, d_mx = to_dev(offs), to_dev(mn), to_dev(mx)
    rc = rtcdf.rtcdf_sort_batched_device_ws(x.data_ptr(), out.data_ptr(), d_o.data_ptr(), d_mn.data_ptr(),
                                            d_mx.data_ptr(), S, N, max_R, ws.data_ptr(), wsb, s)
    assert rc == rtcdf.OK  # found on the device, not on the host
    rc, bits = rtcdf.rtcdf_batch_status_get(ws.data_ptr(), s)
    assert rc == rtcdf.ERR_INVALID_ARG and bits & rtcdf.DEV_BAD_SEGMENT, (rc, bits)
    assert (out == -77).all(), "nothing may be written"
    # the workspace serves a valid call right after
    x2, offs2, mn2, mx2 = make_layout(lengths, Rs, mins, [0, 1, 2, 0], [5, 6, 7, 8], cap=N)
    d_o, d_mn, d_mx = to_dev(offs2), to_dev(mn2), to_dev(mx2)
    rc = rtcdf.rtcdf_sort_batched_device_ws(x2.data_ptr(), out.data_ptr(), d_o.data_ptr(), d_mn.data_ptr(),
                                            d_mx.data_ptr(), S, N, max_R, ws.data_ptr(), wsb, s)
    assert rc == rtcdf.OK
    assert rtcdf.rtcdf_batch_status_get(ws.data_ptr(), s) == (rtcdf.OK, 0)
    check_segments(x2, out, offs2, mn2, mx2)


@pytest.fixture(scope="module")
def emitter(tmp_path_factory):
    cxx = shutil.which("g++")
    if not cxx:
        pytest.skip("no C++ compiler")
    cuda_inc = os.path.join(os.path.dirname(os.path.dirname(_build.nvcc())), "include")
    lib_dir = os.path.dirname(_build.lib_path())
    exe = str(tmp_path_factory.mktemp("devplan") / "planner_check")
    cmd = [cxx, "-std=c++17", "-O1", os.path.join(HERE, "planner_check.cpp"),
           "-I", os.path.join(ROOT, "paper_2609_00843_gb300", "csrc"), "-I", cuda_inc,
           "-L", lib_dir, "-lrtcdf", f"-Wl,-rpath,{lib_dir}", "-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-3000:]
    return exe


def test_gpu_planner_writes_what_the_host_emulation_computes(emitter, tmp_path):
    """The planner kernel's descriptors, list lengths and items, read back from
    the workspace, equal the host emulation of the same rules (planner_check
    --emit) field by field: 2600 segments, so three planner CTAs hand their
    counts on through the lookback, every eleventh segment empty, and items
    in each of the lists by size."""
    L, mn, R, dist, seeds = gen.batched_segments(gen.derive_seed(32), 2600, n_lo=1, n_hi=1e5, r_hi=2 ** 18)
    L = L.copy()
    L[::11] = 0
    # some segments with histogram items of each size class (a whole chunk
    # of 2^19 keys and a short rest, 200000 keys, 300000 keys)
    L[1::50], L[2::50], L[3::50] = 600_000, 200_000, 300_000
    mn = mn.astype(np.int64)
    x, offs, mns, mxs = make_layout(L, R, mn, dist, seeds)
    S, N, max_R = len(L), x.numel(), 1 << 18
    meta = tmp_path / "meta.txt"
    meta.write_text(f"{S} {N} {max_R}\n" + " ".join(map(str, offs)) + "\n" + " ".join(map(str, mns)) + "\n"
                    + " ".join(map(str, mxs)) + "\n")
    r = subprocess.run([emitter, "--emit", str(meta)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-2000:]
    lines = r.stdout.splitlines()
    lay = [int(v) for v in lines[0].split()[1:]]
    hist_b, first_b, scan_b, small2_b, fill_b = [int(v) for v in lines[1].split()[1:]]
    assert lines[2] == "rc 0"
    hdr = [int(v) for v in lines[3].split()[1:]]
    segs = [[int(v) for v in ln.split()[1:]] for ln in lines if ln.startswith("seg ")]
    items = np.asarray([[int(v) for v in ln.split()[1:]] for ln in lines if ln.startswith("item ")],
                       dtype=np.int64)
    wsb = rtcdf.rtcdf_batch_device_workspace_size(S, N, max_R)
    assert wsb == lay[5] * 4
    ws = torch.zeros(wsb // 4 + 64, dtype=torch.int32, device="cuda")
    out = torch.empty_like(x)
    s = stream_handle()
    d_o, d_mn, d_mx = to_dev(offs), to_dev(mns), to_dev(mxs)
    rc = rtcdf.rtcdf_sort_batched_device_ws(x.data_ptr(), out.data_ptr(), d_o.data_ptr(), d_mn.data_ptr(),
                                            d_mx.data_ptr(), S, N, max_R, ws.data_ptr(), wsb, s)
    assert rc == rtcdf.OK
    assert rtcdf.rtcdf_batch_status_get(ws.data_ptr(), s) == (rtcdf.OK, 0)
    check_segments(x, out, offs, mns, mxs)
    w = ws.cpu().numpy().view(np.uint32)
    _, hdr_off, seg_off, look_off, item_off, _ = lay
    assert w[hdr_off:hdr_off + 13].tolist() == hdr
    # the output launch left the planner's lookback records zeroed for the next run
    assert not w[look_off:look_off + 32 * ((S + 1023) // 1024)].any()
    seg_dt = np.dtype([("off", "<u8"), ("out_off", "<u8"), ("n", "<u4"), ("R", "<u4"), ("minVal", "<i4"),
                       ("T", "<u4"), ("m", "<u4"), ("hist_items", "<u4"), ("fill_items", "<u4"),
                       ("fill_chunk", "<u4"), ("scan_chunks", "<u4"), ("single_hist", "<u4"), ("hist_off", "<u8"),
                       ("run_end_off", "<u8"), ("run_val_off", "<u8"), ("start_run_off", "<u8"),
                       ("state_off", "<u8")])
    assert seg_dt.itemsize == 96
    g = w[seg_off:seg_off + S * 24].view(seg_dt)
    fields = ["off", "n", "R", "minVal", "T", "m", "hist_items", "fill_items", "fill_chunk", "scan_chunks",
              "single_hist", "hist_off", "run_end_off", "run_val_off", "start_run_off", "state_off"]
    for i in range(S):
        got = [int(g[i][f]) for f in fields]
        assert got == segs[i], f"segment {i}: {got} != {segs[i]}"
    item_dt = np.dtype([("kind", "<u4"), ("seg", "<u4"), ("a", "<u8"), ("b", "<u8"), ("tile", "<u4"),
                        ("aux", "<u4")])
    it = w[item_off:item_off + len(items) * 8].view(item_dt)
    got = np.stack([it[f].astype(np.int64) for f in ("kind", "seg", "a", "b", "tile", "aux")], axis=1)
    # every list at its fixed base, compared up to its length
    n_first, n_scan, n_small2, n_fill, n_hist, n_small1, nh0, nh1, nh2, ns0, ns1, nf0, nf1 = hdr
    assert n_small1 > 0 and n_small2 > 0 and min(nh0, nh1, nh2, ns0, ns1, nf0, nf1) > 0
    fb = first_b + 2 * scan_b + small2_b
    for base, n in ((0, nh0), (hist_b, nh1), (2 * hist_b, nh2), (3 * hist_b, n_small1), (first_b, ns0),
                    (first_b + scan_b, ns1), (first_b + 2 * scan_b, n_small2), (fb, nf0), (fb + fill_b, nf1)):
        np.testing.assert_array_equal(got[base:base + n], items[base:base + n])


def test_benchmark_batched_workload_device_planned():
    """The benchmark's segmented workload (4096 segments, 5.8e8 keys) through
    the device-planned entry point, replayed from a CUDA graph: every segment
    against the oracle."""
    L, mn, R, dist, seeds = gen.batched_segments(gen.derive_seed(4), 4096)
    x, offs, mns, mxs = make_layout(L, R, mn, dist, seeds)
    S, N, max_R = len(L), x.numel(), 1 << 16
    wsb = rtcdf.rtcdf_batch_device_workspace_size(S, N, max_R)
    ws = torch.zeros(wsb // 4 + 64, dtype=torch.int32, device="cuda")
    out = torch.empty_like(x)
    d_o, d_mn, d_mx = to_dev(offs), to_dev(mns), to_dev(mxs)
    st = torch.cuda.Stream()
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=st):
        assert rtcdf.rtcdf_sort_batched_device_ws(x.data_ptr(), out.data_ptr(), d_o.data_ptr(), d_mn.data_ptr(),
                                                  d_mx.data_ptr(), S, N, max_R, ws.data_ptr(), wsb,
                                                  st.cuda_stream) == rtcdf.OK
    for _ in range(2):
        out.fill_(-1)
        torch.cuda.synchronize()
        g.replay()
        torch.cuda.synchronize()
        assert rtcdf.rtcdf_batch_status_get(ws.data_ptr(), st.cuda_stream) == (rtcdf.OK, 0)
        check_segments(x, out, offs, mns, mxs)


def _device_sort(x, offs, mns, mxs, max_R, ws=None):
    """One device-planned sort on a caller workspace (a fresh zeroed one by
    default); returns the output, the workspace and its status."""
    S, N = len(mns), x.numel()
    wsb = rtcdf.rtcdf_batch_device_workspace_size(S, N, max_R)
    if ws is None:
        ws = torch.zeros(wsb // 4 + 64, dtype=torch.int32, device="cuda")
    out = torch.full_like(x, 0x7FFFFFFF)
    s = stream_handle()
    d_o, d_mn, d_mx = to_dev(offs), to_dev(mns), to_dev(mxs)
    rc = rtcdf.rtcdf_sort_batched_device_ws(x.data_ptr(), out.data_ptr(), d_o.data_ptr(), d_mn.data_ptr(),
                                            d_mx.data_ptr(), S, N, max_R, ws.data_ptr(), wsb, s)
    assert rc == rtcdf.OK, rtcdf.rtcdf_status_str(rc)
    return out, ws, rtcdf.rtcdf_batch_status_get(ws.data_ptr(), s)


@pytest.mark.parametrize("S", [1, 1023, 1024, 1025, 2049])
def test_segment_counts_around_a_planner_cta(S):
    """Segment counts at and around the 1024 segments one planner CTA
    classifies (the lists of later CTAs are placed after the counts they get
    through the lookback), mixed small, large and empty segments, twice on the
    same workspace: every segment against the oracle."""
    L, mn, R, dist, seeds = gen.batched_segments(gen.derive_seed(40, S), S, n_lo=1, n_hi=3e5, r_hi=2 ** 17)
    L = L.copy()
    L[::7] = 0
    x, offs, mns, mxs = make_layout(L, R, mn.astype(np.int64), dist, seeds)
    out, ws, st = _device_sort(x, offs, mns, mxs, 1 << 17)
    assert st == (rtcdf.OK, 0)
    check_segments(x, out, offs, mns, mxs)
    out2, _, st2 = _device_sort(x, offs, mns, mxs, 1 << 17, ws)
    assert st2 == (rtcdf.OK, 0)
    assert torch.equal(out, out2)


@pytest.mark.parametrize("case", ["all_empty", "all_small", "one_large", "widest"])
def test_degenerate_layouts(case):
    """Layouts where some lists are empty: every segment empty (nothing to do;
    the keys stay untouched), only in-CTA segments (no histogram, scan or
    output items), one large segment alone, and one segment of the widest
    range (2^20 values, 256 scan chunks in one lookback chain)."""
    if case == "all_empty":
        L, R = [0] * 300, [5] * 300
    elif case == "all_small":
        L, R = [100 + 37 * i for i in range(1500)], [1 + (i * 977) % 50000 for i in range(1500)]
    elif case == "one_large":
        L, R = [2_500_000], [70_000]
    else:
        L, R = [3_000_000], [1 << 20]
    S = len(L)
    mins = [(-1) ** i * (i * 1013) % 100_000 for i in range(S)]
    x, offs, mns, mxs = make_layout(L, R, mins, [i % 3 for i in range(S)], [gen.derive_seed(41, i) for i in range(S)],
                                    cap=max(1, sum(L)))
    max_R = max(R)
    out, ws, st = _device_sort(x, offs, mns, mxs, max_R)
    assert st == (rtcdf.OK, 0)
    if case == "all_empty":
        assert int(out[0]) == 0x7FFFFFFF
    else:
        check_segments(x, out, offs, mns, mxs)


def test_lists_longer_than_the_scan_grid():
    """More in-CTA segments than the scan launch's capped grid (65536 CTAs):
    66000 segments of a few keys and 100 of 70000 keys, all within 4096
    values (a workspace slot per segment is sized by the widest range), so
    that CTAs take several in-CTA segments each and then loop over the chunk
    tickets.  Every segment is checked: the large ones and a sample of the
    small ones against the oracle, all of them as sorted permutations of
    their keys (one sort by segment and key)."""
    n_small, n_large = 66_000, 100
    L = np.concatenate([3 + (np.arange(n_small) * 7919) % 40, np.full(n_large, 70_000)]).astype(np.int64)
    R = np.concatenate([1 + (np.arange(n_small) * 104729) % 4096, np.full(n_large, 4096)]).astype(np.int64)
    perm = np.random.default_rng(gen.derive_seed(43)).permutation(len(L))  # large ones spread among the small
    L, R = L[perm], R[perm]
    S = len(L)
    mins = ((np.arange(S) * 7777) % 200_000 - 100_000).astype(np.int64)
    x, offs, mns, mxs = make_layout(L, R, mins, np.arange(S) % 3, [gen.derive_seed(44, i) for i in range(S)])
    out, ws, st = _device_sort(x, offs, mns, mxs, 4096)
    assert st == (rtcdf.OK, 0)
    a = x.cpu().numpy()
    b = out.cpu().numpy()
    seg_of = np.repeat(np.arange(S), L)
    order = np.lexsort((a, seg_of))
    np.testing.assert_array_equal(b, a[order])
    for s in list(np.nonzero(L == 70_000)[0]) + list(range(0, S, 997)):
        lo, hi = int(offs[s]), int(offs[s + 1])
        np.testing.assert_array_equal(b[lo:hi], oracle.counting_sort(a[lo:hi], int(mns[s]), int(mxs[s])))
