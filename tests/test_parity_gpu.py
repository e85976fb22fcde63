"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle,
element by element, on seeded inputs.  Integer sort: the bar is bit-exact."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_2609_00843_gb300 import _build, gen, rtcdf
from gpu_util import assert_matches_oracle, dev_keys, gpu_sort, stream_handle

pytestmark = pytest.mark.gpu

DISTS = (gen.UNIFORM, gen.NORMAL, gen.ALL_EQUAL)


@pytest.fixture(scope="module", autouse=True)
def built():
    _build.build()
    torch.cuda.init()


def test_single_array_n1e6_R128_uniform_seed0():
    x = dev_keys(1_000_000, 0, 128, gen.UNIFORM, 0)
    out = gpu_sort(x, 0, 128)
    assert_matches_oracle(x, out, 0, 128)


@pytest.mark.parametrize("R", [1, 2, 3, 127, 128, 129, 1000, 4097, 16384, 40000, 65539, 1 << 18])
@pytest.mark.parametrize("dist", DISTS)
def test_sizes_and_ranges(R, dist):
    for n in (1, 2, 3, 4, 5, 31, 32, 33, 1023, 4097, 65537):
        x = dev_keys(n, -7, R, dist, gen.derive_seed(2, R, dist, n))
        out = gpu_sort(x, -7, -7 + R)
        assert_matches_oracle(x, out, -7, -7 + R)


@pytest.mark.parametrize("R", [128, 4097, 1 << 14, 1 << 16, 1 << 18])
def test_million_keys(R):
    for dist in DISTS:
        x = dev_keys(1_000_003, 12345, R, dist, gen.derive_seed(3, R, dist))
        out = gpu_sort(x, 12345, 12345 + R)
        assert_matches_oracle(x, out, 12345, 12345 + R)


@pytest.mark.parametrize("n", [5, 1001, 100_003])
def test_misaligned_views(n):
    base_in = dev_keys(n + 8, 0, 300, gen.UNIFORM, 9)
    for oi in range(4):
        for oo in range(4):
            x = base_in[oi:oi + n]
            out_base = torch.full((n + 8,), -1, dtype=torch.int32, device="cuda")
            out = out_base[oo:oo + n]
            gpu_sort(x, 0, 300, out=out)
            assert_matches_oracle(x, out, 0, 300)
            ob = out_base.cpu().numpy()
            assert (ob[:oo] == -1).all() and (ob[oo + n:] == -1).all(), "wrote outside the view"


def test_int32_extremes():
    lo = -(1 << 31)
    x = dev_keys(200_001, lo, 1000, gen.UNIFORM, 4)
    assert_matches_oracle(x, gpu_sort(x, lo, lo + 1000), lo, lo + 1000)
    hi = 1 << 31
    x = dev_keys(200_001, hi - 1000, 1000, gen.NORMAL, 5)
    assert_matches_oracle(x, gpu_sort(x, hi - 1000, hi), hi - 1000, hi)
    x = torch.tensor([hi - 1, lo + 5, hi - 1], dtype=torch.int32, device="cuda")
    # whole int32 space is wider than the largest supported range
    assert rtcdf.rtcdf_sort(x.data_ptr(), x.data_ptr(), 3, lo, hi, stream_handle()) == rtcdf.ERR_RANGE


@pytest.mark.parametrize("R", [128, 4097, 1 << 18])
def test_all_equal_first_middle_last_bin(R):
    for v in (0, R // 2, R - 1):
        x = torch.full((300_007,), -50 + v, dtype=torch.int32, device="cuda")
        out = gpu_sort(x, -50, -50 + R)
        assert torch.equal(out, x)


def test_in_place():
    x = dev_keys(1_234_567, -3, 5000, gen.NORMAL, 6)
    a = x.cpu().numpy()
    gpu_sort(x, -3, 4997, out=x)
    np.testing.assert_array_equal(x.cpu().numpy(), oracle.counting_sort(a, -3, 4997))


def test_output_poisoned_every_position_written():
    for R in (128, 70000):
        x = dev_keys(999_999, 0, R, gen.UNIFORM, 7)
        out = torch.full_like(x, 0x7FFFFFFF)
        gpu_sort(x, 0, R, out=out)
        assert_matches_oracle(x, out, 0, R)


def test_key_out_of_range_sets_status_then_clears():
    x = dev_keys(100_000, 0, 128, gen.UNIFORM, 8)
    x[777] = 128
    out = torch.empty_like(x)
    s = stream_handle()
    assert rtcdf.rtcdf_sort(x.data_ptr(), out.data_ptr(), x.numel(), 0, 128, s) == rtcdf.OK
    rc, bits = rtcdf.rtcdf_status_get(s)
    assert rc == rtcdf.ERR_KEY_OUT_OF_RANGE and bits & rtcdf.DEV_KEY_OUT_OF_RANGE
    x[777] = -1
    assert rtcdf.rtcdf_sort(x.data_ptr(), out.data_ptr(), x.numel(), 0, 128, s) == rtcdf.OK
    rc, bits = rtcdf.rtcdf_status_get(s)
    assert rc == rtcdf.ERR_KEY_OUT_OF_RANGE
    x[777] = 5
    gpu_sort(x, 0, 128, out=out)  # status was cleared by the read; now clean
    assert_matches_oracle(x, out, 0, 128)


@pytest.mark.parametrize("R,T", [(4, 2), (1000, 1), (1000, 3), (1000, 128), (5000, 1000),
                                 (5000, 4096), (70000, 8192)])
def test_forced_tiles_intermediates_match_algorithms_5_to_7(R, T):
    """White-box: with an explicit tile width, the tile histograms (Alg. 5),
    O[t] + local CDF and the tile offsets (Alg. 6) equal the oracle's."""
    n = 50_021
    x = dev_keys(n, -11, R, gen.NORMAL, gen.derive_seed(10, R, T))
    out = torch.empty_like(x)
    ws_bytes = rtcdf.rtcdf_workspace_size(R)
    ws = torch.zeros(ws_bytes // 4 + 64, dtype=torch.int32, device="cuda")
    m = -(-R // T)
    th = torch.empty(R, dtype=torch.int32, device="cuda")
    cdf = torch.empty(R, dtype=torch.int32, device="cuda")
    off = torch.empty(m, dtype=torch.int32, device="cuda")
    p = rtcdf.Params(tile_width=T)
    d = rtcdf.Debug(th.data_ptr(), cdf.data_ptr(), off.data_ptr())
    rc = rtcdf.rtcdf_sort_ex(x.data_ptr(), out.data_ptr(), n, -11, -11 + R, p, ws.data_ptr(),
                             ws_bytes, d, stream_handle())
    assert rc == rtcdf.OK
    r = oracle.rtcdf_sort(x.cpu().numpy(), -11, -11 + R, T)
    assert r["m"] == m
    np.testing.assert_array_equal(th.cpu().numpy().astype(np.uint64), r["tile_hist"])
    np.testing.assert_array_equal(off.cpu().numpy().astype(np.uint64), r["O"])
    tile_of = np.arange(R) // T
    np.testing.assert_array_equal(cdf.cpu().numpy().astype(np.uint64),
                                  r["local_cdf"] + r["O"][tile_of])
    np.testing.assert_array_equal(out.cpu().numpy(), r["B"])


@pytest.mark.parametrize("ht,hg,ft,fc", [(256, 1, 256, 1), (512, 3, 1024, 7), (1024, 1000, 512, 4096),
                                        (1024, 0, 256, 3000)])
def test_launch_parameters_do_not_change_result(ht, hg, ft, fc):
    for R in (130, 1 << 16):
        x = dev_keys(777_777, 0, R, gen.UNIFORM, gen.derive_seed(11, R))
        out = torch.empty_like(x)
        ws_bytes = rtcdf.rtcdf_workspace_size(R)
        ws = torch.zeros(ws_bytes // 4 + 64, dtype=torch.int32, device="cuda")
        p = rtcdf.Params(hist_threads=ht, hist_ctas_per_tile=hg, fill_threads=ft, fill_ctas=fc)
        rc = rtcdf.rtcdf_sort_ex(x.data_ptr(), out.data_ptr(), x.numel(), 0, R, p, ws.data_ptr(),
                                 ws_bytes, None, stream_handle())
        assert rc == rtcdf.OK
        assert_matches_oracle(x, out, 0, R)


def test_caller_workspace_reused_across_ranges():
    ws_bytes = rtcdf.rtcdf_workspace_size(1 << 18)
    ws = torch.zeros(ws_bytes // 4 + 64, dtype=torch.int32, device="cuda")
    s = stream_handle()
    for i, R in enumerate([1 << 18, 7, 1 << 14, 1 << 18, 100]):
        x = dev_keys(300_000 + i, 5, R, DISTS[i % 3], gen.derive_seed(12, i))
        out = torch.empty_like(x)
        rc = rtcdf.rtcdf_sort_ws(x.data_ptr(), out.data_ptr(), x.numel(), 5, 5 + R, ws.data_ptr(),
                                 ws_bytes, s)
        assert rc == rtcdf.OK
        assert rtcdf.rtcdf_ws_status_get(ws.data_ptr(), s) == (rtcdf.OK, 0)
        assert_matches_oracle(x, out, 5, 5 + R)


def test_workspace_exactly_sized_for_mixed_ranges():
    """One caller workspace of exactly the largest requirement and ranges that
    grow and shrink between calls: every sort must find its histogram region
    zeroed by the previous one."""
    Rs = [128, 20480, 128, 4097, 65536, 8192, 128, 1 << 17, 3000]
    ws_bytes = max(rtcdf.rtcdf_workspace_size(R) for R in Rs)
    ws = torch.zeros(ws_bytes // 4, dtype=torch.int32, device="cuda")
    s = stream_handle()
    for i, R in enumerate(Rs):
        x = dev_keys(500_000 + 7 * i, -3, R, DISTS[i % 3], gen.derive_seed(18, i))
        out = torch.empty_like(x)
        rc = rtcdf.rtcdf_sort_ws(x.data_ptr(), out.data_ptr(), x.numel(), -3, -3 + R,
                                 ws.data_ptr(), ws_bytes, s)
        assert rc == rtcdf.OK
        assert rtcdf.rtcdf_ws_status_get(ws.data_ptr(), s) == (rtcdf.OK, 0)
        assert_matches_oracle(x, out, -3, -3 + R)


def test_two_streams_do_not_share_workspace():
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    xs = [dev_keys(2_000_000, 0, R, gen.UNIFORM, R) for R in (128, 1 << 18)]
    torch.cuda.synchronize()
    outs = [torch.empty_like(x) for x in xs]
    for _ in range(3):
        for x, o, s, R in zip(xs, outs, (s1, s2), (128, 1 << 18)):
            with torch.cuda.stream(s):
                assert rtcdf.rtcdf_sort(x.data_ptr(), o.data_ptr(), x.numel(), 0, R, s.cuda_stream) == 0
    torch.cuda.synchronize()
    for x, o, R in zip(xs, outs, (128, 1 << 18)):
        assert_matches_oracle(x, o, 0, R)


def test_cuda_graph_capture_and_replay():
    s = torch.cuda.Stream()
    R = 1 << 14
    x = dev_keys(3_000_000, -1000, R, gen.NORMAL, 13)
    out = torch.empty_like(x)
    torch.cuda.synchronize()
    assert rtcdf.rtcdf_reserve(R, s.cuda_stream) == 0
    with torch.cuda.stream(s):  # warm-up on the capture stream
        assert rtcdf.rtcdf_sort(x.data_ptr(), out.data_ptr(), x.numel(), -1000, -1000 + R, s.cuda_stream) == 0
    s.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        assert rtcdf.rtcdf_sort(x.data_ptr(), out.data_ptr(), x.numel(), -1000, -1000 + R, s.cuda_stream) == 0
    for seed in (14, 15):
        x.copy_(dev_keys(3_000_000, -1000, R, gen.UNIFORM, seed))
        torch.cuda.synchronize()
        out.fill_(0)
        g.replay()
        torch.cuda.synchronize()
        assert_matches_oracle(x, out, -1000, -1000 + R)


@pytest.mark.parametrize("pinned", [True, False])
def test_host_buffer_entry_point(pinned):
    """rtcdf_sort_host: host input and output, chunked upload, alternating
    device buffer sets across consecutive calls, growing sizes."""
    s = torch.cuda.Stream()
    cases = [(5, 128, 0), (1_000_003, 4097, 1), (50_000_000, 1 << 14, 1), (3_000_000, 1 << 18, 0),
             (17, 3, 2), (20_000_000, 1000, 2)]
    hosts = []
    for i, (n, R, dist) in enumerate(cases):
        x = dev_keys(n, -77, R, dist, gen.derive_seed(60, i)).cpu()
        if pinned:
            x = x.pin_memory()
        off = i % 3  # misaligned host views too
        xin = torch.empty(n + off, dtype=torch.int32, pin_memory=pinned)[off:]
        xin.copy_(x)
        xout = torch.full((n + off,), -1, dtype=torch.int32, pin_memory=pinned)[off:]
        hosts.append((xin, xout, n, R))
    torch.cuda.synchronize()
    for xin, xout, n, R in hosts:  # back to back: downloads overlap the next uploads
        assert rtcdf.rtcdf_sort_host(xin.data_ptr(), xout.data_ptr(), n, -77, -77 + R,
                                     s.cuda_stream) == rtcdf.OK
    s.synchronize()
    for xin, xout, n, R in hosts:
        np.testing.assert_array_equal(xout.numpy(), oracle.counting_sort(xin.numpy(), -77, -77 + R))


def test_sparse_wide_ranges():
    """Few distinct values spread over a wide range: the output walks many
    empty values between runs."""
    for R in (1 << 18, 1 << 24):
        x = torch.tensor([R - 1, 0, R - 1, R // 2] * 25_000 + [1], dtype=torch.int32, device="cuda")
        out = gpu_sort(x, 0, R)
        assert_matches_oracle(x, out, 0, R)
    x = dev_keys(1_000_000, 0, 1 << 24, gen.UNIFORM, 16)
    assert_matches_oracle(x, gpu_sort(x, 0, 1 << 24), 0, 1 << 24)
    # Runs of two or three keys: most vectors straddle runs and each output
    # CTA walks its positions in several windows of runs.
    for dist in (gen.UNIFORM, gen.NORMAL):
        x = dev_keys(10_000_000, -3, 1 << 22, dist, 17 + dist)
        assert_matches_oracle(x, gpu_sort(x, -3, -3 + (1 << 22)), -3, -3 + (1 << 22))


@pytest.mark.parametrize("tiles", [7, 8, 9])
def test_built_in_plan_at_the_tile_form_boundary(tiles):
    """Built-in plan (explicit all-zero parameters: no tuning table) at the
    ranges where the tile count steps around the boundary between the
    two-to-eight-tile form (trash word, sampled prefetch, the sample's last
    tile slot) and the plain predicated form of nine tiles and more: R =
    tiles x T_max, the largest range with `tiles` tiles of the widest width
    the device's opt-in shared memory allows, and R + 1, one tile more."""
    t_max = (torch.cuda.get_device_properties(0).shared_memory_per_block_optin // 4) & ~1023
    n, mn = 1_000_003, -77
    for R in (tiles * t_max, tiles * t_max + 1):
        ws_bytes = rtcdf.rtcdf_workspace_size(R)
        ws = torch.zeros(ws_bytes // 4 + 64, dtype=torch.int32, device="cuda")
        for dist in DISTS:
            x = dev_keys(n, mn, R, dist, gen.derive_seed(18, R, dist))
            out = torch.empty_like(x)
            rc = rtcdf.rtcdf_sort_ex(x.data_ptr(), out.data_ptr(), n, mn, mn + R, rtcdf.Params(),
                                     ws.data_ptr(), ws_bytes, None, stream_handle())
            assert rc == rtcdf.OK
            rc, bits = rtcdf.rtcdf_ws_status_get(ws.data_ptr(), stream_handle())
            assert rc == rtcdf.OK and bits == 0
            assert_matches_oracle(x, out, mn, mn + R)


def test_host_and_device_generators_agree():
    for dist in DISTS:
        for R, mn in ((128, 0), (1 << 14, -1000), (1 << 18, (1 << 31) - (1 << 18)), (3, -(1 << 31))):
            seed = gen.derive_seed(17, dist, R)
            d = dev_keys(300_000, mn, R, dist, seed, first=12345).cpu().numpy()
            h = gen.keys_host(300_000, mn, R, dist, seed, first=12345)
            np.testing.assert_array_equal(d, h)


# ---------------------------------------------------------------- full-size workloads
SWEEP_R = [1 << 7, 1 << 10, 1 << 14, 1 << 18]


@pytest.mark.parametrize("R", SWEEP_R)
@pytest.mark.parametrize("dist", DISTS)
def test_sweep_n1e8_exact(R, dist):
    """Sweep workload: n = 1e8, minVal = -1000, default launch plan (the one
    the benchmark times); full element-by-element comparison."""
    n, mn = 100_000_000, -1000
    x = dev_keys(n, mn, R, dist, gen.derive_seed(1, dist, R.bit_length() - 1))
    out = gpu_sort(x, mn, mn + R)
    assert_matches_oracle(x, out, mn, mn + R)
    del x, out
    torch.cuda.empty_cache()


@pytest.mark.parametrize("R,dist", [(1 << 12, gen.UNIFORM), (1 << 16, gen.NORMAL), (1 << 18, gen.UNIFORM),
                                    (1 << 18, gen.NORMAL)])
def test_large_n1e9(R, dist):
    """Large workload: n = 1e9 (4 GB in, 4 GB out).  Checked with the oracle's
    invariant checker (Lemma 3: every position holds the value whose interval
    contains it, computed from the input's CDF).  R = 2^18 normal is the
    five-tile histogram with one tile holding 58 % of the keys, where the
    L2 prefetch is switched off from the input sample."""
    n = 1_000_000_000
    x = dev_keys(n, 0, R, dist, gen.derive_seed(2, dist, R.bit_length() - 1))
    out = gpu_sort(x, 0, R)
    a = x.cpu().numpy()
    b = out.cpu().numpy()
    del x, out
    torch.cuda.empty_cache()
    ok, bad = oracle.check_sorted(a, b, 0, R)
    assert ok, f"first bad position {bad}"


def test_largest_n_accepted():
    """n = 2^32 - 1, the largest length the ABI accepts (32-bit counts and
    positions): 17 GB in, 17 GB out, checked with the oracle's Lemma-3 checker;
    n = 2^32 is refused on the host."""
    n = (1 << 32) - 1
    R = 1 << 12
    x = dev_keys(n, -9, R, gen.UNIFORM, gen.derive_seed(4, 32))
    out = gpu_sort(x, -9, -9 + R)
    a = x.cpu().numpy()
    b = out.cpu().numpy()
    assert rtcdf.rtcdf_sort(x.data_ptr(), out.data_ptr(), n + 1, -9, -9 + R,
                            stream_handle()) == rtcdf.ERR_INVALID_ARG
    del x, out
    torch.cuda.empty_cache()
    ok, bad = oracle.check_sorted(a, b, -9, -9 + R)
    assert ok, f"first bad position {bad}"


def test_bounded_wait_runs_out_and_reports_timeout():
    """Failure detection without a GPU fault: a workspace whose scan ticket is
    not zero makes one lookback chunk go unpublished; its successor's bounded
    wait runs out, the sort returns, the device status says TIMEOUT, and the
    context stays usable (the next sort on a cleared workspace is exact)."""
    R, n = 1 << 14, 200_000                      # four scan chunks
    x = dev_keys(n, 0, R, gen.UNIFORM, gen.derive_seed(80))
    out = torch.empty_like(x)
    wsb = rtcdf.rtcdf_workspace_size(R)
    ws = torch.zeros(wsb // 4 + 64, dtype=torch.int32, device="cuda")
    ws[1] = 1                                    # control block word 1: the scan ticket
    s = stream_handle()
    p = rtcdf.Params(hist_threads=1024)
    rc = rtcdf.rtcdf_sort_ex(x.data_ptr(), out.data_ptr(), n, 0, R, p, ws.data_ptr(), wsb, None, s)
    assert rc == rtcdf.OK
    rc, bits = rtcdf.rtcdf_ws_status_get(ws.data_ptr(), s)
    assert rc == rtcdf.ERR_TIMEOUT and bits & rtcdf.DEV_TIMEOUT, (rc, bits)
    ws.zero_()
    out.fill_(0)
    rc = rtcdf.rtcdf_sort_ex(x.data_ptr(), out.data_ptr(), n, 0, R, p, ws.data_ptr(), wsb, None, s)
    assert rc == rtcdf.OK
    assert rtcdf.rtcdf_ws_status_get(ws.data_ptr(), s) == (rtcdf.OK, 0)
    assert_matches_oracle(x, out, 0, R)
