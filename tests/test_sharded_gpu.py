"""Sharded single-array sort on one GPU: P ranks are emulated by P slices of
one array.  Each slice is counted with rtcdf_hist_accumulate into its own
counts array, the P arrays are summed on the device (the all-reduce), and
each rank's window of the sorted array is written by rtcdf_fill_from_counts
-- compared with the oracle's sorted array element by element.  The sorted
output depends on the global counts alone (Section 3.1, Algorithms 4 and 7;
Section 3.2, Lemma 3)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2609_00843_gb300 import _build, dist as rdist, gen, rtcdf
from gpu_util import dev_keys, stream_handle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    _build.build()
    torch.cuda.init()


def _check(rc, what):
    assert rc == rtcdf.OK, f"{what}: {rtcdf.rtcdf_status_str(rc)}"


def sharded(x, mn, R, P, pad=0):
    """Sort x as P emulated ranks; returns the P windows (each written with
    `pad` elements of offset into its own buffer, so windows start at every
    alignment) and the P local count arrays."""
    n = x.numel()
    s = stream_handle()
    local = []
    for r in range(P):
        lo, hi = rdist.slice_bounds(n, P, r)
        c = torch.zeros(R, dtype=torch.int32, device="cuda")
        _check(rtcdf.rtcdf_hist_accumulate(x[lo:].data_ptr() if hi > lo else 0, hi - lo, mn, mn + R,
                                           c.data_ptr(), s), "rtcdf_hist_accumulate")
        local.append(c)
    g = torch.stack(local).sum(dim=0, dtype=torch.int64).to(torch.int32)  # the all-reduce
    wsb = rtcdf.rtcdf_workspace_size(R)
    ws = torch.zeros(wsb // 4 + 64, dtype=torch.int32, device="cuda")
    windows = []
    for r in range(P):
        lo, hi = rdist.slice_bounds(n, P, r)
        buf = torch.full((hi - lo + pad + 1,), 0x7FFFFFFF, dtype=torch.int32, device="cuda")
        w = buf[pad:pad + hi - lo]
        _check(rtcdf.rtcdf_fill_from_counts(g.data_ptr(), n, mn, mn + R, lo, hi,
                                            w.data_ptr() if hi > lo else 0, ws.data_ptr(), wsb, s),
               "rtcdf_fill_from_counts")
        assert buf[pad + hi - lo].item() == 0x7FFFFFFF, "wrote past the window"
        windows.append(w)
    rc, bits = rtcdf.rtcdf_ws_status_get(ws.data_ptr(), s)
    assert rc == rtcdf.OK and bits == 0, (rc, bits)
    return windows, local


@pytest.mark.parametrize("n,R,dist,P", [
    (1_000_003, 128, gen.UNIFORM, 2), (1_000_003, 128, gen.UNIFORM, 8),
    (3_000_001, 1 << 18, gen.NORMAL, 4), (2_000_000, 1 << 14, gen.ALL_EQUAL, 3),
    (777_777, 60_000, gen.UNIFORM, 5), (1001, 1, gen.UNIFORM, 4), (5, 5000, gen.NORMAL, 8),
    (10_000_019, 1 << 16, gen.NORMAL, 2)])
def test_sharded_windows_match_oracle(n, R, dist, P):
    mn = -12345
    x = dev_keys(n, mn, R, dist, gen.derive_seed(61, n, R, dist, P))
    a = x.cpu().numpy()
    want = oracle.counting_sort(a, mn, mn + R)
    for pad in (0, 1, 3):
        windows, local = sharded(x, mn, R, P, pad)
        for r in range(P):
            lo, hi = rdist.slice_bounds(n, P, r)
            got = windows[r].cpu().numpy()
            bad = np.nonzero(got != want[lo:hi])[0]
            assert bad.size == 0, (f"P={P} rank {r} pad {pad}: {bad.size} positions of [{lo}, {hi}) "
                                   f"differ, first {(bad[:8] + lo).tolist()}")
            h = oracle.histogram(a[lo:hi], mn, mn + R)
            assert np.array_equal(local[r].cpu().numpy().astype(np.uint64), h), f"rank {r} counts"


def test_counts_of_several_slices_add_up():
    n, mn, R = 2_500_000, 3, 1 << 18
    x = dev_keys(n, mn, R, gen.UNIFORM, gen.derive_seed(62))
    c = torch.zeros(R, dtype=torch.int32, device="cuda")
    for lo, hi in ((0, 1), (1, 1_000_001), (1_000_001, n)):
        _check(rtcdf.rtcdf_hist_accumulate(x[lo:].data_ptr(), hi - lo, mn, mn + R, c.data_ptr(),
                                           stream_handle()), "accumulate")
    assert np.array_equal(c.cpu().numpy().astype(np.uint64), oracle.histogram(x.cpu().numpy(), mn, mn + R))


def test_counts_that_do_not_add_up_set_the_status():
    n, mn, R = 100_000, 0, 1000
    x = dev_keys(n, mn, R, gen.UNIFORM, gen.derive_seed(63))
    c = torch.zeros(R, dtype=torch.int32, device="cuda")
    s = stream_handle()
    _check(rtcdf.rtcdf_hist_accumulate(x.data_ptr(), n - 10, mn, mn + R, c.data_ptr(), s), "accumulate")
    wsb = rtcdf.rtcdf_workspace_size(R)
    ws = torch.zeros(wsb // 4 + 64, dtype=torch.int32, device="cuda")
    out = torch.empty(n, dtype=torch.int32, device="cuda")
    _check(rtcdf.rtcdf_fill_from_counts(c.data_ptr(), n, mn, mn + R, 0, n, out.data_ptr(), ws.data_ptr(),
                                        wsb, s), "fill")
    rc, bits = rtcdf.rtcdf_ws_status_get(ws.data_ptr(), s)
    assert rc == rtcdf.ERR_KEY_OUT_OF_RANGE and bits & rtcdf.DEV_KEY_OUT_OF_RANGE
    # the workspace is ready again: a consistent call on it is exact
    c.zero_()
    _check(rtcdf.rtcdf_hist_accumulate(x.data_ptr(), n, mn, mn + R, c.data_ptr(), s), "accumulate")
    _check(rtcdf.rtcdf_fill_from_counts(c.data_ptr(), n, mn, mn + R, 0, n, out.data_ptr(), ws.data_ptr(),
                                        wsb, s), "fill")
    rc, bits = rtcdf.rtcdf_ws_status_get(ws.data_ptr(), s)
    assert rc == rtcdf.OK and bits == 0
    assert np.array_equal(out.cpu().numpy(), oracle.counting_sort(x.cpu().numpy(), mn, mn + R))


def test_sharded_sorter_single_rank_equals_rtcdf_sort():
    """The torch-level helper with one rank (no process group): hist, no-op
    exchange, fill of the whole window."""
    n, mn, R = 4_000_037, -1000, 1 << 18
    x = dev_keys(n, mn, R, gen.NORMAL, gen.derive_seed(64))
    srt = rdist.ShardedSorter(R)
    out = torch.empty_like(x)
    srt.sort(x, n, mn, mn + R, out, rank=0, world=1)
    rc, bits = srt.status()
    assert rc == rtcdf.OK and bits == 0
    assert np.array_equal(out.cpu().numpy(), oracle.counting_sort(x.cpu().numpy(), mn, mn + R))
