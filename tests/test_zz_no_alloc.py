"""The scratch-free entry point, rtcdf_sort_static.

It serves callers that cannot allocate device memory (code under another
framework's memory manager, fixed-budget serving loops, hot paths that cannot
take an allocation's synchronisation): its scratch is a fixed array inside
the library.  Its output must equal rtcdf_sort's, bit for bit, on consecutive
calls that reuse the same scratch.  This file is collected last so that a run
stopping at the first failure has already run every other test.
"""
import pytest
import torch

from paper_2609_00843_gb300 import _build, gen, rtcdf
from gpu_util import dev_keys, gpu_sort, stream_handle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    _build.build()
    torch.cuda.init()


def test_static_entry_matches_rtcdf_sort_on_two_calls_in_a_row():
    s = stream_handle()
    cases = [(1 << 16, gen.NORMAL, 3_000_001, -500), (1000, gen.UNIFORM, 1_000_003, 7),
             (1 << 16, gen.ALL_EQUAL, 65_537, 0)]
    for R, dist, n, mn in cases:
        x = dev_keys(n, mn, R, dist, gen.derive_seed(40, R, dist))
        want = gpu_sort(x, mn, mn + R)  # the existing entry point
        got = torch.full_like(x, 0x7FFFFFFF)
        rc = rtcdf.rtcdf_sort_static(x.data_ptr(), got.data_ptr(), n, mn, mn + R, s)
        assert rc == rtcdf.OK, rtcdf.rtcdf_status_str(rc)
        torch.cuda.synchronize()
        assert torch.equal(got, want), f"R={R} dist={dist}"


def test_static_entry_rejects_ranges_beyond_its_scratch():
    x = dev_keys(1000, 0, 100, gen.UNIFORM, 41)
    out = torch.full_like(x, -1)
    R = rtcdf.STATIC_MAX_R + 1
    rc = rtcdf.rtcdf_sort_static(x.data_ptr(), out.data_ptr(), 1000, 0, R, stream_handle())
    assert rc == rtcdf.ERR_RANGE
    torch.cuda.synchronize()
    assert (out == -1).all()
