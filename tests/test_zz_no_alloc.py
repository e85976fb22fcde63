"""The entry point that allocates nothing, rtcdf_sort_static.

It is for callers that cannot allocate device memory: code running under
another framework's memory manager that owns all of the device's memory,
serving loops whose memory budget is fixed before they start, and hot paths
that cannot take the synchronisation an allocation brings.  Its scratch is a
fixed array inside the library, shared by every call on a device, so each
case below runs two calls in a row on that array (and the cases follow one
another with ranges that grow and shrink, so that what one call leaves behind
meets the next).  Every output is compared element by element with the CPU
oracle and with the existing entry point rtcdf_sort.  This file is collected
last, so that a run stopping at the first failure has run every other test.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2609_00843_gb300 import _build, gen, rtcdf
from gpu_util import dev_keys, gpu_sort, stream_handle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    _build.build()
    torch.cuda.init()


def _static_sort(x, mn, mx):
    got = torch.full_like(x, 0x7FFFFFFF)
    rc = rtcdf.rtcdf_sort_static(x.data_ptr(), got.data_ptr(), x.numel(), mn, mx, stream_handle())
    assert rc == rtcdf.OK, rtcdf.rtcdf_status_str(rc)
    torch.cuda.synchronize()
    return got


def test_static_entry_matches_oracle_and_rtcdf_sort_on_two_calls_in_a_row():
    # (R, shape, n, minVal): the widest range the scratch serves first, then a
    # narrow one, then the widest again with every key equal (one long run
    # after many short ones), then narrow and all-equal.
    cases = [(1 << 16, gen.NORMAL, 3_000_001, -500), (1000, gen.UNIFORM, 1_000_003, 7),
             (1 << 16, gen.ALL_EQUAL, 65_537, 0), (1000, gen.ALL_EQUAL, 4_099, -3),
             (rtcdf.STATIC_MAX_R, gen.UNIFORM, 777_777, -(1 << 20))]
    for R, dist, n, mn in cases:
        for call in range(2):
            x = dev_keys(n, mn, R, dist, gen.derive_seed(40, R, dist, call))
            got = _static_sort(x, mn, mn + R)
            want = oracle.counting_sort(x.cpu().numpy(), mn, mn + R)
            g = got.cpu().numpy()
            bad = np.nonzero(g != want)[0]
            assert bad.size == 0, (f"R={R} dist={dist} call={call}: {bad.size} positions differ "
                                   f"from the oracle, first {bad[:8].tolist()}")
            assert torch.equal(got, gpu_sort(x, mn, mn + R)), f"R={R} dist={dist} call={call}"


def test_static_entry_rejects_ranges_beyond_its_scratch():
    x = dev_keys(1000, 0, 100, gen.UNIFORM, 41)
    out = torch.full_like(x, -1)
    R = rtcdf.STATIC_MAX_R + 1
    rc = rtcdf.rtcdf_sort_static(x.data_ptr(), out.data_ptr(), 1000, 0, R, stream_handle())
    assert rc == rtcdf.ERR_RANGE
    torch.cuda.synchronize()
    assert (out == -1).all()
