"""Helpers for the GPU tests: device inputs from the seeded generator, calls
through the C ABI, and exact comparison with the CPU oracle."""
import numpy as np
import torch

import oracle
from paper_2609_00843_gb300 import gen, rtcdf


def dev_keys(n, minVal, R, dist, seed, first=0):
    x = torch.empty(int(n), dtype=torch.int32, device="cuda")
    if n:
        gen.keys_device(x.data_ptr(), n, minVal, R, dist, seed, first=first,
                        stream=torch.cuda.current_stream().cuda_stream)
    return x


def stream_handle():
    return torch.cuda.current_stream().cuda_stream


def gpu_sort(x, minVal, maxVal, out=None):
    if out is None:
        out = torch.empty_like(x)
    rc = rtcdf.rtcdf_sort(x.data_ptr() if x.numel() else 0, out.data_ptr() if out.numel() else 0,
                          x.numel(), int(minVal), int(maxVal), stream_handle())
    assert rc == rtcdf.OK, rtcdf.rtcdf_status_str(rc)
    rc, bits = rtcdf.rtcdf_status_get(stream_handle())
    assert rc == rtcdf.OK and bits == 0, (rc, bits)
    return out


def assert_matches_oracle(x, out, minVal, maxVal):
    a = x.cpu().numpy()
    want = oracle.counting_sort(a, minVal, maxVal)
    got = out.cpu().numpy()
    if not np.array_equal(got, want):
        bad = np.nonzero(got != want)[0]
        raise AssertionError(f"{bad.size} positions differ, first {bad[:8].tolist()}: "
                             f"got {got[bad[:8]].tolist()} want {want[bad[:8]].tolist()}")
