"""C-ABI checks that need no GPU: the libraries load, export every declared
symbol, and reject bad arguments on the host before touching the device."""
import ctypes
import os
import re

import pytest

from paper_2609_00843_gb300 import _build, rtcdf

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    _build.build()


def _declared(header):
    text = open(os.path.join(ROOT, "include", header)).read()
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(rtcdf_\w+)\s*\(", text, re.M)))


def test_rtcdf_exports_every_declared_symbol():
    names = _declared("rtcdf.h")
    assert "rtcdf_sort" in names and "rtcdf_sort_ws" in names and len(names) >= 10
    lib = ctypes.CDLL(rtcdf.LIB_PATH)
    for name in names:
        assert hasattr(lib, name), name
    assert names == rtcdf.declared_functions()


def test_gen_exports_every_declared_symbol():
    from paper_2609_00843_gb300 import gen
    lib = ctypes.CDLL(gen.lib_path())
    for name in _declared("rtcdf_gen.h"):
        assert hasattr(lib, name), name


def test_version_and_status_strings():
    assert "sm_103a" in rtcdf.rtcdf_version()
    for code in range(7):
        assert rtcdf.rtcdf_status_str(code) != "unknown status"
    assert rtcdf.rtcdf_status_str(99) == "unknown status"


def test_workspace_size_is_linear_in_R_and_independent_of_n():
    s1 = rtcdf.rtcdf_workspace_size(128)
    s2 = rtcdf.rtcdf_workspace_size(1 << 18)
    assert 0 < s1 < s2
    # O(R): three 4-byte arrays of R entries plus small fixed regions.
    assert 12 * (1 << 18) <= s2 < 12 * (1 << 18) + 64 * 1024
    with pytest.raises(rtcdf.RtcdfError):
        rtcdf.rtcdf_workspace_size(0)
    with pytest.raises(rtcdf.RtcdfError):
        rtcdf.rtcdf_workspace_size(rtcdf.MAX_R + 1)


@pytest.mark.parametrize("minVal,maxVal,code", [
    (5, 5, rtcdf.ERR_RANGE),
    (5, 4, rtcdf.ERR_RANGE),
    (0, rtcdf.MAX_R + 1, rtcdf.ERR_RANGE),
    (-(1 << 31) - 1, 0, rtcdf.ERR_RANGE),
    ((1 << 31) - 2, (1 << 31) + 1, rtcdf.ERR_RANGE),
])
def test_range_errors_on_host(minVal, maxVal, code):
    assert rtcdf.rtcdf_sort(4096, 8192, 10, minVal, maxVal, 0) == code


def test_argument_errors_on_host():
    # null pointers, misalignment, partial overlap, n >= 2^32 -- all rejected
    # before any CUDA call, so they run without a GPU.
    assert rtcdf.rtcdf_sort(0, 8192, 10, 0, 128, 0) == rtcdf.ERR_INVALID_ARG
    assert rtcdf.rtcdf_sort(4096, 0, 10, 0, 128, 0) == rtcdf.ERR_INVALID_ARG
    assert rtcdf.rtcdf_sort(4098, 8192, 10, 0, 128, 0) == rtcdf.ERR_INVALID_ARG
    assert rtcdf.rtcdf_sort(4096, 4100, 10, 0, 128, 0) == rtcdf.ERR_INVALID_ARG
    assert rtcdf.rtcdf_sort(4096, 8192, 1 << 32, 0, 128, 0) == rtcdf.ERR_INVALID_ARG
    # n == 0 is a no-op
    assert rtcdf.rtcdf_sort(0, 0, 0, 0, 128, 0) == rtcdf.OK
    # caller workspace: null or misaligned workspace, too small
    assert rtcdf.rtcdf_sort_ws(4096, 1 << 20, 10, 0, 128, 0, 1 << 20, 0) == rtcdf.ERR_INVALID_ARG
    assert rtcdf.rtcdf_sort_ws(4096, 1 << 20, 10, 0, 128, 1 << 24 | 8, 1 << 20, 0) == rtcdf.ERR_INVALID_ARG
    assert rtcdf.rtcdf_sort_ws(4096, 1 << 20, 10, 0, 128, 1 << 24, 16, 0) == rtcdf.ERR_NO_MEMORY


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    monkeypatch.setattr(rtcdf, "_lib", None)
    monkeypatch.setattr(rtcdf, "LIB_PATH", str(tmp_path / "nope.so"))
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        rtcdf.rtcdf_sort(0, 0, 0, 0, 1, 0)


def test_batched_plan_rejects_bad_metadata_on_host():
    import ctypes
    import numpy as np
    lib = rtcdf.lib()
    h = ctypes.c_void_p(0)

    def create(offs, mn, mx):
        o = np.asarray(offs, np.int64); a = np.asarray(mn, np.int64); b = np.asarray(mx, np.int64)
        return lib.rtcdf_batch_plan_create(o.ctypes.data_as(ctypes.c_void_p),
                                           a.ctypes.data_as(ctypes.c_void_p),
                                           b.ctypes.data_as(ctypes.c_void_p), len(a), ctypes.byref(h))
    assert create([0, 10, 5], [0, 0], [4, 4]) == rtcdf.ERR_INVALID_ARG       # offsets decrease
    assert create([-1, 10], [0], [4]) == rtcdf.ERR_INVALID_ARG               # negative offset
    assert create([0, 10], [3], [3]) == rtcdf.ERR_RANGE                      # R = 0
    assert create([0, 10], [0], [(1 << 20) + 1]) == rtcdf.ERR_RANGE          # R too wide
    assert create([0, 10], [-(1 << 31) - 1], [0]) == rtcdf.ERR_RANGE         # outside int32
    assert lib.rtcdf_batch_plan_create(None, None, None, -1, ctypes.byref(h)) == rtcdf.ERR_INVALID_ARG


@pytest.mark.parametrize("field,value", [("hist_chunk", 100), ("hist_chunk", -1), ("fill_chunk", 4095),
                                         ("small_max_n", 65536), ("small_max_n", -2),
                                         ("small_scan_max_R", 16769), ("small_scan_max_R", -1),
                                         ("small_by_time", 2), ("small_by_time", -2)])
def test_batched_plan_rejects_bad_work_item_sizes_on_host(field, value):
    import ctypes
    import numpy as np
    o = np.asarray([0, 10], np.int64); a = np.asarray([0], np.int64); b = np.asarray([4], np.int64)
    p = rtcdf.BatchParams(**{field: value})
    h = ctypes.c_void_p(0)
    rc = rtcdf.lib().rtcdf_batch_plan_create_ex(o.ctypes.data_as(ctypes.c_void_p),
                                                a.ctypes.data_as(ctypes.c_void_p),
                                                b.ctypes.data_as(ctypes.c_void_p), 1, ctypes.byref(p),
                                                ctypes.byref(h))
    assert rc == rtcdf.ERR_INVALID_ARG and not h.value


def test_server_rejects_bad_config_and_requests_on_host():
    import ctypes
    lib = rtcdf.lib()
    res = (rtcdf.Result * 2)()
    st = rtcdf.ServeStats()
    good = rtcdf.make_requests([10, 20], [0, -5], [128, 1000], [0, 1], [1, 2], [0.0, 0.0])

    def cfg(**kw):
        c = rtcdf.ServerConfig(budget_bytes=1 << 30, num_streams=2, max_batch=8, single_min_keys=1 << 20,
                               fill=1, digests=0, max_large_inflight=0)
        for k, v in kw.items():
            setattr(c, k, v)
        return c

    for fname in ("rtcdf_serve_trace", "rtcdf_serve_sequential"):
        f = getattr(lib, fname)
        assert f(None, good, 2, res, ctypes.byref(st)) == rtcdf.ERR_INVALID_ARG
        assert f(ctypes.byref(cfg(fill=None)), good, 2, res, ctypes.byref(st)) == rtcdf.ERR_INVALID_ARG
        assert f(ctypes.byref(cfg()), None, 2, res, ctypes.byref(st)) == rtcdf.ERR_INVALID_ARG
        assert f(ctypes.byref(cfg()), good, 2, None, ctypes.byref(st)) == rtcdf.ERR_INVALID_ARG
        assert f(ctypes.byref(cfg()), good, -1, res, ctypes.byref(st)) == rtcdf.ERR_INVALID_ARG
        for n, mn, mx in [(10, 5, 5), (10, 0, rtcdf.MAX_R + 1), (10, -(1 << 31) - 1, 0), (1 << 32, 0, 128)]:
            bad = rtcdf.make_requests([10, n], [0, mn], [128, mx], [0, 0], [1, 2], [0.0, 0.0])
            assert f(ctypes.byref(cfg()), bad, 2, res, ctypes.byref(st)) == rtcdf.ERR_RANGE
    # the continuous-batching server also bounds streams, batch size and R (segmented launches)
    trace = lib.rtcdf_serve_trace
    for kw in ({"num_streams": 0}, {"num_streams": 17}, {"max_batch": 0}):
        assert trace(ctypes.byref(cfg(**kw)), good, 2, res, ctypes.byref(st)) == rtcdf.ERR_INVALID_ARG
    wide = rtcdf.make_requests([10], [0], [(1 << 20) + 1], [0], [1], [0.0])
    assert trace(ctypes.byref(cfg()), wide, 1, res, ctypes.byref(st)) == rtcdf.ERR_RANGE


def test_sharded_entry_points_reject_bad_arguments_on_host():
    # Every case returns before any CUDA call, so it runs without a GPU.
    h, f = rtcdf.rtcdf_hist_accumulate, rtcdf.rtcdf_fill_from_counts
    assert h(4096, 10, 5, 5, 1 << 20, 0) == rtcdf.ERR_RANGE                  # R = 0
    assert h(4096, 10, 0, rtcdf.MAX_R + 1, 1 << 20, 0) == rtcdf.ERR_RANGE
    assert h(4096, 10, 0, 128, 0, 0) == rtcdf.ERR_INVALID_ARG                # null counts
    assert h(4096, 10, 0, 128, (1 << 20) + 2, 0) == rtcdf.ERR_INVALID_ARG    # misaligned counts
    assert h(0, 10, 0, 128, 1 << 20, 0) == rtcdf.ERR_INVALID_ARG             # null input
    assert h(4098, 10, 0, 128, 1 << 20, 0) == rtcdf.ERR_INVALID_ARG          # misaligned input
    assert h(4096, 1 << 32, 0, 128, 1 << 30, 0) == rtcdf.ERR_INVALID_ARG     # n >= 2^32
    assert h(4096, 1000, 0, 128, 4096 + 400, 0) == rtcdf.ERR_INVALID_ARG     # input overlaps counts
    assert h(0, 0, 0, 128, 1 << 20, 0) == rtcdf.OK                           # empty slice
    ws = 1 << 24
    wsb = rtcdf.rtcdf_workspace_size(128)
    assert f(1 << 20, 100, 3, 3, 0, 100, 1 << 22, ws, wsb, 0) == rtcdf.ERR_RANGE
    assert f(1 << 20, 1 << 32, 0, 128, 0, 100, 1 << 22, ws, wsb, 0) == rtcdf.ERR_INVALID_ARG
    assert f(1 << 20, 100, 0, 128, 60, 50, 1 << 22, ws, wsb, 0) == rtcdf.ERR_INVALID_ARG   # begin > end
    assert f(1 << 20, 100, 0, 128, 0, 101, 1 << 22, ws, wsb, 0) == rtcdf.ERR_INVALID_ARG   # end > n
    assert f(0, 100, 0, 128, 0, 100, 1 << 22, ws, wsb, 0) == rtcdf.ERR_INVALID_ARG         # null counts
    assert f(1 << 20, 100, 0, 128, 0, 100, 0, ws, wsb, 0) == rtcdf.ERR_INVALID_ARG         # null out
    assert f(1 << 20, 100, 0, 128, 0, 100, (1 << 22) + 1, ws, wsb, 0) == rtcdf.ERR_INVALID_ARG
    assert f(1 << 20, 100, 0, 128, 0, 100, 1 << 22, ws + 16, wsb, 0) == rtcdf.ERR_INVALID_ARG
    assert f(1 << 20, 100, 0, 128, 0, 100, 1 << 22, ws, 64, 0) == rtcdf.ERR_NO_MEMORY
    assert f(1 << 20, 100, 0, 128, 0, 100, (1 << 20) + 64, ws, wsb, 0) == rtcdf.ERR_INVALID_ARG  # out on counts
    assert f(1 << 20, 100, 0, 128, 0, 100, ws + 256, ws, wsb, 0) == rtcdf.ERR_INVALID_ARG  # out on workspace
    assert f(1 << 20, 100, 0, 128, 40, 40, 0, 0, 0, 0) == rtcdf.OK           # empty window


def test_device_planned_segmented_sort_rejects_bad_arguments_on_host():
    # All returned before any CUDA call.
    size = rtcdf.rtcdf_batch_device_workspace_size
    assert 0 < size(10, 1000, 100) < size(10, 1000, 1 << 20) < size(20, 1000, 1 << 20)
    assert size(10, 1000, 100) < size(10, 10**9, 100)
    for bad in ((10, 1000, 0), (10, 1000, (1 << 20) + 1)):
        with pytest.raises(rtcdf.RtcdfError):
            size(*bad)
    f = rtcdf.rtcdf_sort_batched_device_ws
    inp, out, o, a, b, ws = 1 << 24, 1 << 26, 1 << 20, (1 << 20) + 4096, (1 << 20) + 8192, 1 << 28
    wsb = size(3, 1000, 100)
    ok = dict(S=3, N=1000, R=100)

    def call(i=inp, q=out, oo=o, aa=a, bb=b, S=3, N=1000, R=100, w=ws, wb=wsb):
        return f(i, q, oo, aa, bb, S, N, R, w, wb, 0)
    assert call(S=-1) == rtcdf.ERR_INVALID_ARG
    assert call(R=0) == rtcdf.ERR_RANGE and call(R=(1 << 20) + 1) == rtcdf.ERR_RANGE
    assert call(N=1 << 40) == rtcdf.ERR_INVALID_ARG
    assert call(S=0) == rtcdf.OK and call(N=0) == rtcdf.OK      # nothing to sort
    assert call(i=0) == rtcdf.ERR_INVALID_ARG and call(oo=0) == rtcdf.ERR_INVALID_ARG
    assert call(w=0) == rtcdf.ERR_INVALID_ARG
    assert call(i=inp + 2) == rtcdf.ERR_INVALID_ARG              # keys 4-byte aligned
    assert call(oo=o + 4) == rtcdf.ERR_INVALID_ARG               # metadata 8-byte aligned
    assert call(w=ws + 128) == rtcdf.ERR_INVALID_ARG             # workspace 256-byte aligned
    assert call(q=inp + 400) == rtcdf.ERR_INVALID_ARG            # partial overlap
    assert call(wb=wsb - 4) == rtcdf.ERR_NO_MEMORY
    g = rtcdf.rtcdf_sort_batched
    assert g(inp, out, o, a, b, -1, 1000, 100, 0) == rtcdf.ERR_INVALID_ARG
    assert g(inp, out, o, a, b, 3, 1000, 0, 0) == rtcdf.ERR_RANGE
    assert g(inp, out, o, a, b, 0, 1000, 100, 0) == rtcdf.OK
    assert g(0, out, o, a, b, 3, 1000, 100, 0) == rtcdf.ERR_INVALID_ARG
    assert ok
