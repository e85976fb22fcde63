"""Python binding of librtcdf (include/rtcdf.h): argument marshalling only.

Every function named ``rtcdf_*`` here calls the C entry point of the same name
with plain integers (device pointers, sizes, a ``cudaStream_t`` handle) and
returns what it returns.  :func:`sort` is a convenience over torch tensors.
There is no fallback: if the CUDA library is missing, every call raises.
"""
from __future__ import annotations

import ctypes
import os
import re
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "librtcdf.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "rtcdf.h")

OK = 0
ERR_INVALID_ARG = 1
ERR_RANGE = 2
ERR_KEY_OUT_OF_RANGE = 3
ERR_CUDA = 4
ERR_NO_MEMORY = 5
ERR_TIMEOUT = 6
DEV_KEY_OUT_OF_RANGE = 0x1
DEV_TIMEOUT = 0x2
DEV_BAD_SEGMENT = 0x4
MAX_R = 1 << 24
STATIC_MAX_R = 1 << 16

_lock = threading.Lock()
_lib = None


class RtcdfError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        msg = status_str(code) if _lib is not None else str(code)
        super().__init__(f"{what}: rtcdf status {code} ({msg})")
        self.code = code


class Params(ctypes.Structure):
    _fields_ = [("tile_width", ctypes.c_int32), ("hist_ctas_per_tile", ctypes.c_int32),
                ("hist_threads", ctypes.c_int32), ("fill_ctas", ctypes.c_int32),
                ("fill_threads", ctypes.c_int32), ("fill_chunk", ctypes.c_int32),
                ("reserved", ctypes.c_int32 * 2)]


class BatchParams(ctypes.Structure):
    _fields_ = [("hist_chunk", ctypes.c_int32), ("fill_chunk", ctypes.c_int32),
                ("small_max_n", ctypes.c_int32), ("small_scan_max_R", ctypes.c_int32),
                ("small_by_time", ctypes.c_int32), ("reserved", ctypes.c_int32 * 3)]


class TuneEntry(ctypes.Structure):
    _fields_ = [("log2_R", ctypes.c_int32), ("n_class", ctypes.c_int32), ("params", Params)]


class TuneCase(ctypes.Structure):
    _fields_ = [("in_ptr", ctypes.c_void_p), ("out_ptr", ctypes.c_void_p), ("n", ctypes.c_uint64),
                ("minVal", ctypes.c_int64), ("maxVal", ctypes.c_int64)]


class Debug(ctypes.Structure):
    _fields_ = [("tile_hist", ctypes.c_void_p), ("cdf", ctypes.c_void_p),
                ("tile_offset", ctypes.c_void_p), ("stage_events", ctypes.c_void_p * 4)]


class BatchInfo(ctypes.Structure):
    _fields_ = [("num_segments", ctypes.c_uint32), ("small_segments", ctypes.c_uint32),
                ("large_segments", ctypes.c_uint32), ("work_items", ctypes.c_uint32),
                ("workers", ctypes.c_uint32), ("reserved", ctypes.c_uint32),
                ("total_keys", ctypes.c_uint64), ("workspace_bytes", ctypes.c_uint64)]


class ServerConfig(ctypes.Structure):
    _fields_ = [("budget_bytes", ctypes.c_uint64), ("num_streams", ctypes.c_int32),
                ("max_batch", ctypes.c_int32), ("single_min_keys", ctypes.c_uint64),
                ("fill", ctypes.c_void_p), ("digests", ctypes.c_int32),
                ("max_large_inflight", ctypes.c_int32), ("outputs", ctypes.c_void_p),
                ("large_priority", ctypes.c_int32), ("reserved2", ctypes.c_int32),
                ("fill_at_launch", ctypes.c_int32), ("large_queue_burst", ctypes.c_int32)]


class Request(ctypes.Structure):
    _fields_ = [("n", ctypes.c_uint64), ("minVal", ctypes.c_int64), ("maxVal", ctypes.c_int64),
                ("dist", ctypes.c_int32), ("reserved", ctypes.c_int32), ("seed", ctypes.c_uint64),
                ("arrival_s", ctypes.c_double)]


class Result(ctypes.Structure):
    _fields_ = [("admit_s", ctypes.c_double), ("launch_s", ctypes.c_double),
                ("done_s", ctypes.c_double), ("digest", ctypes.c_uint64),
                ("status", ctypes.c_int32), ("batch_id", ctypes.c_int32)]


class ServeStats(ctypes.Structure):
    _fields_ = [("makespan_s", ctypes.c_double), ("total_keys", ctypes.c_uint64),
                ("launches_batched", ctypes.c_uint64), ("launches_single", ctypes.c_uint64),
                ("batched_requests", ctypes.c_uint64), ("peak_bytes", ctypes.c_uint64),
                ("max_inflight", ctypes.c_int32), ("reserved", ctypes.c_int32)]


def declared_functions() -> list[str]:
    """Names of the functions declared in include/rtcdf.h."""
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(rtcdf_\w+)\s*\(", text, re.M)))


def lib():
    """The loaded CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(
                    f"librtcdf.so not found at {LIB_PATH}; build it with "
                    "paper_2609_00843_gb300._build.build() (no CPU fallback exists)")
            L = ctypes.CDLL(LIB_PATH)
            vp, u64, i64, i32 = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int64, ctypes.c_int32
            sz = ctypes.c_size_t
            L.rtcdf_sort.argtypes = [vp, vp, u64, i64, i64, vp]
            L.rtcdf_sort_ws.argtypes = [vp, vp, u64, i64, i64, vp, sz, vp]
            L.rtcdf_sort_ex.argtypes = [vp, vp, u64, i64, i64, ctypes.POINTER(Params), vp, sz,
                                        ctypes.POINTER(Debug), vp]
            L.rtcdf_reserve.argtypes = [i64, vp]
            L.rtcdf_workspace_size.argtypes = [i64, ctypes.POINTER(sz)]
            L.rtcdf_status_get.argtypes = [vp, ctypes.POINTER(i32)]
            L.rtcdf_ws_status_get.argtypes = [vp, vp, ctypes.POINTER(i32)]
            L.rtcdf_plan.argtypes = [u64, i64, ctypes.POINTER(Params)]
            L.rtcdf_sort_static.argtypes = [vp, vp, u64, i64, i64, vp]
            L.rtcdf_hist_accumulate.argtypes = [vp, u64, i64, i64, vp, vp]
            L.rtcdf_fill_from_counts.argtypes = [vp, u64, i64, i64, u64, u64, vp, vp, sz, vp]
            L.rtcdf_sort_host.argtypes = [vp, vp, u64, i64, i64, vp]
            L.rtcdf_batch_plan_create.argtypes = [vp, vp, vp, i32, ctypes.POINTER(vp)]
            L.rtcdf_batch_plan_create_ex.argtypes = [vp, vp, vp, i32, ctypes.POINTER(BatchParams),
                                                     ctypes.POINTER(vp)]
            L.rtcdf_batch_plan_create_ex.restype = ctypes.c_int
            L.rtcdf_batch_plan_destroy.argtypes = [vp]
            L.rtcdf_batch_workspace_size.argtypes = [vp, ctypes.POINTER(sz)]
            L.rtcdf_batch_plan_info.argtypes = [vp, ctypes.POINTER(BatchInfo)]
            L.rtcdf_sort_batched_ws.argtypes = [vp, vp, vp, vp, sz, vp]
            L.rtcdf_batch_status_get.argtypes = [vp, vp, ctypes.POINTER(i32)]
            L.rtcdf_sort_batched_profiled.argtypes = [vp, vp, vp, vp, sz, vp, vp]
            L.rtcdf_sort_batched_profiled.restype = ctypes.c_int
            L.rtcdf_sort_batched_host.argtypes = [vp, vp, vp, vp, vp, i32, vp]
            L.rtcdf_sort_batched.argtypes = [vp, vp, vp, vp, vp, i32, u64, i64, vp]
            L.rtcdf_sort_batched_device_ws.argtypes = [vp, vp, vp, vp, vp, i32, u64, i64, vp, sz, vp]
            L.rtcdf_batch_device_workspace_size.argtypes = [i32, u64, i64, ctypes.POINTER(sz)]
            L.rtcdf_batch_reserve.argtypes = [i32, u64, i64, vp]
            L.rtcdf_tune_n_class.argtypes = [u64]
            L.rtcdf_tune_n_class.restype = i32
            L.rtcdf_tune_set.argtypes = [ctypes.POINTER(TuneEntry), i32]
            L.rtcdf_tune_reset.argtypes = []
            L.rtcdf_tune_get.argtypes = [ctypes.POINTER(TuneEntry), i32, ctypes.POINTER(i32)]
            L.rtcdf_autotune.argtypes = [ctypes.POINTER(TuneCase), i32, ctypes.POINTER(Params), i32,
                                         i32, vp, sz, ctypes.POINTER(ctypes.c_float),
                                         ctypes.POINTER(ctypes.c_double), ctypes.POINTER(i32), vp]
            for f in ("rtcdf_tune_set", "rtcdf_tune_reset", "rtcdf_tune_get", "rtcdf_autotune"):
                getattr(L, f).restype = ctypes.c_int
            for f in ("rtcdf_serve_trace", "rtcdf_serve_sequential"):
                getattr(L, f).argtypes = [ctypes.POINTER(ServerConfig), ctypes.POINTER(Request),
                                          i64, ctypes.POINTER(Result), ctypes.POINTER(ServeStats)]
                getattr(L, f).restype = ctypes.c_int
            for f in ("rtcdf_sort", "rtcdf_sort_ws", "rtcdf_sort_ex", "rtcdf_reserve",
                      "rtcdf_workspace_size", "rtcdf_status_get", "rtcdf_ws_status_get",
                      "rtcdf_plan", "rtcdf_sort_static", "rtcdf_sort_host", "rtcdf_batch_plan_create",
                      "rtcdf_batch_plan_destroy", "rtcdf_batch_workspace_size",
                      "rtcdf_batch_plan_info", "rtcdf_sort_batched_ws", "rtcdf_batch_status_get",
                      "rtcdf_sort_batched", "rtcdf_hist_accumulate", "rtcdf_fill_from_counts",
                      "rtcdf_sort_batched_host", "rtcdf_sort_batched_device_ws",
                      "rtcdf_batch_device_workspace_size", "rtcdf_batch_reserve"):
                getattr(L, f).restype = ctypes.c_int
            L.rtcdf_status_str.argtypes = [ctypes.c_int]
            L.rtcdf_status_str.restype = ctypes.c_char_p
            L.rtcdf_version.restype = ctypes.c_char_p
            _lib = L
    return _lib


# ---------------------------------------------------------------- C entry points
def rtcdf_sort(in_ptr: int, out_ptr: int, n: int, minVal: int, maxVal: int, stream: int = 0) -> int:
    return lib().rtcdf_sort(in_ptr, out_ptr, n, minVal, maxVal, stream)


def rtcdf_sort_ws(in_ptr, out_ptr, n, minVal, maxVal, ws_ptr, ws_bytes, stream=0) -> int:
    return lib().rtcdf_sort_ws(in_ptr, out_ptr, n, minVal, maxVal, ws_ptr, ws_bytes, stream)


def rtcdf_sort_ex(in_ptr, out_ptr, n, minVal, maxVal, params: Params | None, ws_ptr, ws_bytes,
                  debug: Debug | None = None, stream=0) -> int:
    p = ctypes.byref(params) if params is not None else None
    d = ctypes.byref(debug) if debug is not None else None
    return lib().rtcdf_sort_ex(in_ptr, out_ptr, n, minVal, maxVal, p, ws_ptr, ws_bytes, d, stream)


def rtcdf_sort_static(in_ptr: int, out_ptr: int, n: int, minVal: int, maxVal: int,
                      stream: int = 0) -> int:
    return lib().rtcdf_sort_static(in_ptr, out_ptr, n, minVal, maxVal, stream)


def rtcdf_hist_accumulate(in_ptr: int, n: int, minVal: int, maxVal: int, counts_ptr: int,
                          stream: int = 0) -> int:
    """Add the counts of n device keys into a device uint32[R] array."""
    return lib().rtcdf_hist_accumulate(in_ptr, n, minVal, maxVal, counts_ptr, stream)


def rtcdf_fill_from_counts(counts_ptr: int, total_n: int, minVal: int, maxVal: int, pos_begin: int,
                           pos_end: int, out_ptr: int, ws_ptr: int, ws_bytes: int,
                           stream: int = 0) -> int:
    """Write positions [pos_begin, pos_end) of the sorted array with the given
    global counts into out (out[0] = position pos_begin)."""
    return lib().rtcdf_fill_from_counts(counts_ptr, total_n, minVal, maxVal, pos_begin, pos_end,
                                        out_ptr, ws_ptr, ws_bytes, stream)


def _i64_array(xs):
    import numpy as np
    a = np.ascontiguousarray(np.asarray(xs, dtype=np.int64))
    return a, a.ctypes.data_as(ctypes.c_void_p)


BATCH_PROFILE_WORDS = 20
BATCH_ITEM_KINDS = ("hist", "small", "scan", "fill")


def batch_profile_summary(words, workers: int) -> dict:
    """Turn the profile words of rtcdf_sort_batched_profiled into per-kind
    figures: busy ms per resident CTA slot (sum of item durations / workers),
    items, start and end of the phase (ms from the first item), wait share."""
    t0 = min(words[8 + k] for k in range(4) if words[4 + k])
    out = {}
    for k, name in enumerate(BATCH_ITEM_KINDS):
        if not words[4 + k]:
            continue
        out[name] = {"items": int(words[4 + k]),
                     "busy_ms_per_worker": round(words[k] / workers / 1e6, 4),
                     "start_ms": round((words[8 + k] - t0) / 1e6, 4),
                     "end_ms": round((words[12 + k] - t0) / 1e6, 4),
                     "wait_share": round(words[16 + k] / words[k], 4) if words[k] else 0.0}
    return out


class BatchPlan:
    """A segmented-sort plan (rtcdf_batch_plan_create / _destroy)."""

    def __init__(self, seg_offsets, seg_minVal, seg_maxVal, params: BatchParams | None = None):
        self._keep = [_i64_array(seg_offsets), _i64_array(seg_minVal), _i64_array(seg_maxVal)]
        S = len(self._keep[1][0])
        if len(self._keep[0][0]) != S + 1 or len(self._keep[2][0]) != S:
            raise ValueError("seg_offsets needs S+1 entries, seg_minVal/seg_maxVal S entries")
        h = ctypes.c_void_p(0)
        rc = lib().rtcdf_batch_plan_create_ex(self._keep[0][1], self._keep[1][1], self._keep[2][1], S,
                                              ctypes.byref(params) if params is not None else None,
                                              ctypes.byref(h))
        if rc != OK:
            raise RtcdfError(rc, "rtcdf_batch_plan_create")
        self.handle = h

    def workspace_size(self) -> int:
        out = ctypes.c_size_t(0)
        rc = lib().rtcdf_batch_workspace_size(self.handle, ctypes.byref(out))
        if rc != OK:
            raise RtcdfError(rc, "rtcdf_batch_workspace_size")
        return out.value

    def info(self) -> dict:
        inf = BatchInfo()
        rc = lib().rtcdf_batch_plan_info(self.handle, ctypes.byref(inf))
        if rc != OK:
            raise RtcdfError(rc, "rtcdf_batch_plan_info")
        return {f: getattr(inf, f) for f, _ in BatchInfo._fields_ if f != "reserved"}

    def run(self, in_ptr: int, out_ptr: int, ws_ptr: int, ws_bytes: int, stream: int = 0) -> int:
        return lib().rtcdf_sort_batched_ws(self.handle, in_ptr, out_ptr, ws_ptr, ws_bytes, stream)

    def run_profiled(self, in_ptr: int, out_ptr: int, ws_ptr: int, ws_bytes: int,
                     prof_ptr: int, stream: int = 0) -> int:
        """rtcdf_sort_batched_profiled; prof_ptr: device array of PROFILE_WORDS uint64."""
        return lib().rtcdf_sort_batched_profiled(self.handle, in_ptr, out_ptr, ws_ptr, ws_bytes,
                                                 prof_ptr, stream)

    def close(self):
        if getattr(self, "handle", None):
            lib().rtcdf_batch_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def rtcdf_batch_status_get(ws_ptr: int, stream: int = 0) -> tuple[int, int]:
    bits = ctypes.c_int32(0)
    rc = lib().rtcdf_batch_status_get(ws_ptr, stream, ctypes.byref(bits))
    return rc, bits.value


def rtcdf_sort_batched_host(in_ptr: int, out_ptr: int, seg_offsets, seg_minVal, seg_maxVal,
                            stream: int = 0) -> int:
    """One-shot segmented sort over host metadata (synchronises)."""
    o, op = _i64_array(seg_offsets)
    mn, mnp = _i64_array(seg_minVal)
    mx, mxp = _i64_array(seg_maxVal)
    return lib().rtcdf_sort_batched_host(in_ptr, out_ptr, op, mnp, mxp, len(mn), stream)


def rtcdf_sort_batched(in_ptr: int, out_ptr: int, d_offsets_ptr: int, d_min_ptr: int, d_max_ptr: int,
                       num_segments: int, max_total_keys: int, max_R: int, stream: int = 0) -> int:
    """Segmented sort with int64 metadata in device memory, planned on the
    device (asynchronous; library-owned workspace per stream)."""
    return lib().rtcdf_sort_batched(in_ptr, out_ptr, d_offsets_ptr, d_min_ptr, d_max_ptr, num_segments,
                                    max_total_keys, max_R, stream)


def rtcdf_sort_batched_device_ws(in_ptr: int, out_ptr: int, d_offsets_ptr: int, d_min_ptr: int,
                                 d_max_ptr: int, num_segments: int, max_total_keys: int, max_R: int,
                                 ws_ptr: int, ws_bytes: int, stream: int = 0) -> int:
    """rtcdf_sort_batched with a caller workspace (no allocation; capturable)."""
    return lib().rtcdf_sort_batched_device_ws(in_ptr, out_ptr, d_offsets_ptr, d_min_ptr, d_max_ptr,
                                              num_segments, max_total_keys, max_R, ws_ptr, ws_bytes,
                                              stream)


def rtcdf_batch_device_workspace_size(num_segments: int, max_total_keys: int, max_R: int) -> int:
    out = ctypes.c_size_t(0)
    rc = lib().rtcdf_batch_device_workspace_size(num_segments, max_total_keys, max_R, ctypes.byref(out))
    if rc != OK:
        raise RtcdfError(rc, "rtcdf_batch_device_workspace_size")
    return out.value


def rtcdf_batch_reserve(num_segments: int, max_total_keys: int, max_R: int, stream: int = 0) -> int:
    return lib().rtcdf_batch_reserve(num_segments, max_total_keys, max_R, stream)


def make_requests(n, minVal, maxVal, dist, seed, arrival_s):
    """A ctypes array of rtcdf_request from equal-length sequences."""
    count = len(n)
    arr = (Request * max(1, count))()
    for i in range(count):
        arr[i] = Request(int(n[i]), int(minVal[i]), int(maxVal[i]), int(dist[i]), 0,
                         int(seed[i]) & ((1 << 64) - 1), float(arrival_s[i]))
    return arr


def _serve(fname, cfg: ServerConfig, reqs, count: int):
    results = (Result * max(1, count))()
    stats = ServeStats()
    rc = getattr(lib(), fname)(ctypes.byref(cfg), reqs, count, results, ctypes.byref(stats))
    if rc != OK:
        raise RtcdfError(rc, fname)
    return results, stats


def rtcdf_serve_trace(cfg: ServerConfig, reqs, count: int):
    """Continuous-batching server over a request trace; returns (results, stats)."""
    return _serve("rtcdf_serve_trace", cfg, reqs, count)


def rtcdf_serve_sequential(cfg: ServerConfig, reqs, count: int):
    """The same trace served one request at a time; returns (results, stats)."""
    return _serve("rtcdf_serve_sequential", cfg, reqs, count)


def rtcdf_sort_host(in_ptr: int, out_ptr: int, n: int, minVal: int, maxVal: int,
                    stream: int = 0) -> int:
    """Sort host buffers (pinned for overlap); returns when enqueued."""
    return lib().rtcdf_sort_host(in_ptr, out_ptr, n, minVal, maxVal, stream)


def rtcdf_reserve(max_R: int, stream: int = 0) -> int:
    return lib().rtcdf_reserve(max_R, stream)


def rtcdf_workspace_size(R: int) -> int:
    out = ctypes.c_size_t(0)
    rc = lib().rtcdf_workspace_size(R, ctypes.byref(out))
    if rc != OK:
        raise RtcdfError(rc, "rtcdf_workspace_size")
    return out.value


def rtcdf_status_get(stream: int = 0) -> tuple[int, int]:
    bits = ctypes.c_int32(0)
    rc = lib().rtcdf_status_get(stream, ctypes.byref(bits))
    return rc, bits.value


def rtcdf_ws_status_get(ws_ptr: int, stream: int = 0) -> tuple[int, int]:
    bits = ctypes.c_int32(0)
    rc = lib().rtcdf_ws_status_get(ws_ptr, stream, ctypes.byref(bits))
    return rc, bits.value


def rtcdf_plan(n: int, R: int) -> Params:
    p = Params()
    rc = lib().rtcdf_plan(n, R, ctypes.byref(p))
    if rc != OK:
        raise RtcdfError(rc, "rtcdf_plan")
    return p


def rtcdf_tune_n_class(n: int) -> int:
    return lib().rtcdf_tune_n_class(n)


def rtcdf_tune_set(entries) -> None:
    """Install a tuning table: an iterable of (log2_R, n_class, Params)."""
    entries = list(entries)
    arr = (TuneEntry * max(1, len(entries)))()
    for i, (lr, nc, p) in enumerate(entries):
        arr[i].log2_R, arr[i].n_class, arr[i].params = lr, nc, p
    rc = lib().rtcdf_tune_set(arr, len(entries))
    if rc != OK:
        raise RtcdfError(rc, "rtcdf_tune_set")


def rtcdf_tune_reset() -> None:
    rc = lib().rtcdf_tune_reset()
    if rc != OK:
        raise RtcdfError(rc, "rtcdf_tune_reset")


def rtcdf_tune_get() -> list:
    """The current tuning table as a list of (log2_R, n_class, Params)."""
    cnt = ctypes.c_int32(0)
    rc = lib().rtcdf_tune_get(None, 0, ctypes.byref(cnt))
    if rc != OK:
        raise RtcdfError(rc, "rtcdf_tune_get")
    arr = (TuneEntry * max(1, cnt.value))()
    rc = lib().rtcdf_tune_get(arr, cnt.value, ctypes.byref(cnt))
    if rc != OK:
        raise RtcdfError(rc, "rtcdf_tune_get")
    return [(arr[i].log2_R, arr[i].n_class, arr[i].params) for i in range(cnt.value)]


def rtcdf_autotune(cases, candidates, reps: int, ws_ptr: int, ws_bytes: int, stream: int = 0):
    """cases: iterable of (in_ptr, out_ptr, n, minVal, maxVal); candidates: Params list.
    Returns (times_ms [cases x candidates] as nested lists, geomeans, best index)."""
    cases = list(cases)
    candidates = list(candidates)
    carr = (TuneCase * len(cases))()
    for i, (ip, op, n, a, b) in enumerate(cases):
        carr[i].in_ptr, carr[i].out_ptr, carr[i].n, carr[i].minVal, carr[i].maxVal = ip, op, n, a, b
    parr = (Params * len(candidates))(*candidates)
    times = (ctypes.c_float * (len(cases) * len(candidates)))()
    gm = (ctypes.c_double * len(candidates))()
    best = ctypes.c_int32(-1)
    rc = lib().rtcdf_autotune(carr, len(cases), parr, len(candidates), reps, ws_ptr, ws_bytes,
                              times, gm, ctypes.byref(best), stream)
    if rc != OK:
        raise RtcdfError(rc, "rtcdf_autotune")
    k = len(candidates)
    t = [[times[c * k + j] for j in range(k)] for c in range(len(cases))]
    return t, [gm[j] for j in range(k)], best.value


def rtcdf_status_str(code: int) -> str:
    return lib().rtcdf_status_str(code).decode()


def rtcdf_version() -> str:
    return lib().rtcdf_version().decode()


status_str = rtcdf_status_str


# ---------------------------------------------------------------- torch convenience
def _stream_handle(stream) -> int:
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream) if hasattr(stream, "cuda_stream") else int(stream)


def sort(x, minVal: int, maxVal: int, out=None, stream=None, check: bool = False):
    """Sort a contiguous int32 CUDA tensor whose keys lie in [minVal, maxVal).

    Returns ``out`` (allocated if None).  With ``check=True`` the device status
    is read (a stream synchronisation) and an out-of-range key raises.
    """
    import torch
    if x.dtype != torch.int32 or not x.is_cuda or not x.is_contiguous():
        raise ValueError("x must be a contiguous int32 CUDA tensor")
    if out is None:
        out = torch.empty_like(x)
    s = _stream_handle(stream)
    rc = rtcdf_sort(x.data_ptr(), out.data_ptr(), x.numel(), int(minVal), int(maxVal), s)
    if rc != OK:
        raise RtcdfError(rc, "rtcdf_sort")
    if check:
        rc, _ = rtcdf_status_get(s)
        if rc != OK:
            raise RtcdfError(rc, "rtcdf_sort (device status)")
    return out
