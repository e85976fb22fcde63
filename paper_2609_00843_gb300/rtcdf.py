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
                ("fill_threads", ctypes.c_int32), ("reserved", ctypes.c_int32 * 3)]


class Debug(ctypes.Structure):
    _fields_ = [("tile_hist", ctypes.c_void_p), ("cdf", ctypes.c_void_p),
                ("tile_offset", ctypes.c_void_p), ("stage_events", ctypes.c_void_p * 4)]


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
            for f in ("rtcdf_sort", "rtcdf_sort_ws", "rtcdf_sort_ex", "rtcdf_reserve",
                      "rtcdf_workspace_size", "rtcdf_status_get", "rtcdf_ws_status_get",
                      "rtcdf_plan", "rtcdf_sort_static"):
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
