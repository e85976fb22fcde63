"""CPU oracle for Range-Tiled CDF sort (RT-CDF).

TEST INFRASTRUCTURE, NOT PART OF THE PRODUCT.  Only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline / reference arm of
``bench.py`` may import this package.  The product path (the CUDA library and
its binding) never imports it and has no fallback to it.

The arithmetic lives in ``oracle.c`` (plain sequential C, integer only); this
module compiles it with gcc on first use and wraps it with ctypes and numpy.
Each function cites the part of the paper it follows:

* :func:`counting_sort` -- the plain definition of the output (Section 2.1).
* :func:`kolonias_sort` -- Algorithm 1 (interval fill per value).
* :func:`hp_sort`       -- Algorithm 2 (H-P sort).
* :func:`refhp_sort`    -- Algorithm 3 (CDF steps + inclusive prefix maximum).
* :func:`rtcdf_sort`    -- Algorithms 4-7 step by step, with intermediates.
* :func:`check_sorted`  -- Lemmas 1-3 / Theorem 1 as a checker of any output.
* :func:`cdf`, :func:`values_at` -- single output values from the CDF
  (position p holds min{v : CDF[v] >= p + 1}, Algorithm 7's rule applied to the
  whole range).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "liboracle.so")

OK = 0
ERR_INVALID_ARG = 1
ERR_RANGE = 2
ERR_KEY_OUT_OF_RANGE = 3
ERR_NO_MEMORY = 5


class OracleError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"oracle {what} failed with code {code}")
        self.code = code


_lock = threading.Lock()
_lib = None


def build(force: bool = False, src: str = _SRC, out: str = _LIB_PATH) -> str:
    """Compile ``oracle.c`` into a shared library (gcc, -O2, no vector ISA flags)."""
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(src):
        return out
    os.makedirs(os.path.dirname(out), exist_ok=True)
    tmp = out + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, src])
    os.replace(tmp, out)
    return out


def _declare(lib):
    i32p = ctypes.c_void_p
    u64 = ctypes.c_uint64
    i64 = ctypes.c_int64
    for name in ("oracle_counting_sort", "oracle_kolonias_sort", "oracle_hp_sort",
                 "oracle_refhp_sort"):
        f = getattr(lib, name)
        f.argtypes = [i32p, i32p, u64, i64, i64]
        f.restype = ctypes.c_int
    lib.oracle_histogram.argtypes = [i32p, u64, i64, i64, ctypes.c_void_p]
    lib.oracle_histogram.restype = ctypes.c_int
    lib.oracle_cdf.argtypes = [i32p, u64, i64, i64, ctypes.c_void_p]
    lib.oracle_cdf.restype = ctypes.c_int
    lib.oracle_rtcdf_sort.argtypes = [i32p, i32p, u64, i64, i64, i64, ctypes.c_void_p,
                                      ctypes.c_void_p, ctypes.c_void_p]
    lib.oracle_rtcdf_sort.restype = ctypes.c_int
    lib.oracle_check_sorted.argtypes = [i32p, i32p, u64, i64, i64,
                                        ctypes.POINTER(ctypes.c_uint64)]
    lib.oracle_check_sorted.restype = ctypes.c_int
    return lib


def load(path: str | None = None):
    """Load (building if needed) the oracle library.  ``path`` selects another
    build of the same source, e.g. a deliberately mutated copy in a test."""
    global _lib
    if path is not None:
        return _declare(ctypes.CDLL(path))
    with _lock:
        if _lib is None:
            _lib = _declare(ctypes.CDLL(build()))
    return _lib


def _keys(a) -> np.ndarray:
    a = np.ascontiguousarray(a)
    if a.dtype != np.int32:
        raise TypeError(f"keys must be int32, got {a.dtype}")
    return a


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _range(minVal: int, maxVal: int) -> int:
    R = int(maxVal) - int(minVal)
    if R <= 0:
        raise OracleError(ERR_RANGE, "range check")
    return R


def _sort_with(fname: str, a, minVal: int, maxVal: int, lib=None) -> np.ndarray:
    lib = lib or load()
    a = _keys(a)
    b = np.empty_like(a)
    rc = getattr(lib, fname)(_ptr(a), _ptr(b), a.size, int(minVal), int(maxVal))
    if rc != OK:
        raise OracleError(rc, fname)
    return b


def counting_sort(a, minVal: int, maxVal: int, lib=None) -> np.ndarray:
    """Plain counting sort: value v occupies [sum_{u<v} c_u, sum_{u<=v} c_u) (Section 2.1)."""
    return _sort_with("oracle_counting_sort", a, minVal, maxVal, lib)


def kolonias_sort(a, minVal: int, maxVal: int, lib=None) -> np.ndarray:
    """Algorithm 1: prefix sums P, every value v fills [P[v], P[v+1])."""
    return _sort_with("oracle_kolonias_sort", a, minVal, maxVal, lib)


def hp_sort(a, minVal: int, maxVal: int, lib=None) -> np.ndarray:
    """Algorithm 2: histogram of the CDF values, then its prefix sums."""
    return _sort_with("oracle_hp_sort", a, minVal, maxVal, lib)


def refhp_sort(a, minVal: int, maxVal: int, lib=None) -> np.ndarray:
    """Algorithm 3: scatter each value at its interval start, then prefix maximum."""
    return _sort_with("oracle_refhp_sort", a, minVal, maxVal, lib)


def histogram(a, minVal: int, maxVal: int, lib=None) -> np.ndarray:
    """c_v for every normalised value v in [0, R) (Section 2.1), as uint64."""
    lib = lib or load()
    a = _keys(a)
    cnt = np.empty(_range(minVal, maxVal), dtype=np.uint64)
    rc = lib.oracle_histogram(_ptr(a), a.size, int(minVal), int(maxVal), _ptr(cnt))
    if rc != OK:
        raise OracleError(rc, "oracle_histogram")
    return cnt


def cdf(a, minVal: int, maxVal: int, lib=None) -> np.ndarray:
    """Inclusive CDF[v] = sum_{u<=v} c_u, as uint64."""
    lib = lib or load()
    a = _keys(a)
    out = np.empty(_range(minVal, maxVal), dtype=np.uint64)
    rc = lib.oracle_cdf(_ptr(a), a.size, int(minVal), int(maxVal), _ptr(out))
    if rc != OK:
        raise OracleError(rc, "oracle_cdf")
    return out


def values_at(cdf_: np.ndarray, minVal: int, positions) -> np.ndarray:
    """Output values at the given positions: B[p] = minVal + min{v : CDF[v] >= p + 1}.

    The smallest such v is found by a library binary search
    (``numpy.searchsorted`` with side='right' returns the number of CDF
    entries <= p, i.e. the number of values whose interval ends at or before p).
    """
    pos = np.asarray(positions, dtype=np.uint64)
    v = np.searchsorted(cdf_, pos, side="right").astype(np.int64)
    return (v + int(minVal)).astype(np.int32)


def rtcdf_sort(a, minVal: int, maxVal: int, T: int, lib=None) -> dict:
    """Algorithms 4-7, sequential, returning every intermediate.

    Returns a dict with ``B`` (int32 output), ``tile_hist`` and ``local_cdf``
    (uint64[R], the array H after Algorithm 5 and after the per-tile scans),
    ``O`` (uint64[m], Algorithm 6) and ``m``.
    """
    lib = lib or load()
    a = _keys(a)
    R = _range(minVal, maxVal)
    T = int(T)
    if T <= 0:
        raise OracleError(ERR_INVALID_ARG, "tile width")
    m = (R + T - 1) // T
    b = np.empty_like(a)
    th = np.empty(R, dtype=np.uint64)
    lc = np.empty(R, dtype=np.uint64)
    O = np.empty(m, dtype=np.uint64)
    rc = lib.oracle_rtcdf_sort(_ptr(a), _ptr(b), a.size, int(minVal), int(maxVal), T,
                               _ptr(th), _ptr(lc), _ptr(O))
    if rc != OK:
        raise OracleError(rc, "oracle_rtcdf_sort")
    return {"B": b, "tile_hist": th, "local_cdf": lc, "O": O, "m": m}


def check_sorted(a, b, minVal: int, maxVal: int, lib=None):
    """Check Lemma 3 / Theorem 1 on a claimed output ``b`` of input ``a``.

    Returns ``(True, None)`` or ``(False, first_bad_position)``.
    """
    lib = lib or load()
    a = _keys(a)
    b = _keys(b)
    if a.size != b.size:
        return False, None
    bad = ctypes.c_uint64(0)
    rc = lib.oracle_check_sorted(_ptr(a), _ptr(b), a.size, int(minVal), int(maxVal),
                                 ctypes.byref(bad))
    if rc == OK:
        return True, None
    if rc == -1:
        return False, int(bad.value)
    raise OracleError(rc, "oracle_check_sorted")
