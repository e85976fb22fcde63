"""Seeded synthetic inputs for RT-CDF: host (numpy) and device (CUDA) generators.

This module holds none of the sort's arithmetic.  It is the one piece shared by
the CPU oracle's tests and the CUDA path's tests and benchmarks: both sides are
fed keys produced here, so a host-generated array and a device-generated array
with the same (seed, index range) are bit-identical.

Counter-based stream
--------------------
SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014): the k-th output of a stream seeded with ``s`` is
``mix64(s + (k + 1) * 0x9E3779B97F4A7C15)`` with the published finaliser
``mix64``.  Element ``i`` of an array uses the outputs ``k = 16 i + j``.

Distributions (the three input shapes of the paper's evaluation, Section 4)
-----------------------------------------------------------------------------
* ``UNIFORM``   key = minVal + floor(u32 * R / 2^32), u32 the high half of
  output ``16 i`` (multiply-shift range reduction).
* ``NORMAL``    mean minVal + R/2, standard deviation R/8, rounded half away
  from zero and clipped to [minVal, minVal + R - 1].  The normal variate is the
  Irwin-Hall sum of twelve 32-bit uniforms (both halves of outputs
  ``16 i .. 16 i + 5``) minus 6, which has mean 0 and variance 1.  The offset
  R/2 + (R/8) z is computed in IEEE-754 single precision, one correctly
  rounded operation at a time (exact integers up to 2^24), so that host and
  device agree exactly; minVal is added in integer arithmetic.
* ``ALL_EQUAL`` key = minVal + floor(R / 3).
"""
from __future__ import annotations

import ctypes
import math
import os

import numpy as np

UNIFORM = 0
NORMAL = 1
ALL_EQUAL = 2
DIST_NAMES = {"uniform": UNIFORM, "normal": NORMAL, "all_equal": ALL_EQUAL}

GOLDEN = 0x9E3779B97F4A7C15
_M1 = 0xBF58476D1CE4E5B9
_M2 = 0x94D049BB133111EB
_MASK = (1 << 64) - 1

_HERE = os.path.dirname(os.path.abspath(__file__))


def mix64_int(z: int) -> int:
    """SplitMix64 finaliser on a Python int (mod 2^64)."""
    z &= _MASK
    z = ((z ^ (z >> 30)) * _M1) & _MASK
    z = ((z ^ (z >> 27)) * _M2) & _MASK
    return z ^ (z >> 31)


def derive_seed(*parts: int) -> int:
    """Fold integers (config id, distribution, log2 R, segment id, ...) into a seed."""
    s = 0x243F6A8885A308D3
    for p in parts:
        s = mix64_int(s ^ (int(p) & _MASK)) + GOLDEN
        s &= _MASK
    return s


def _mix64(z: np.ndarray) -> np.ndarray:
    z = z ^ (z >> np.uint64(30))
    z = z * np.uint64(_M1)
    z = z ^ (z >> np.uint64(27))
    z = z * np.uint64(_M2)
    return z ^ (z >> np.uint64(31))


def words(seed: int, ctr: np.ndarray) -> np.ndarray:
    """SplitMix64 outputs number ``ctr`` (uint64 array) of the stream ``seed``."""
    with np.errstate(over="ignore"):
        z = np.uint64(seed & _MASK) + (ctr + np.uint64(1)) * np.uint64(GOLDEN)
        return _mix64(z)


def _check(minVal: int, R: int):
    if R <= 0 or R > (1 << 32):
        raise ValueError(f"range size R={R} outside [1, 2^32]")
    if minVal < -(1 << 31) or minVal + R > (1 << 31):
        raise ValueError("range [minVal, minVal + R) must lie in the int32 key space")


def keys_host(n: int, minVal: int, R: int, dist: int, seed: int, first: int = 0,
              chunk: int = 1 << 22) -> np.ndarray:
    """Keys ``first .. first + n - 1`` of the stream, as an int32 numpy array."""
    minVal = int(minVal)
    R = int(R)
    _check(minVal, R)
    out = np.empty(int(n), dtype=np.int32)
    if dist == ALL_EQUAL:
        out[:] = minVal + R // 3
        return out
    for s in range(0, int(n), chunk):
        e = min(int(n), s + chunk)
        idx = np.arange(first + s, first + e, dtype=np.uint64)
        base = idx * np.uint64(16)
        if dist == UNIFORM:
            u = words(seed, base) >> np.uint64(32)
            x = (u * np.uint64(R)) >> np.uint64(32)
            out[s:e] = (x.astype(np.int64) + minVal).astype(np.int32)
        elif dist == NORMAL:
            S = np.zeros(e - s, dtype=np.uint64)
            for j in range(6):
                wj = words(seed, base + np.uint64(j))
                S += (wj >> np.uint64(32)) + (wj & np.uint64(0xFFFFFFFF))
            f32 = np.float32
            z = S.astype(f32) * f32(2.0 ** -32) - f32(6.0)
            half = f32(R) / f32(2.0)
            sigma = f32(R) / f32(8.0)
            o = half + sigma * z
            r = np.where(o >= f32(0), np.floor(o + f32(0.5)), -np.floor(-o + f32(0.5)))
            r = np.clip(r.astype(np.int64), 0, R - 1)
            out[s:e] = (r + minVal).astype(np.int32)
        else:
            raise ValueError(f"unknown distribution {dist}")
    return out


# ---------------------------------------------------------------------------
# Device generator (librtcdf_gen.so, built from gen.cu)
# ---------------------------------------------------------------------------
_gen_lib = None


def lib_path() -> str:
    return os.path.join(_HERE, "_build", "librtcdf_gen.so")


def load_device_lib():
    """Load the device generator library; raises if it has not been built."""
    global _gen_lib
    if _gen_lib is None:
        path = lib_path()
        if not os.path.exists(path):
            raise RuntimeError(f"device generator library missing: {path} (run build())")
        lib = ctypes.CDLL(path)
        lib.rtcdf_gen_keys.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint64,
                                       ctypes.c_int64, ctypes.c_int64, ctypes.c_int,
                                       ctypes.c_uint64, ctypes.c_void_p]
        lib.rtcdf_gen_keys.restype = ctypes.c_int
        _gen_lib = lib
    return _gen_lib


def keys_device(out_ptr: int, n: int, minVal: int, R: int, dist: int, seed: int,
                first: int = 0, stream: int = 0) -> None:
    """Write keys ``first .. first + n - 1`` into device memory at ``out_ptr``."""
    _check(int(minVal), int(R))
    rc = load_device_lib().rtcdf_gen_keys(ctypes.c_void_p(out_ptr), int(n), int(first),
                                          int(minVal), int(R), int(dist),
                                          ctypes.c_uint64(seed & _MASK),
                                          ctypes.c_void_p(stream))
    if rc != 0:
        raise RuntimeError(f"rtcdf_gen_keys failed with code {rc}")


# ---------------------------------------------------------------------------
# Workload shapes (segment / request metadata), host only
# ---------------------------------------------------------------------------
def _unit(seed: int, ctr: np.ndarray) -> np.ndarray:
    """Doubles in [0, 1) from the top 53 bits of the stream."""
    return (words(seed, ctr) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def log_uniform_ints(seed: int, count: int, lo: float, hi: float, slot: int = 0) -> np.ndarray:
    """floor(exp(U(ln lo, ln hi))) for ``count`` items, as int64."""
    u = _unit(seed, np.arange(count, dtype=np.uint64) * np.uint64(16) + np.uint64(slot))
    v = np.floor(np.exp(math.log(lo) + u * (math.log(hi) - math.log(lo))))
    return np.clip(v, lo, hi).astype(np.int64)


def uniform_ints(seed: int, count: int, lo: int, hi: int, slot: int = 0) -> np.ndarray:
    """Integers uniform on [lo, hi] (inclusive), as int64."""
    w = words(seed, np.arange(count, dtype=np.uint64) * np.uint64(16) + np.uint64(slot))
    span = np.uint64(hi - lo + 1)
    return ((w >> np.uint64(32)) * span >> np.uint64(32)).astype(np.int64) + lo


def batched_segments(seed: int, num_segments: int = 4096, n_lo: float = 1e3,
                     n_hi: float = 1e6, r_lo: float = 2 ** 7, r_hi: float = 2 ** 16,
                     min_lo: int = -(1 << 20), min_hi: int = 1 << 20):
    """Segment shapes of the batched workload: lengths log-uniform in
    [n_lo, n_hi], range sizes log-uniform in [r_lo, r_hi], minVal uniform in
    [min_lo, min_hi], distribution uniform over the three shapes.

    Returns (lengths, minVal, R, dist, per-segment seeds) as int64 / uint64 arrays.
    """
    lengths = log_uniform_ints(seed, num_segments, n_lo, n_hi, slot=0)
    R = log_uniform_ints(seed, num_segments, r_lo, r_hi, slot=1)
    minv = uniform_ints(seed, num_segments, min_lo, min_hi, slot=2)
    dist = uniform_ints(seed, num_segments, 0, 2, slot=3)
    seeds = np.array([derive_seed(seed, 7, i) for i in range(num_segments)], dtype=np.uint64)
    return lengths, minv, R, dist, seeds


def serving_requests(seed: int, count: int = 20000, n_lo: float = 1e4, n_hi: float = 1e8,
                     r_lo: float = 2 ** 7, r_hi: float = 2 ** 18):
    """Request shapes of the serving workload: n log-uniform in [n_lo, n_hi],
    R log-uniform in [r_lo, r_hi], minVal uniform in [-2^20, 2^20], shape
    uniform over the three.  Returns (n, minVal, R, dist, seeds)."""
    n = log_uniform_ints(seed, count, n_lo, n_hi, slot=0)
    R = log_uniform_ints(seed, count, r_lo, r_hi, slot=1)
    minv = uniform_ints(seed, count, -(1 << 20), 1 << 20, slot=2)
    dist = uniform_ints(seed, count, 0, 2, slot=3)
    seeds = np.array([derive_seed(seed, 9, i) for i in range(count)], dtype=np.uint64)
    return n, minv, R, dist, seeds


def poisson_arrivals(seed: int, count: int, rate_per_s: float) -> np.ndarray:
    """Arrival times (seconds) of a Poisson process: cumulative exponential gaps."""
    u = _unit(seed, np.arange(count, dtype=np.uint64) * np.uint64(16) + np.uint64(5))
    gaps = -np.log1p(-u) / rate_per_s
    return np.cumsum(gaps)


def fill_function_address() -> int:
    """Address of rtcdf_gen_keys, usable as a server's fill callback."""
    return ctypes.cast(load_device_lib().rtcdf_gen_keys, ctypes.c_void_p).value


def digest(sorted_keys: np.ndarray) -> int:
    """Order-dependent digest of an array, as the server computes it on the
    device: sum over positions i of mix64((i << 32) | uint32(key_i)), mod 2^64."""
    a = np.ascontiguousarray(sorted_keys).view(np.uint32).astype(np.uint64)
    i = np.arange(a.size, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return int(_mix64((i << np.uint64(32)) | a).sum(dtype=np.uint64))
