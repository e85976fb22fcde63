"""In-tree build of the CUDA libraries for sm_103a (GB300).

``build()`` compiles every translation unit of ``csrc/`` in parallel with nvcc
(``-gencode arch=compute_103a,code=sm_103a``, static CUDA runtime) and links
``_build/librtcdf.so``; it also builds ``gen/_build/librtcdf_gen.so`` (input
generator) and ``cub_baseline/_build/librtcdf_cub.so`` (the CUB comparison
used by the benchmark).  A
library is rebuilt only when a source or header is newer than it.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
              "--expt-relaxed-constexpr"]


def nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found (CUDA toolkit required to build librtcdf)")
    return cand


def _newest(paths) -> float:
    return max(os.path.getmtime(p) for p in paths)


def _compile(src: str, obj: str, extra=()) -> None:
    cmd = [nvcc(), *ARCH, *NVCC_FLAGS, *extra, "-c", src, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")


def _build_lib(srcs, headers, out_so: str, jobs: int, extra=()) -> str:
    deps = list(srcs) + list(headers)
    if os.path.exists(out_so) and os.path.getmtime(out_so) >= _newest(deps):
        return out_so
    bdir = os.path.join(os.path.dirname(out_so), "obj")
    os.makedirs(bdir, exist_ok=True)
    objs = [os.path.join(bdir, os.path.basename(s) + ".o") for s in srcs]
    with cf.ThreadPoolExecutor(max_workers=jobs) as ex:
        futs = [ex.submit(_compile, s, o, extra) for s, o in zip(srcs, objs)]
        for f in futs:
            f.result()
    tmp = out_so + f".tmp{os.getpid()}"
    cmd = [nvcc(), *ARCH, "-shared", "-cudart", "static", "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed for {out_so}:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, out_so)
    return out_so


def lib_path() -> str:
    return os.path.join(HERE, "_build", "librtcdf.so")


def build(jobs: int | None = None) -> dict:
    """Build librtcdf.so and librtcdf_gen.so; returns their paths."""
    jobs = jobs or max(1, min(8, os.cpu_count() or 1))
    csrc = os.path.join(HERE, "csrc")
    srcs = sorted(glob.glob(os.path.join(csrc, "*.cu")) + glob.glob(os.path.join(csrc, "*.cpp")))
    headers = glob.glob(os.path.join(csrc, "*.h")) + glob.glob(os.path.join(csrc, "*.cuh")) + \
        glob.glob(os.path.join(csrc, "*.inc")) + \
        glob.glob(os.path.join(ROOT, "include", "*.h"))
    out = {"rtcdf": _build_lib(srcs, headers, lib_path(), jobs)}
    gsrc = [os.path.join(HERE, "gen", "gen.cu")]
    out["gen"] = _build_lib(gsrc, [os.path.join(ROOT, "include", "rtcdf_gen.h")],
                            os.path.join(HERE, "gen", "_build", "librtcdf_gen.so"), jobs)
    csrc_cub = [os.path.join(HERE, "cub_baseline", "cub_sort.cu")]
    out["cub"] = _build_lib(csrc_cub, [], os.path.join(HERE, "cub_baseline", "_build",
                                                     "librtcdf_cub.so"), jobs)
    return out


if __name__ == "__main__":
    print(build())
