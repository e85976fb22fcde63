"""The segmented-sort planner, on the host: a small C++ program links the
library, builds plans for random segment shapes under every schedule and
checks the invariants the three launches rely on (kinds in the right launch,
scan chunks of a segment in ascending ticket order, exact coverage of keys
and positions, disjoint workspace regions, output items by non-increasing
estimated cost)."""
import os
import shutil
import subprocess

import pytest

from paper_2609_00843_gb300 import _build

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    _build.build()
    cxx = shutil.which("g++")
    if not cxx:
        pytest.skip("no C++ compiler")
    cuda_inc = os.path.join(os.path.dirname(os.path.dirname(_build.nvcc())), "include")
    lib_dir = os.path.dirname(_build.lib_path())
    exe = str(tmp_path_factory.mktemp("planner") / "planner_check")
    cmd = [cxx, "-std=c++17", "-O1", os.path.join(HERE, "planner_check.cpp"),
           "-I", os.path.join(ROOT, "paper_2609_00843_gb300", "csrc"), "-I", cuda_inc,
           "-L", lib_dir, "-lrtcdf", f"-Wl,-rpath,{lib_dir}", "-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-3000:]
    return exe


@pytest.mark.parametrize("seed,segments", [(1, 300), (2, 1200), (3, 40), (4, 1)])
def test_planner_invariants(checker, seed, segments):
    r = subprocess.run([checker, str(seed), str(segments)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == "OK", r.stdout + r.stderr
