"""Tuning table and the tuner's selection rule, without a GPU: the table API
of the C library (set / get / reset / size classes, argument checks) and the
host-side pieces of the tune module (candidate sets, the geometric-mean rule
of Section 4.1, the table file format)."""
import math
import os
import re

import pytest

from paper_2609_00843_gb300 import _build, rtcdf, tune

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
INC = os.path.join(ROOT, "paper_2609_00843_gb300", "csrc", "tune_table.inc")


@pytest.fixture(scope="module", autouse=True)
def built():
    _build.build()
    yield
    rtcdf.rtcdf_tune_reset()


def _inc_entries():
    text = open(INC).read()
    return re.findall(r"^\{(-?\d+), (-?\d+), \{(-?\d+), 0, (-?\d+), 0, (-?\d+), (-?\d+), \{0, 0\}\}\},$",
                      text, re.M)


def test_n_class_boundaries():
    f = rtcdf.rtcdf_tune_n_class
    assert [f(0), f(1), f((1 << 20) - 1)] == [0, 0, 0]
    assert [f(1 << 20), f((1 << 26) - 1)] == [1, 1]
    assert [f(1 << 26), f(100_000_000), f((1 << 32) - 1)] == [2, 2, 2]


def test_set_get_reset_roundtrip():
    builtin = rtcdf.rtcdf_tune_get()
    assert len(builtin) == len(_inc_entries())
    e = [(14, 0, rtcdf.Params(tile_width=4096, hist_threads=512)),
         (18, 2, rtcdf.Params(fill_threads=256, fill_chunk=65536))]
    rtcdf.rtcdf_tune_set(e)
    got = rtcdf.rtcdf_tune_get()
    assert [(a, b, p.tile_width, p.hist_threads, p.fill_threads, p.fill_chunk) for a, b, p in got] == \
        [(14, 0, 4096, 512, 0, 0), (18, 2, 0, 0, 256, 65536)]
    rtcdf.rtcdf_tune_set([])
    assert rtcdf.rtcdf_tune_get() == []
    rtcdf.rtcdf_tune_reset()
    assert len(rtcdf.rtcdf_tune_get()) == len(builtin)


@pytest.mark.parametrize("entry", [
    (25, 0, rtcdf.Params()),                     # range class beyond 2^24
    (-1, 0, rtcdf.Params()),
    (10, 3, rtcdf.Params()),                     # no such size class
    (10, 0, rtcdf.Params(hist_threads=384)),     # threads not 256/512/1024
    (10, 0, rtcdf.Params(fill_threads=128)),
    (10, 0, rtcdf.Params(tile_width=-5)),
    (10, 0, rtcdf.Params(fill_ctas=-1)),
])
def test_set_rejects_bad_entries_and_keeps_table(entry):
    rtcdf.rtcdf_tune_set([(7, 1, rtcdf.Params(hist_threads=512))])
    with pytest.raises(rtcdf.RtcdfError):
        rtcdf.rtcdf_tune_set([entry])
    assert len(rtcdf.rtcdf_tune_get()) == 1
    rtcdf.rtcdf_tune_reset()


def test_geomean_rule_matches_hand_computation():
    # two conditions, three candidates; candidate 2 cannot run condition 1
    t = [[1.0, 2.0, 4.0], [3.0, 1.5, -1.0]]
    gm = tune._geomean(t)
    assert gm[0] == pytest.approx(math.sqrt(1.0 * 2.0))
    assert gm[1] == pytest.approx(math.sqrt(2.0 * 1.0))
    assert gm[2] == float("inf")
    # r(T) >= 1 with equality for the fastest: a candidate fastest everywhere has gm 1
    assert tune._geomean([[1.0, 2.0], [1.0, 3.0]])[0] == 1.0


def test_pick_keeps_builtin_rule_within_margin():
    assert tune._pick([1.005, 1.0, 1.2], 0.01) == 0
    assert tune._pick([1.05, 1.0, 1.2], 0.01) == 1
    assert tune._pick([1.0, 1.0], 0.01) == 0


def test_hist_candidates_cover_tile_counts():
    ws = lambda R: sorted({p.tile_width for p in tune.hist_candidates(R, 57344)})
    assert ws(128) == [0, 128]
    assert ws(1 << 14) == [0, 6144, 8192, 16384]
    # R = 2^18 > t_max: m = 5, 6, 7 balanced tiles and the full t_max
    w = ws(1 << 18)
    assert 57344 in w and 53248 in w and all(-(-(1 << 18) // T) in (5, 6, 7) for T in w if T)
    for p in tune.hist_candidates(1 << 18, 57344):
        assert p.hist_threads in (0, 512, 1024) and p.tile_width <= 57344


def test_fill_candidates_keep_stage_one_choice():
    base = rtcdf.Params(tile_width=8192, hist_threads=512)
    c = tune.fill_candidates(base)
    assert c[0].fill_threads == 0 and c[0].fill_chunk == 0
    assert all(p.tile_width == 8192 and p.hist_threads == 512 for p in c)
    assert len({(p.fill_threads, p.fill_chunk) for p in c}) == len(c)


def test_write_inc_format_is_what_the_library_parses(tmp_path):
    path = str(tmp_path / "t.inc")
    tune.write_inc([{"log2_R": 18, "n_class": 2, "tile_width": 53248, "hist_threads": 1024,
                     "fill_threads": 256, "fill_chunk": 65536}], path)
    text = open(path).read()
    assert "{18, 2, {53248, 0, 1024, 0, 256, 65536, {0, 0}}}," in text
    for line in text.splitlines():
        assert line.startswith("//") or line.startswith("{")
