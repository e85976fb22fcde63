"""Pins for the CPU oracle (no GPU).

The oracle is checked against things other than itself: the paper's worked
examples (golden fixtures), exhaustive brute force on tiny inputs against
Python's ``sorted``, numpy's sort on random inputs, the Lemmas of Section 3.2
computed with independent numpy routines, special cases, and planted mistakes
that must be caught.
"""
import itertools
import json
import os
import subprocess
import sys
import tempfile

import numpy as np
import pytest

import oracle
from paper_2609_00843_gb300 import gen

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

SORTS = {
    "counting": oracle.counting_sort,
    "kolonias": oracle.kolonias_sort,
    "hp": oracle.hp_sort,
    "refhp": oracle.refhp_sort,
}


def _rtcdf_B(T):
    return lambda a, lo, hi: oracle.rtcdf_sort(a, lo, hi, T)["B"]


def test_rtcdf_worked_example_matches_paper_table():
    g = json.load(open(os.path.join(GOLDEN, "rtcdf_tiled_example.json")))
    a = np.array(g["A"], dtype=np.int32)
    r = oracle.rtcdf_sort(a, g["minVal"], g["minVal"] + g["R"], g["T"])
    assert r["m"] == 2
    assert r["tile_hist"].tolist() == sum(g["tile_hist"], [])
    assert r["local_cdf"].tolist() == sum(g["local_cdf"], [])
    assert r["O"].tolist() == g["O"]
    assert r["B"].tolist() == g["B"]
    for f in SORTS.values():
        assert f(a, g["minVal"], g["minVal"] + g["R"]).tolist() == g["B"]


def test_hp_sort_worked_example_matches_paper():
    g = json.load(open(os.path.join(GOLDEN, "hp_sort_example.json")))
    counts = g["counts"]
    a = np.array(sum(([v] * c for v, c in enumerate(counts)), []), dtype=np.int32)
    a = a[::-1].copy()  # any order of the same multiset
    assert np.cumsum(counts).tolist() == g["P1"]
    assert oracle.cdf(a, 0, len(counts)).tolist() == g["P1"]
    for f in SORTS.values():
        assert f(a, 0, len(counts)).tolist() == g["B"]


@pytest.mark.parametrize("minVal", [0, -2, 7])
def test_exhaustive_brute_force_tiny(minVal):
    """Every array of length <= 6 over every range size R <= 4 against sorted()."""
    lib = oracle.load()
    for R in range(1, 5):
        for L in range(0, 7):
            for tup in itertools.product(range(minVal, minVal + R), repeat=L):
                a = np.array(tup, dtype=np.int32)
                want = sorted(tup)
                for name, f in SORTS.items():
                    assert f(a, minVal, minVal + R, lib).tolist() == want, (name, tup, R)
                for T in (1, 2, 3, 4):
                    got = oracle.rtcdf_sort(a, minVal, minVal + R, T, lib)["B"]
                    assert got.tolist() == want, ("rtcdf", T, tup, R)


@pytest.mark.parametrize("seed", range(6))
def test_random_against_numpy_sort(seed):
    rng = np.random.default_rng(seed)
    for _ in range(8):
        R = int(rng.choice([1, 2, 3, 31, 127, 128, 129, 1000, 4096, 5000, 70000]))
        minVal = int(rng.integers(-(1 << 31), (1 << 31) - R))
        n = int(rng.integers(0, 20000))
        a = (rng.integers(0, R, size=n) + minVal).astype(np.int32)
        want = np.sort(a)
        for name, f in SORTS.items():
            np.testing.assert_array_equal(f(a, minVal, minVal + R), want, err_msg=name)
        for T in {1, 7, 128, R, max(1, R // 3)}:
            np.testing.assert_array_equal(oracle.rtcdf_sort(a, minVal, minVal + R, T)["B"], want)


def test_int32_extremes():
    lo, hi = -(1 << 31), (1 << 31)
    a = np.array([hi - 1, lo, 0, hi - 1, lo, -1, 1], dtype=np.int32)
    # Whole int32 key space is too large for an R-sized histogram here; use the
    # two ends of it separately.
    a_lo = np.array([lo + 3, lo, lo + 1, lo], dtype=np.int32)
    assert oracle.counting_sort(a_lo, lo, lo + 4).tolist() == sorted(a_lo.tolist())
    a_hi = np.array([hi - 1, hi - 3, hi - 1, hi - 2], dtype=np.int32)
    assert oracle.counting_sort(a_hi, hi - 4, hi).tolist() == sorted(a_hi.tolist())
    with pytest.raises(oracle.OracleError) as e:
        oracle.counting_sort(a, -8, 8)
    assert e.value.code == oracle.ERR_KEY_OUT_OF_RANGE


@pytest.mark.parametrize("T", [1, 5, 64, 1000])
def test_lemmas_on_intermediates(T):
    """Lemma 1 (local CDF), Lemma 2 (tile offsets), sum of tile totals = n."""
    rng = np.random.default_rng(T)
    R, minVal, n = 777, -50, 30000
    a = (rng.integers(0, R, size=n) + minVal).astype(np.int32)
    a[: n // 4] = minVal + 400  # a heavy value
    r = oracle.rtcdf_sort(a, minVal, minVal + R, T)
    c = np.bincount(a.astype(np.int64) - minVal, minlength=R)
    m = -(-R // T)
    assert r["m"] == m
    np.testing.assert_array_equal(r["tile_hist"], c)
    totals = []
    for t in range(m):
        b, w = t * T, min(T, R - t * T)
        np.testing.assert_array_equal(r["local_cdf"][b:b + w], np.cumsum(c[b:b + w]))
        assert r["O"][t] == c[:b].sum()
        totals.append(r["local_cdf"][b + w - 1])
    assert sum(int(x) for x in totals) == n
    np.testing.assert_array_equal(r["B"], np.sort(a))


def test_value_intervals_lemma3():
    """Value v occupies exactly [CDF(v-1), CDF(v)) in the output."""
    rng = np.random.default_rng(3)
    R, minVal = 300, 10
    a = (rng.integers(0, R, size=5000) ** 2 // R + minVal).astype(np.int32)
    b = oracle.counting_sort(a, minVal, minVal + R)
    c = np.bincount(a - minVal, minlength=R)
    cum = np.concatenate([[0], np.cumsum(c)])
    for v in range(R):
        seg = b[cum[v]:cum[v + 1]]
        assert (seg == v + minVal).all()
    assert (np.diff(b) >= 0).all()


def test_special_cases():
    # n = 0 and n = 1
    for f in SORTS.values():
        assert f(np.empty(0, np.int32), 0, 5).size == 0
        assert f(np.array([4], np.int32), 0, 5).tolist() == [4]
    # R = 1: everything equals minVal
    a = np.full(17, -9, np.int32)
    for f in SORTS.values():
        assert f(a, -9, -8).tolist() == a.tolist()
    # all-equal input: output equals input
    a = np.full(1000, 42, np.int32)
    for f in SORTS.values():
        np.testing.assert_array_equal(f(a, 0, 128), a)
    # already sorted and reverse sorted
    s = np.repeat(np.arange(50, dtype=np.int32), 3)
    for f in SORTS.values():
        np.testing.assert_array_equal(f(s, 0, 50), s)
        np.testing.assert_array_equal(f(s[::-1].copy(), 0, 50), s)
    # range errors
    with pytest.raises(oracle.OracleError) as e:
        oracle.counting_sort(a, 5, 5)
    assert e.value.code == oracle.ERR_RANGE
    with pytest.raises(oracle.OracleError) as e:
        oracle.counting_sort(np.array([128], np.int32), 0, 128)
    assert e.value.code == oracle.ERR_KEY_OUT_OF_RANGE
    with pytest.raises(oracle.OracleError) as e:
        oracle.counting_sort(np.array([-1], np.int32), 0, 128)
    assert e.value.code == oracle.ERR_KEY_OUT_OF_RANGE


def test_check_sorted_accepts_truth_and_rejects_corruptions():
    rng = np.random.default_rng(11)
    a = rng.integers(-20, 20, size=4000).astype(np.int32)
    b = np.sort(a)
    assert oracle.check_sorted(a, b, -20, 20) == (True, None)
    bad = b.copy(); bad[1234] += 1
    ok, pos = oracle.check_sorted(a, bad, -20, 20)
    assert not ok and pos is not None and pos <= 1234
    bad = b.copy(); i = int(np.argmax(np.diff(b) > 0)); bad[i], bad[i + 1] = bad[i + 1], bad[i]
    assert not oracle.check_sorted(a, bad, -20, 20)[0]
    bad = np.roll(b, 1)
    assert not oracle.check_sorted(a, bad, -20, 20)[0]
    assert not oracle.check_sorted(a, b[:-1], -20, 20)[0]


def test_values_at_matches_full_sort():
    rng = np.random.default_rng(5)
    for R in (1, 2, 100, 4097):
        a = (rng.integers(0, R, size=10007) - 3).astype(np.int32)
        full = oracle.counting_sort(a, -3, R - 3)
        cdf = oracle.cdf(a, -3, R - 3)
        pos = rng.integers(0, a.size, size=500)
        pos = np.concatenate([pos, [0, a.size - 1]])
        np.testing.assert_array_equal(oracle.values_at(cdf, -3, pos), full[pos])


def test_oracle_on_generated_workload_shapes():
    """The three input shapes from the generator sort correctly; the oracle and
    numpy agree on them (this also exercises the generator's range)."""
    for dist in (gen.UNIFORM, gen.NORMAL, gen.ALL_EQUAL):
        for R in (1, 3, 128, 1 << 14):
            a = gen.keys_host(50000, -1000, R, dist, gen.derive_seed(1, dist, R))
            assert a.min() >= -1000 and a.max() < -1000 + R
            np.testing.assert_array_equal(oracle.counting_sort(a, -1000, -1000 + R), np.sort(a))


# ---------------------------------------------------------------------------
# Planted mistakes: a plausible slip anywhere in the oracle must fail a pin.
# Each mutant is a copy of oracle.c with one substitution, compiled to a
# temporary library and run in a subprocess (a mutant may write out of bounds).
# ---------------------------------------------------------------------------
MUTANTS = [
    ("histogram bound", "if (x < 0 || x >= R) return OR_ERR_KEY_OUT_OF_RANGE;\n        cnt[x] += 1;",
     "if (x < 0 || x > R) return OR_ERR_KEY_OUT_OF_RANGE;\n        cnt[x] += 1;"),
    ("counting value", "B[p++] = (int32_t)(minVal + v);", "B[p++] = (int32_t)(minVal + v + (v > 0));"),
    ("counting range", "for (int64_t v = 0; v < R; v++) {\n        for (uint64_t c",
     "for (int64_t v = 1; v < R; v++) {\n        for (uint64_t c"),
    ("kolonias prefix", "P[v + 1] = P[v] + H[v];", "P[v + 1] = P[v] + H[v + 1 < R ? v + 1 : v];"),
    ("hp index", "acc += H2[i];", "acc += H2[i + 1];"),
    ("refhp scatter", "Bn[P1[d - 1]] = d;", "Bn[P1[d - 1]] = d - 1;"),
    ("refhp max", "if (Bn[i] > run) run = Bn[i];", "run = Bn[i];"),
    ("rtcdf tile test", "if (0 <= x && x < w) S[x] += 1;", "if (0 < x && x < w) S[x] += 1;"),
    ("rtcdf scan", "for (int64_t x = 1; x < w; x++) H[b + x] += H[b + x - 1];",
     "for (int64_t x = 2; x < w; x++) H[b + x] += H[b + x - 1];"),
    ("rtcdf offset", "offset += H[b + w - 1];", "offset += H[b + w - 1 - (w > 1)];"),
    ("rtcdf search", "while (C[j] < p + 1) j++;", "while (C[j] < p) j++;"),
    ("rtcdf value", "B[tileStart + p] = (int32_t)(minVal + b + j);", "B[tileStart + p] = (int32_t)(minVal + j);"),
    ("check compare", "if (v >= R || got != v)", "if (v >= R || got > v)"),
]

_PIN_SCRIPT = r"""
import sys, json, numpy as np
sys.path.insert(0, {root!r})
import oracle
lib = oracle.load({path!r})
g = json.load(open({golden!r}))
a = np.array(g["A"], dtype=np.int32)
fails = []
def chk(name, got, want):
    if list(map(int, got)) != list(map(int, want)):
        fails.append(name)
for f in ("counting_sort", "kolonias_sort", "hp_sort", "refhp_sort"):
    chk(f, getattr(oracle, f)(a, 0, 4, lib), g["B"])
r = oracle.rtcdf_sort(a, 0, 4, 2, lib)
chk("rtcdf_B", r["B"], g["B"]); chk("rtcdf_O", r["O"], g["O"])
chk("rtcdf_lc", r["local_cdf"], sum(g["local_cdf"], []))
rng = np.random.default_rng(1)
for R, T in ((5, 2), (128, 128), (1000, 7)):
    x = rng.integers(0, R, size=3000).astype(np.int32)
    want = np.sort(x)
    for f in ("counting_sort", "kolonias_sort", "hp_sort", "refhp_sort"):
        chk(f + str(R), getattr(oracle, f)(x, 0, R, lib), want)
    chk("rtcdf" + str(R), oracle.rtcdf_sort(x, 0, R, T, lib)["B"], want)
    i = int(np.searchsorted(want, want[-1]))  # first position of the largest value
    for pos, delta in ((0, 1), (i, -1)):
        bad = want.copy(); bad[pos] += delta
        if delta < 0 and i == 0:
            continue
        ok, _ = oracle.check_sorted(x, bad, 0, R, lib)
        if ok: fails.append("checker")
try:
    oracle.counting_sort(np.array([4], np.int32), 0, 4, lib); fails.append("range")
except oracle.OracleError:
    pass
print("FAILS", len(fails))
"""


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_is_caught(name, old, new, tmp_path):
    src = open(os.path.join(os.path.dirname(oracle.__file__), "oracle.c")).read()
    assert src.count(old) == 1, f"mutation anchor not unique for {name}"
    mut = tmp_path / "oracle_mut.c"
    mut.write_text(src.replace(old, new))
    so = tmp_path / "liboracle_mut.so"
    oracle.build(force=True, src=str(mut), out=str(so))
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    script = _PIN_SCRIPT.format(root=root, path=str(so),
                                golden=os.path.join(GOLDEN, "rtcdf_tiled_example.json"))
    p = subprocess.run([sys.executable, "-c", script], capture_output=True, text=True, timeout=120)
    caught = p.returncode != 0 or "FAILS 0" not in p.stdout
    assert caught, f"mutant '{name}' passed every pin: {p.stdout} {p.stderr}"


def test_unmutated_oracle_passes_the_mutation_pins(tmp_path):
    src = os.path.join(os.path.dirname(oracle.__file__), "oracle.c")
    so = tmp_path / "liboracle_copy.so"
    oracle.build(force=True, src=src, out=str(so))
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    script = _PIN_SCRIPT.format(root=root, path=str(so),
                                golden=os.path.join(GOLDEN, "rtcdf_tiled_example.json"))
    p = subprocess.run([sys.executable, "-c", script], capture_output=True, text=True, timeout=120)
    assert p.returncode == 0 and "FAILS 0" in p.stdout, p.stdout + p.stderr
