"""Host generator checks (no GPU): determinism, range and the shapes of the
three input distributions of the paper's evaluation."""
import numpy as np

from paper_2609_00843_gb300 import gen


def test_splitmix64_stream_definition():
    # First outputs of SplitMix64 seeded with 0 (the stream state advances by
    # the golden gamma before each mix).  Computed with the integer definition.
    def ref(seed, k):
        return gen.mix64_int(seed + (k + 1) * gen.GOLDEN)
    got = gen.words(0, np.arange(4, dtype=np.uint64))
    assert [int(x) for x in got] == [ref(0, k) for k in range(4)]
    # Published first output of SplitMix64 from state 0.
    assert int(got[0]) == 0xE220A8397B1DCDAF


def test_deterministic_and_sliceable():
    a = gen.keys_host(10000, -5, 1000, gen.NORMAL, 123)
    b = gen.keys_host(10000, -5, 1000, gen.NORMAL, 123)
    np.testing.assert_array_equal(a, b)
    c = gen.keys_host(3000, -5, 1000, gen.NORMAL, 123, first=7000)
    np.testing.assert_array_equal(a[7000:], c)
    d = gen.keys_host(10000, -5, 1000, gen.NORMAL, 124)
    assert (a != d).any()


def test_uniform_shape():
    R = 1 << 10
    a = gen.keys_host(1 << 20, -1000, R, gen.UNIFORM, 9)
    assert a.min() == -1000 and a.max() == -1000 + R - 1
    c = np.bincount(a + 1000, minlength=R)
    exp = a.size / R
    chi2 = ((c - exp) ** 2 / exp).sum()
    assert chi2 < R + 6 * np.sqrt(2 * R)


def test_normal_shape():
    R = 1 << 14
    a = gen.keys_host(1 << 20, -1000, R, gen.NORMAL, 10).astype(np.float64)
    mu, sd = -1000 + R / 2, R / 8
    assert abs(a.mean() - mu) < 0.01 * sd
    assert abs(a.std() - sd) < 0.01 * sd
    # about 68.3% within one standard deviation
    frac = np.mean(np.abs(a - mu) <= sd)
    assert 0.67 < frac < 0.695
    assert a.min() >= -1000 and a.max() <= -1000 + R - 1


def test_all_equal_and_small_ranges():
    a = gen.keys_host(100, 7, 128, gen.ALL_EQUAL, 0)
    assert (a == 7 + 128 // 3).all()
    for dist in (gen.UNIFORM, gen.NORMAL, gen.ALL_EQUAL):
        a = gen.keys_host(1000, 3, 1, dist, 1)
        assert (a == 3).all()
    top = gen.keys_host(1000, (1 << 31) - 4, 4, gen.UNIFORM, 2)
    assert top.min() >= (1 << 31) - 4


def test_batched_segment_shapes():
    L, mn, R, dist, seeds = gen.batched_segments(gen.derive_seed(4), 4096)
    assert L.min() >= 1000 and L.max() <= 1000000
    assert R.min() >= 128 and R.max() <= 1 << 16
    assert mn.min() >= -(1 << 20) and mn.max() <= 1 << 20
    assert set(np.unique(dist)) == {0, 1, 2}
    # log-uniform: the median length is near sqrt(1e3 * 1e6)
    assert 2.0e4 < np.median(L) < 5.0e4
    assert len(set(seeds.tolist())) == 4096
