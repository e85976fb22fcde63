"""The tuner on the GPU: rtcdf_autotune measures every runnable candidate and
ranks by the geometric mean of normalised times; a tuning-table entry changes
the launch shape rtcdf_sort uses (and nothing else: results stay bit-exact);
entries that do not fit the device fall back to the built-in rules."""
import math

import pytest
import torch

from paper_2609_00843_gb300 import _build, gen, rtcdf

from gpu_util import assert_matches_oracle, dev_keys, gpu_sort, stream_handle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    _build.build()
    torch.cuda.init()
    yield
    rtcdf.rtcdf_tune_reset()


def test_autotune_measures_and_ranks():
    R = 1 << 14
    xs = [dev_keys(n, -7, R, d, gen.derive_seed(60, n, d)) for n in (50_000, 300_001) for d in (0, 1)]
    outs = [torch.empty_like(x) for x in xs]
    cases = [(x.data_ptr(), o.data_ptr(), x.numel(), -7, -7 + R) for x, o in zip(xs, outs)]
    cands = [rtcdf.Params(), rtcdf.Params(tile_width=4096), rtcdf.Params(tile_width=1 << 20),
             rtcdf.Params(fill_threads=256, fill_chunk=8192)]
    wsb = rtcdf.rtcdf_workspace_size(R)
    ws = torch.zeros(wsb // 4 + 64, dtype=torch.int32, device="cuda")
    t, gm, best = rtcdf.rtcdf_autotune(cases, cands, 3, ws.data_ptr(), wsb, stream_handle())
    for row in t:
        assert row[2] == -1.0                       # T beyond shared memory: cannot run
        assert all(v > 0 for j, v in enumerate(row) if j != 2)
    assert gm[2] == float("inf")
    finite = [g for g in gm if g != float("inf")]
    assert all(g >= 1.0 for g in finite) and best == gm.index(min(finite))
    # the geometric mean is the one of the returned times
    k = 0
    want = math.exp(sum(math.log(row[k] / min(v for v in row if v > 0)) for row in t) / len(t))
    assert gm[k] == pytest.approx(want, rel=1e-5)
    # the last candidate's sorts left correct outputs
    for x, o in zip(xs, outs):
        assert_matches_oracle(x, o, -7, -7 + R)


def test_table_entry_changes_the_launch_shape_not_the_result():
    R, n = 1 << 14, 200_003
    rtcdf.rtcdf_tune_set([])
    base = rtcdf.rtcdf_plan(n, R)
    assert base.tile_width == R
    try:
        rtcdf.rtcdf_tune_set([(14, rtcdf.rtcdf_tune_n_class(n),
                               rtcdf.Params(tile_width=2048, hist_threads=512,
                                            fill_threads=256, fill_chunk=4096))])
        p = rtcdf.rtcdf_plan(n, R)
        assert (p.tile_width, p.hist_threads, p.fill_threads) == (2048, 512, 256)
        assert p.fill_ctas == -(-n // 4096) or abs(p.fill_ctas - n / 4096) <= 2
        # another size class is untouched
        q = rtcdf.rtcdf_plan(1 << 22, R)
        assert q.tile_width == R
        for d in (0, 1, 2):
            x = dev_keys(n, 3, R, d, gen.derive_seed(61, d))
            assert_matches_oracle(x, gpu_sort(x, 3, 3 + R), 3, 3 + R)
    finally:
        rtcdf.rtcdf_tune_reset()


def test_entry_that_does_not_fit_falls_back_to_rules():
    R, n = 1 << 16, 100_000
    rtcdf.rtcdf_tune_set([])
    rule = rtcdf.rtcdf_plan(n, R)
    try:
        rtcdf.rtcdf_tune_set([(16, 0, rtcdf.Params(tile_width=1 << 20))])
        p = rtcdf.rtcdf_plan(n, R)
        assert p.tile_width == rule.tile_width
        x = dev_keys(n, 0, R, 0, gen.derive_seed(62))
        assert_matches_oracle(x, gpu_sort(x, 0, R), 0, R)
    finally:
        rtcdf.rtcdf_tune_reset()


def test_builtin_table_entries_give_exact_sorts():
    """Every compiled-in entry, exercised at a size of its class."""
    entries = rtcdf.rtcdf_tune_get()
    sizes = {0: 70_001, 1: 3_000_017, 2: 1 << 26}
    for lr, nc, _ in entries[:40]:
        R = 1 << lr
        n = sizes[nc]
        x = dev_keys(n, -5, R, 1, gen.derive_seed(63, lr, nc))
        out = gpu_sort(x, -5, -5 + R)
        if n <= 4_000_000:
            assert_matches_oracle(x, out, -5, -5 + R)
        else:
            o = out.cpu().numpy()
            assert (o[1:] >= o[:-1]).all()
            h = torch.bincount((x.long() + 5), minlength=R)
            assert torch.equal(torch.bincount(out.long() + 5, minlength=R), h)
