"""Host-side pieces of the benchmark (no GPU): the roofline denominator, the
validity check of the committed DRAM-traffic records, and the reference arm's
JSON line (the CPU oracle on a sample of the sweep)."""
import importlib.util
import json
import os
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


HIST = ["paper_2609_00843_gb300/csrc/hist.cu", "paper_2609_00843_gb300/csrc/rtcdf_internal.h"]
FILL = ["paper_2609_00843_gb300/csrc/fill.cu", "paper_2609_00843_gb300/csrc/rtcdf_internal.h"]


def test_peak_is_the_measured_copy_bandwidth(bench):
    with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
        measured = float(json.load(f)["hbm_gbs"])
    assert bench.peaks() == (measured, "measured")


def test_code_digest_ignores_comments_and_whitespace_only(bench, tmp_path, monkeypatch):
    src = "// header\nint f(int x) {  /* note */\n    return x + 1;   // tail\n}\n"
    (tmp_path / "a.cu").write_text(src)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    d0 = bench.code_sha256(["a.cu"])
    (tmp_path / "a.cu").write_text("/* another\n header */ int f(int x) {\n\treturn x + 1;\n}\n")
    assert bench.code_sha256(["a.cu"]) == d0
    (tmp_path / "a.cu").write_text("int f(int x) { return x + 2; }\n")
    assert bench.code_sha256(["a.cu"]) != d0


def test_traffic_records_are_current_or_null(bench):
    # A record is reported only while the kernel code is the code it was
    # captured on (else null); a reported record is within a few percent of
    # the kernel's algorithmic 4n bytes at n = 1e8.
    with open(os.path.join(ROOT, "profiles", "ncu_traffic.json")) as f:
        rec = json.load(f)
    for kernel, files in (("hist_kernel", HIST), ("fill_kernel", FILL)):
        assert rec.get(kernel), kernel
        t = bench.traffic_for(kernel, files)
        current = any(r["code_sha256"] == bench.code_sha256(files) for r in rec[kernel].values())
        assert (t is not None) == current, kernel
        if t is not None:
            assert 0.8 * 4e8 < t < 1.1 * 4e8, (kernel, t)


def test_traffic_is_null_once_the_kernel_changes(bench, tmp_path, monkeypatch):
    for p in HIST + ["profiles/ncu_traffic.json"]:
        os.makedirs(tmp_path / os.path.dirname(p), exist_ok=True)
        shutil.copy(os.path.join(ROOT, p), tmp_path / p)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    # A record taken on the code as it stands in the copy...
    with open(tmp_path / "profiles/ncu_traffic.json") as f:
        rec = json.load(f)
    for r in rec["hist_kernel"].values():
        r["code_sha256"] = bench.code_sha256(HIST)
    with open(tmp_path / "profiles/ncu_traffic.json", "w") as f:
        json.dump(rec, f)
    assert bench.traffic_for("hist_kernel", HIST) is not None
    # ...survives a comment, not a code change.
    with open(tmp_path / HIST[0], "a") as f:
        f.write("\n// a comment keeps the record\n")
    assert bench.traffic_for("hist_kernel", HIST) is not None
    with open(tmp_path / HIST[0], "a") as f:
        f.write("\nstatic int changed_code = 1;\n")
    assert bench.traffic_for("hist_kernel", HIST) is None


def test_reference_arm_prints_the_contract_line(bench, monkeypatch, capsys):
    # The reference arm (the CPU oracle) on a small sample of the sweep.
    import types
    monkeypatch.setattr(bench, "N_SWEEP", 1_000_000)
    args = types.SimpleNamespace(steps=1, warmup=0)
    assert bench.run_reference(args, 0, 1) == 0
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC
    assert line["unit"] == "GKeys/s" and line["value"] > 0 and line["higher_is_better"] is True
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] == 1
    assert line["e2e"] == {"value": line["value"], "unit": "GKeys/s",
                           "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert line["config"]["arrays"] == 12 and line["config"]["n_per_array"] == 1_000_000
    # Other ranks of a multi-process launch do no work and print nothing.
    assert bench.run_reference(args, 1, 2) == 0
    assert capsys.readouterr().out == ""
