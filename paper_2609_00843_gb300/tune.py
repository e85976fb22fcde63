"""Autotuner for the launch parameters of the single-array sort and the
work-item sizes of the segmented sort.

The paper fixes one tile width per range size by measuring every candidate
width on 20 conditions (10 input sizes x 2 input distributions), normalising
each time by the fastest candidate of its condition and keeping the width with
the smallest geometric mean of the normalised times (Section 4.1).  This module
applies that rule on the device at hand to every launch parameter, in two
stages per (range class, size class):

1. histogram: tile width T and threads per histogram CTA;
2. output: threads per output CTA and output positions per CTA,
   with the stage-1 winner fixed.

The measurement itself is ``rtcdf_autotune`` in the library (CUDA events on
the launching stream, median of ``reps`` sorts per condition and candidate,
the geometric-mean ranking).  A candidate replaces the built-in rule only when
its geometric mean beats the built-in rule's by more than ``margin`` (1 %);
otherwise the class keeps the rule, so that timing noise does not turn into
table entries.

Conditions: R = 2^l for range class l; input sizes spread over the size class
(small n < 2^20, medium n < 2^26, large); uniform and normal keys (the
generator's shapes).  Run on the target GPU::

    python -m paper_2609_00843_gb300.tune --out DIR

which writes DIR/tune_table.json (every measured time and geometric mean) and
DIR/tune_table.inc (the table in the form csrc/tune_table.inc takes; copy it
there and rebuild to make it the library's built-in table).  With
``--batched`` it ranks the segmented sort's work-item sizes (histogram keys
per item, output positions per item, longest in-CTA segment) over several
segment-shape mixes by the same rule and writes DIR/tune_batched.json.
"""
from __future__ import annotations

import argparse
import json
import os
import time

SIZES = {0: [1 << 14, 1 << 16, 1 << 19], 1: [1 << 21, 1 << 23, 1 << 25],
         2: [1 << 26, 100_000_000, 1 << 28]}
SIZES_WIDE_R = {2: [1 << 26, 1 << 27]}   # range classes >= 20: fewer keys (every tile rescans them)
DISTS = (0, 1)                            # uniform, normal
FILL_THREADS = (256, 512, 1024)
FILL_CHUNKS = (0, 8192, 16384, 32768, 65536, 131072)
MIN_VAL = -1000


def _round1024(x: int) -> int:
    return (x + 1023) // 1024 * 1024


def hist_candidates(R: int, t_max: int):
    """(T, hist_threads) pairs for range size R; T = 0 is the built-in rule."""
    from .rtcdf import Params
    widths = set()
    if R <= t_max:
        widths.add(R)
        for m in (2, 3):
            T = _round1024(-(-R // m))
            if 1024 <= T < R:
                widths.add(T)
    else:
        m0 = -(-R // t_max)
        for m in (m0, m0 + 1, m0 + 2):
            widths.add(min(t_max, _round1024(-(-R // m))))
        widths.add(t_max)
    out = [Params()]
    for T in sorted(widths, reverse=True):
        for ht in (1024, 512):
            out.append(Params(tile_width=T, hist_threads=ht))
    return out


def fill_candidates(base):
    from .rtcdf import Params
    out = [Params(tile_width=base.tile_width, hist_threads=base.hist_threads)]
    for ft in FILL_THREADS:
        for fc in FILL_CHUNKS:
            if ft == 512 and fc == 0:
                continue  # same as the first (built-in rule)
            out.append(Params(tile_width=base.tile_width, hist_threads=base.hist_threads,
                              fill_threads=ft, fill_chunk=fc))
    return out


def _params_dict(p) -> dict:
    return {"tile_width": p.tile_width, "hist_threads": p.hist_threads,
            "fill_threads": p.fill_threads, "fill_chunk": p.fill_chunk}


def _pick(geomean, margin: float) -> int:
    """Index 0 is the built-in rule; another candidate must beat it by `margin`."""
    best = min(range(len(geomean)), key=lambda k: geomean[k])
    if best != 0 and geomean[best] * (1.0 + margin) >= geomean[0]:
        return 0
    return best


def tune(classes, n_classes=(0, 1, 2), reps: int = 5, margin: float = 0.01, log=print) -> dict:
    import torch

    from . import _build, gen, rtcdf
    _build.build()
    torch.cuda.init()
    stream = torch.cuda.Stream()
    sh = stream.cuda_stream
    rtcdf.rtcdf_tune_set([])  # measure against the built-in rules only
    t_max = rtcdf.rtcdf_plan(1 << 20, 1 << 24).tile_width
    n_max = max(max(v) for v in SIZES.values())
    buf_in = torch.empty(n_max, dtype=torch.int32, device="cuda")
    buf_out = torch.empty(n_max, dtype=torch.int32, device="cuda")
    record = {"device": torch.cuda.get_device_name(0), "t_max": t_max, "reps": reps,
              "margin": margin, "groups": []}
    entries = []
    for lr in classes:
        R = 1 << lr
        ws_bytes = rtcdf.rtcdf_workspace_size(R)
        ws = torch.zeros(ws_bytes // 4 + 64, dtype=torch.int32, device="cuda")
        for nc in n_classes:
            sizes = SIZES_WIDE_R.get(nc, SIZES[nc]) if lr >= 20 else SIZES[nc]
            conds = []
            offs = 0
            # Every condition gets its own slice of the buffers.
            if sum(sizes) * len(DISTS) > n_max:
                offs = None
            cases = []
            for n in sizes:
                for d in DISTS:
                    if offs is None:
                        base = 0
                    else:
                        base = offs
                        offs += n
                    conds.append({"n": n, "dist": d, "base": base})
            t0 = time.time()
            # Conditions that share buffer space are tuned one at a time.
            if offs is None:
                groups = [[c] for c in conds]
            else:
                groups = [conds]
            stage_res = []
            best_params = None
            for stage in ("hist", "fill"):
                cands = hist_candidates(R, t_max) if stage == "hist" else fill_candidates(best_params)
                times = [[0.0] * len(cands) for _ in conds]
                ci = 0
                for grp in groups:
                    cases = []
                    for c in grp:
                        seed = gen.derive_seed(11, lr, c["n"], c["dist"])
                        gen.keys_device(buf_in.data_ptr() + 4 * c["base"], c["n"], MIN_VAL, R,
                                        c["dist"], seed, stream=sh)
                        cases.append((buf_in.data_ptr() + 4 * c["base"],
                                      buf_out.data_ptr() + 4 * c["base"], c["n"], MIN_VAL,
                                      MIN_VAL + R))
                    t, _, _ = rtcdf.rtcdf_autotune(cases, cands, reps, ws.data_ptr(), ws_bytes, sh)
                    for row in t:
                        times[ci] = row
                        ci += 1
                gm = _geomean(times)
                k = _pick(gm, margin)
                best_params = cands[k]
                stage_res.append({"stage": stage, "candidates": [_params_dict(p) for p in cands],
                                  "times_ms": times, "geomean": gm, "chosen": k})
            chosen = best_params
            if any((chosen.tile_width, chosen.hist_threads, chosen.fill_threads, chosen.fill_chunk)):
                entries.append((lr, nc, chosen))
            record["groups"].append({"log2_R": lr, "n_class": nc, "conditions": [
                {"n": c["n"], "dist": c["dist"]} for c in conds], "stages": stage_res,
                "chosen": _params_dict(chosen), "seconds": round(time.time() - t0, 2)})
            log(f"log2R={lr:2d} n_class={nc}: {_params_dict(chosen)} "
                f"(hist gm {stage_res[0]['geomean'][stage_res[0]['chosen']]:.3f}, "
                f"fill gm {stage_res[1]['geomean'][stage_res[1]['chosen']]:.3f}, "
                f"{time.time() - t0:.1f} s)")
        del ws
    record["entries"] = [{"log2_R": lr, "n_class": nc, **_params_dict(p)} for lr, nc, p in entries]
    rtcdf.rtcdf_tune_reset()
    return record


BATCH_WORKLOADS = (
    # (segments, n_lo, n_hi, r_lo, r_hi, seed)
    (4096, 1e3, 1e6, 2 ** 7, 2 ** 16, 1),
    (4096, 1e3, 1e6, 2 ** 7, 2 ** 16, 2),
    (16384, 1e2, 1e4, 2 ** 4, 2 ** 12, 3),
    (512, 1e4, 1e7, 2 ** 10, 2 ** 18, 4),
)
BATCH_HIST_CHUNKS = (65536, 131072, 262144, 524288)
BATCH_FILL_CHUNKS = (16384, 32768, 65536, 131072)
BATCH_SMALL_MAX = (16384, 65535)


def tune_batched(reps: int = 5, margin: float = 0.01, log=print) -> dict:
    """Work-item sizes of the segmented sort, by the same geometric-mean rule
    over several segment-shape mixes (candidate 0 is the built-in choice)."""
    import numpy as np
    import torch

    from . import _build, gen, rtcdf
    _build.build()
    stream = torch.cuda.Stream()
    sh = stream.cuda_stream
    cands = [rtcdf.BatchParams()]
    for hc in BATCH_HIST_CHUNKS:
        for fc in BATCH_FILL_CHUNKS:
            for sm in BATCH_SMALL_MAX:
                cands.append(rtcdf.BatchParams(hist_chunk=hc, fill_chunk=fc, small_max_n=sm))
    times = []
    for (S, n_lo, n_hi, r_lo, r_hi, sd) in BATCH_WORKLOADS:
        L, mn, R, dist, seeds = gen.batched_segments(gen.derive_seed(12, sd), S, n_lo=n_lo,
                                                     n_hi=n_hi, r_lo=r_lo, r_hi=r_hi)
        offs = np.zeros(S + 1, dtype=np.int64)
        offs[1:] = np.cumsum(L)
        x = torch.empty(int(offs[-1]), dtype=torch.int32, device="cuda")
        out = torch.empty_like(x)
        for i in range(S):
            gen.keys_device(x.data_ptr() + 4 * int(offs[i]), int(L[i]), int(mn[i]), int(R[i]),
                            int(dist[i]), int(seeds[i]), stream=sh)
        row = []
        for p in cands:
            plan = rtcdf.BatchPlan(offs, mn, mn + R, p)
            wsb = max(256, plan.workspace_size())
            ws = torch.zeros(wsb // 4 + 64, dtype=torch.int32, device="cuda")
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(reps + 1)]
            plan.run(x.data_ptr(), out.data_ptr(), ws.data_ptr(), wsb, sh)
            ev[0].record(stream)
            for r in range(reps):
                rc = plan.run(x.data_ptr(), out.data_ptr(), ws.data_ptr(), wsb, sh)
                if rc != rtcdf.OK:
                    raise rtcdf.RtcdfError(rc, "rtcdf_sort_batched_ws")
                ev[r + 1].record(stream)
            stream.synchronize()
            rc, bits = rtcdf.rtcdf_batch_status_get(ws.data_ptr(), sh)
            if rc != rtcdf.OK:
                raise rtcdf.RtcdfError(rc, "batched device status")
            ts = sorted(ev[r].elapsed_time(ev[r + 1]) for r in range(reps))
            row.append(ts[reps // 2])
            plan.close()
            del ws
        times.append(row)
        log(f"workload {S} segs n[{n_lo:g},{n_hi:g}] R[{r_lo},{r_hi}]: rule {row[0]:.3f} ms, "
            f"best {min(row):.3f} ms")
        del x, out
    gm = _geomean(times)
    k = _pick(gm, margin)
    fields = ("hist_chunk", "fill_chunk", "small_max_n")
    return {"workloads": [list(w) for w in BATCH_WORKLOADS],
            "candidates": [{f: getattr(p, f) for f in fields} for p in cands],
            "times_ms": times, "geomean": gm, "chosen": k,
            "chosen_params": {f: getattr(cands[k], f) for f in fields}}


def _geomean(times):
    """Section 4.1's rule over a [condition][candidate] table (-1 = cannot run)."""
    import math
    k = len(times[0])
    logs = [0.0] * k
    ok = [True] * k
    for row in times:
        valid = [v for v in row if v > 0]
        tmin = min(valid)
        for j, v in enumerate(row):
            if v > 0:
                logs[j] += math.log(v / tmin)
            else:
                ok[j] = False
    return [math.exp(logs[j] / len(times)) if ok[j] else float("inf") for j in range(k)]


def write_inc(entries, path: str) -> None:
    lines = ["// Built-in tuning table: {ceil(log2 R), n class, {T, hist CTAs per tile,",
             "// hist threads, output CTAs, output threads, output chunk, {0, 0}}}.",
             "// Zero = built-in rule.  Written by paper_2609_00843_gb300.tune from",
             "// measurements on GB300."]
    for e in entries:
        lines.append("{%d, %d, {%d, 0, %d, 0, %d, %d, {0, 0}}}," % (
            e["log2_R"], e["n_class"], e["tile_width"], e["hist_threads"], e["fill_threads"],
            e["fill_chunk"]))
    with open(path, "w") as f:
        f.write("\n".join(lines) + "\n")


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--out", required=True)
    ap.add_argument("--log2r", default="1-24", help="range classes, e.g. 1-24 or 7,10,14,18")
    ap.add_argument("--n-classes", default="0,1,2")
    ap.add_argument("--reps", type=int, default=5)
    ap.add_argument("--batched", action="store_true",
                    help="tune the segmented sort's work-item sizes instead")
    args = ap.parse_args()
    os.makedirs(args.out, exist_ok=True)
    if args.batched:
        rec = tune_batched(args.reps)
        with open(os.path.join(args.out, "tune_batched.json"), "w") as f:
            json.dump(rec, f, indent=1)
        print("chosen:", rec["chosen_params"], "geomean", rec["geomean"][rec["chosen"]],
              "rule geomean", rec["geomean"][0])
        return
    if "-" in args.log2r:
        a, b = args.log2r.split("-")
        classes = list(range(int(a), int(b) + 1))
    else:
        classes = [int(x) for x in args.log2r.split(",")]
    ncl = [int(x) for x in args.n_classes.split(",")]
    rec = tune(classes, ncl, args.reps)
    with open(os.path.join(args.out, "tune_table.json"), "w") as f:
        json.dump(rec, f, indent=1)
    write_inc(rec["entries"], os.path.join(args.out, "tune_table.inc"))
    print(f"{len(rec['entries'])} entries written to {args.out}")


if __name__ == "__main__":
    main()
