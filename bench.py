#!/usr/bin/env python
"""RT-CDF sort benchmark: GKeys/s and fraction of the 8n-byte HBM roofline.

One step is one pass of the whole hot path (histogram, local-CDF/offset scan,
output generation) over the sweep workload: twelve int32 arrays of n = 1e8
keys with minVal = -1000, range sizes R in {2^7, 2^10, 2^14, 2^18} and the
uniform / normal / all-equal shapes of the paper's evaluation.  Inputs are
generated on the device by the seeded generator and stay resident in HBM;
each array (400 MB) is larger than L2, so no flush is needed between steps.
The twelve arrays are independent, so the timed step sorts them on
``--streams`` streams (default 12, one per array; round robin when fewer); the same steps on one stream
are reported beside it (``one_stream``), and the per-array figures
(``per_config``) are single-stream.

Prints one JSON line (rank 0).  ``--impl reference`` times the CPU oracle on
the host cores instead (the reference arm of this comparison).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_SWEEP = 100_000_000
MIN_SWEEP = -1000
SWEEP_R = [1 << 7, 1 << 10, 1 << 14, 1 << 18]
DIST_NAMES = ["uniform", "normal", "all_equal"]
# The benchmark's metric: GKeys/s on the sweep (`value`), with the fraction of
# the 8n-byte roofline per R (`per_config`), the segmented sort against looped
# calls (`batched`) and the server's p99 (`serve`) in the same line.
METRIC = "GKeys/s and % of 8n-byte HBM roofline per R; batched vs looped; serve p99"
WORKLOAD = ("sweep: n=1e8 int32 keys per array, minVal=-1000, R in {2^7,2^10,2^14,2^18} x "
            "{uniform, normal(mean minVal+R/2, sd R/8), all-equal(minVal+R/3)}; 12 arrays per step")


SPEC_HBM_GBS = 7900.0  # GB300 HBM3e nominal bandwidth: the second (spec) roofline column


def paper_protocol_ms(sort_once, stream, runs=3, reps=30, warm=10, between=None):
    """The paper's timing protocol (Section 4): `warm` untimed sorts, then
    `runs` runs of `reps` sorts, each sort bracketed by CUDA events on the
    launching stream; the median of the per-run medians.  `between` (e.g. an
    L2 flush) runs after each timed sort, outside its events."""
    import torch
    for _ in range(warm):
        sort_once()
    meds = []
    for _ in range(runs):
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(reps)]
        for a, b in ev:
            a.record(stream)
            sort_once()
            b.record(stream)
            if between is not None:
                between()
        stream.synchronize()
        ts = sorted(a.elapsed_time(b) for a, b in ev)
        meds.append(ts[len(ts) // 2])
    return statistics.median(meds)


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def sweep_cases():
    from paper_2609_00843_gb300 import gen
    cases = []
    for R in SWEEP_R:
        for d, name in enumerate(DIST_NAMES):
            cases.append(dict(R=R, dist=d, dist_name=name,
                              seed=gen.derive_seed(1, d, R.bit_length() - 1)))
    return cases


class ClockSampler:
    """nvidia-smi clock / throttle sampling while the timed region runs."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def code_sha256(src_files) -> str:
    """sha256 of the kernel sources with comments and whitespace removed, so
    that an edit of comments alone keeps committed counters valid."""
    h = hashlib.sha256()
    for p in src_files:
        with open(os.path.join(ROOT, p)) as f:
            text = f.read()
        text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
        text = re.sub(r"//[^\n]*", " ", text)
        h.update(" ".join(text.split()).encode())
    return h.hexdigest()


def traffic_for(kernel: str, src_files):
    """DRAM bytes per launch of `kernel` on the sweep arrays, averaged over the
    ncu captures committed in profiles/ncu_traffic.json -- only if they were
    taken from the current kernel source; otherwise None."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        with open(path) as f:
            table = json.load(f)
    except Exception:
        return None
    digest = code_sha256(src_files)
    ents = [e for k, e in table.get(kernel, {}).items() if k.startswith("sweep_n1e8")]
    if not ents or any(e.get("code_sha256") != digest for e in ents):
        return None
    return round(sum(e["dram_bytes_per_launch"] for e in ents) / len(ents))


def run_reference(args, rank, world):
    """Reference arm: the CPU oracle on the host cores, on the sweep workload."""
    import numpy as np

    import oracle
    from paper_2609_00843_gb300 import gen
    if rank != 0:
        return 0
    # Bounded sample per step: every array of the sweep at n_sample keys,
    # sized so that warm-up + timed steps finish within a few minutes.
    total_steps = args.steps + args.warmup
    n_sample = int(max(1_000_000, min(N_SWEEP, 12_000_000 * 10 // max(1, total_steps))))
    cases = sweep_cases()
    inputs = [gen.keys_host(n_sample, MIN_SWEEP, c["R"], c["dist"], c["seed"]) for c in cases]
    lib = oracle.load()
    times = []
    for step in range(total_steps):
        t0 = time.perf_counter()
        for c, a in zip(cases, inputs):
            oracle.counting_sort(a, MIN_SWEEP, MIN_SWEEP + c["R"], lib)
        dt = time.perf_counter() - t0
        if step >= args.warmup:
            times.append(dt)
    keys = n_sample * len(cases)
    t = sum(times) / len(times)
    value = keys / t / 1e9
    line = {
        "metric": METRIC,
        "value": value, "unit": "GKeys/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "impl": "reference",
        "config": {"workload": WORKLOAD, "n_per_array": n_sample, "arrays": len(cases)},
        "cpu_baseline": {"value": value, "unit": "GKeys/s", "cores": 1, "kind": "oracle",
                         "sample": f"12 sweep arrays at n={n_sample} keys each per step",
                         **cpu_info()},
        "e2e": {"value": value, "unit": "GKeys/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
        "gpu_launches": 0,
    }
    print(json.dumps(line), flush=True)
    return 0


# Arm core part numbers (MIDR_EL1 bits 4..15) of the implementer Arm (0x41)
# and NVIDIA (0x4e) cores a GPU host is likely to have.
_ARM_PARTS = {(0x41, 0xd4f): "Arm Neoverse V2", (0x41, 0xd84): "Arm Neoverse V3",
              (0x41, 0xd40): "Arm Neoverse V1", (0x41, 0xd0c): "Arm Neoverse N1",
              (0x41, 0xd49): "Arm Neoverse N2", (0x4e, 0x004): "NVIDIA Carmel"}


def _lscpu_model() -> str:
    import subprocess
    try:
        r = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10)
    except (OSError, subprocess.SubprocessError):
        return ""
    for ln in r.stdout.splitlines():
        if ln.split(":")[0].strip().lower() == "model name" and ":" in ln:
            name = ln.split(":", 1)[1].strip()
            if name and name != "-":
                return name
    return ""


def _midr_model() -> str:
    try:
        with open("/sys/devices/system/cpu/cpu0/regs/identification/midr_el1") as f:
            midr = int(f.read().strip(), 16)
    except (OSError, ValueError):
        return ""
    impl, part = (midr >> 24) & 0xFF, (midr >> 4) & 0xFFF
    return _ARM_PARTS.get((impl, part), f"Arm core implementer 0x{impl:02x} part 0x{part:03x}")


def cpu_info() -> dict:
    """Host CPU model and core count, for the CPU baseline's record: the model
    name of /proc/cpuinfo (x86), else lscpu's (Arm hosts, whose /proc/cpuinfo
    has none), else the core named by MIDR_EL1, else the architecture."""
    model = ""
    try:
        with open("/proc/cpuinfo") as f:
            for ln in f:
                k = ln.split(":")[0].strip().lower()
                if k in ("model name", "cpu model") and ":" in ln:
                    model = ln.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    model = model or _lscpu_model() or _midr_model()
    if not model:
        import platform
        model = platform.processor() or platform.machine()
    return {"cpu_model": model, "nproc": os.cpu_count()}


def cpu_baseline_sweep(host_inputs, cases):
    """The oracle, as it stands, on one pass over the 12 full-size arrays."""
    import oracle
    lib = oracle.load()
    t0 = time.perf_counter()
    for c, a in zip(cases, host_inputs):
        oracle.counting_sort(a, MIN_SWEEP, MIN_SWEEP + c["R"], lib)
    dt = time.perf_counter() - t0
    keys = sum(a.size for a in host_inputs)
    ci = cpu_info()
    return {"value": keys / dt / 1e9, "unit": "GKeys/s", "cores": 1, "kind": "oracle",
            "sample": f"one pass over the 12 sweep arrays (n=1e8 each, {keys} keys), "
                      f"{dt:.1f} s single-threaded (1 of {ci['nproc']} cores)", **ci}


def single_config(stream):
    """The small workload: n = 1e6 int32 keys, minVal = 0, R = 2^7, uniform,
    seed 0.  Its 8 MB working set sits in L2, so it is timed warm (back-to-back
    sorts of the same array) and with L2 flushed between sorts (a 256 MB buffer
    written after each timed sort, outside its events)."""
    import torch
    from paper_2609_00843_gb300 import gen, rtcdf
    n, R = 1_000_000, 1 << 7
    sh = stream.cuda_stream
    with torch.cuda.stream(stream):
        x = torch.empty(n, dtype=torch.int32, device="cuda")
        gen.keys_device(x.data_ptr(), n, 0, R, gen.UNIFORM, 0, stream=sh)
        out = torch.empty_like(x)
        flush = torch.empty(64 << 20, dtype=torch.int32, device="cuda")
    wsb = rtcdf.rtcdf_workspace_size(R)
    ws = torch.zeros(wsb // 4 + 64, dtype=torch.int32, device="cuda")
    stream.synchronize()

    def once():
        rc = rtcdf.rtcdf_sort_ws(x.data_ptr(), out.data_ptr(), n, 0, R, ws.data_ptr(), wsb, sh)
        if rc != rtcdf.OK:
            raise rtcdf.RtcdfError(rc, "rtcdf_sort_ws")

    def do_flush():
        with torch.cuda.stream(stream):
            flush.fill_(1)
    warm = paper_protocol_ms(once, stream)
    cold = paper_protocol_ms(once, stream, between=do_flush)
    # The same sort captured once in a CUDA graph and replayed (no host work
    # per sort: what a caller that replays a captured pipeline sees).
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        once()
    stream.synchronize()

    def replay():
        with torch.cuda.stream(stream):
            g.replay()
    graph = paper_protocol_ms(replay, stream)
    # Back to back: 200 sorts between two events (no event between sorts, so
    # each sort's launches overlap the tail of the one before).
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(200):
        once()
    e1.record(stream)
    stream.synchronize()
    b2b = e0.elapsed_time(e1) / 200
    # host wall-clock of one call + synchronisation (what a blocking caller sees)
    walls = []
    for _ in range(30):
        t0 = time.perf_counter()
        once()
        stream.synchronize()
        walls.append((time.perf_counter() - t0) * 1e3)
    res = {"workload": "n=1e6 int32, minVal=0, R=2^7, uniform, seed 0",
           "warm_ms": round(warm, 5), "l2_flushed_ms": round(cold, 5),
           "graph_replay_ms": round(graph, 5),
           "back_to_back_ms": round(b2b, 5),
           "warm_GKeys_s": round(n / (warm * 1e-3) / 1e9, 2),
           "graph_replay_GKeys_s": round(n / (graph * 1e-3) / 1e9, 2),
           "l2_flushed_GKeys_s": round(n / (cold * 1e-3) / 1e9, 2),
           "host_wall_ms_median": round(statistics.median(walls), 4),
           "note": "launch-latency bound: 8n bytes at the copy bandwidth take ~1.2 us; warm, "
                   "l2_flushed and graph_replay are the paper protocol (events around each sort), "
                   "back_to_back is 200 sorts between two events"}
    del g, x, out, flush, ws
    return res


def large_config(stream):
    """The large workload: n = 1e9 int32 keys (4 GB in, 4 GB out), minVal = 0,
    R in {2^12, 2^16, 2^18}, uniform and normal; one array at a time."""
    import torch
    from paper_2609_00843_gb300 import gen, rtcdf
    n = 1_000_000_000
    sh = stream.cuda_stream
    hbm, _ = peaks()
    with torch.cuda.stream(stream):
        x = torch.empty(n, dtype=torch.int32, device="cuda")
        out = torch.empty_like(x)
    wsb = rtcdf.rtcdf_workspace_size(1 << 18)
    ws = torch.zeros(wsb // 4 + 64, dtype=torch.int32, device="cuda")
    rows = []
    for R in (1 << 12, 1 << 16, 1 << 18):
        for d, name in ((gen.UNIFORM, "uniform"), (gen.NORMAL, "normal")):
            gen.keys_device(x.data_ptr(), n, 0, R, d, gen.derive_seed(3, d, R.bit_length() - 1),
                            stream=sh)

            def once(R=R):
                rc = rtcdf.rtcdf_sort_ws(x.data_ptr(), out.data_ptr(), n, 0, R, ws.data_ptr(), wsb, sh)
                if rc != rtcdf.OK:
                    raise rtcdf.RtcdfError(rc, "rtcdf_sort_ws")
            ms = paper_protocol_ms(once, stream, runs=3, reps=5, warm=2)
            rc, bits = rtcdf.rtcdf_ws_status_get(ws.data_ptr(), sh)
            if rc != rtcdf.OK:
                raise rtcdf.RtcdfError(rc, "device status (large)")
            rows.append({"R": R, "dist": name, "ms": round(ms, 4),
                         "GKeys_s": round(n / (ms * 1e-3) / 1e9, 1),
                         "frac_8n_roofline": round(8 * n / (ms * 1e-3) / 1e9 / hbm, 4)})
    del x, out, ws
    torch.cuda.empty_cache()
    return {"workload": "n=1e9 int32, minVal=0, R in {2^12,2^16,2^18}, uniform/normal",
            "rows": rows}


def cub_comparison(cases, ins, outs, n, stream, nsteps, ours_ms):
    import ctypes

    import torch
    from paper_2609_00843_gb300 import _build
    path = os.path.join(ROOT, "paper_2609_00843_gb300", "cub_baseline", "_build", "librtcdf_cub.so")
    lib = ctypes.CDLL(path)
    vp, u64, i64 = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int64
    lib.rtcdf_cub_temp_bytes.argtypes = [u64, i64, ctypes.POINTER(ctypes.c_size_t)]
    lib.rtcdf_cub_normalize.argtypes = [vp, vp, u64, i64, vp]
    lib.rtcdf_cub_sort_keys.argtypes = [vp, vp, vp, ctypes.c_size_t, u64, i64, vp]
    lib.rtcdf_cub_denormalize.argtypes = [vp, vp, u64, i64, vp]
    sh = stream.cuda_stream
    k_in = torch.empty(n, dtype=torch.int32, device="cuda")
    k_out = torch.empty(n, dtype=torch.int32, device="cuda")
    res = torch.empty(n, dtype=torch.int32, device="cuda")
    tb = ctypes.c_size_t(0)
    lib.rtcdf_cub_temp_bytes(n, 1 << 18, ctypes.byref(tb))
    temp = torch.empty(tb.value + 256, dtype=torch.uint8, device="cuda")
    rows = []
    for i, c in enumerate(cases):
        R = c["R"]
        ev = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(nsteps)]
        def once(e=None):
            if e: e[0].record(stream)
            assert lib.rtcdf_cub_normalize(ins[i].data_ptr(), k_in.data_ptr(), n, MIN_SWEEP, sh) == 0
            if e: e[1].record(stream)
            assert lib.rtcdf_cub_sort_keys(k_in.data_ptr(), k_out.data_ptr(), temp.data_ptr(),
                                           tb.value, n, R, sh) == 0
            if e: e[2].record(stream)
            assert lib.rtcdf_cub_denormalize(k_out.data_ptr(), res.data_ptr(), n, MIN_SWEEP, sh) == 0
            if e: e[3].record(stream)
        for _ in range(3):
            once()
        for k in range(nsteps):
            once(ev[k])
        stream.synchronize()
        st = [sum(ev[k][j].elapsed_time(ev[k][j + 1]) for k in range(nsteps)) / nsteps for j in range(3)]
        same = bool(torch.equal(res, outs[i]))
        rows.append({"R": R, "dist": c["dist_name"], "cub_sortkeys_ms": round(st[1], 5),
                     "normalize_ms": round(st[0], 5), "denormalize_ms": round(st[2], 5),
                     "rtcdf_ms": round(ours_ms[i], 5),
                     "speedup_vs_cub_sortkeys": round(st[1] / ours_ms[i], 3),
                     "outputs_equal": same})
    del k_in, k_out, res, temp
    return rows


def batched_comparison(args, stream, num_segments=4096):
    """Batched workload: 4096 segments, lengths log-uniform in [1e3, 1e6],
    R log-uniform in [2^7, 2^16], minVal uniform in [-2^20, 2^20], mixed
    shapes.  One plan (three launches, graph-captured) against looped
    rtcdf_sort calls (plain and graph-captured), keys/s of each."""
    import numpy as np
    import torch
    from paper_2609_00843_gb300 import gen, rtcdf
    sh = stream.cuda_stream
    L, mn, R, dist, seeds = gen.batched_segments(gen.derive_seed(4), num_segments)
    offs = np.zeros(num_segments + 1, dtype=np.int64)
    offs[1:] = np.cumsum(L)
    total = int(offs[-1])
    mx = mn + R
    x = torch.empty(total, dtype=torch.int32, device="cuda")
    out = torch.empty_like(x)
    for i in range(num_segments):
        gen.keys_device(x.data_ptr() + 4 * int(offs[i]), int(L[i]), int(mn[i]), int(R[i]),
                        int(dist[i]), int(seeds[i]), stream=sh)
    stream.synchronize()
    plan = rtcdf.BatchPlan(offs, mn, mx)
    wsb = plan.workspace_size()
    ws = torch.zeros(wsb // 4 + 64, dtype=torch.int32, device="cuda")
    steps = max(3, min(args.steps, 10))

    def timed(fn, reps):
        # Everything (including graph replays, which launch on torch's current
        # stream) runs on `stream`, where the events are recorded.
        with torch.cuda.stream(stream):
            fn()
            stream.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(reps):
                fn()
            e1.record(stream)
            stream.synchronize()
        return e0.elapsed_time(e1) / reps

    def batched():
        rc = plan.run(x.data_ptr(), out.data_ptr(), ws.data_ptr(), wsb, sh)
        if rc != rtcdf.OK:
            raise rtcdf.RtcdfError(rc, "rtcdf_sort_batched_ws")
    ms_batched = timed(batched, steps)
    rc, bits = rtcdf.rtcdf_batch_status_get(ws.data_ptr(), sh)
    if rc != rtcdf.OK:
        raise rtcdf.RtcdfError(rc, "batched device status")
    ref = out.clone()

    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        batched()
    ms_batched_graph = timed(g.replay, steps)

    # Looped single-array calls on one stream (library workspace reserved).
    rtcdf.rtcdf_reserve(int(R.max()), sh)
    o_ptr, x_ptr = out.data_ptr(), x.data_ptr()
    segs = [(int(offs[i]), int(L[i]), int(mn[i]), int(mx[i])) for i in range(num_segments)]

    def looped():
        for off, n, a, b in segs:
            rc = rtcdf.rtcdf_sort(x_ptr + 4 * off, o_ptr + 4 * off, n, a, b, sh)
            if rc != rtcdf.OK:
                raise rtcdf.RtcdfError(rc, "rtcdf_sort")
    ms_looped = timed(looped, max(2, steps // 3))
    same = bool(torch.equal(out, ref))
    g2 = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g2, stream=stream):
        looped()
    ms_looped_graph = timed(g2.replay, steps)
    same = same and bool(torch.equal(out, ref))
    # One instrumented run: where the three launches spend their time.
    import torch as _t
    prof = _t.zeros(rtcdf.BATCH_PROFILE_WORDS, dtype=_t.int64, device="cuda")
    prof[8:12] = -1  # UINT64_MAX: earliest-start slots
    with _t.cuda.stream(stream):
        rc = plan.run_profiled(x.data_ptr(), out.data_ptr(), ws.data_ptr(), wsb, prof.data_ptr(), sh)
    stream.synchronize()
    if rc != rtcdf.OK:
        raise rtcdf.RtcdfError(rc, "rtcdf_sort_batched_profiled")
    words = [int(v) & ((1 << 64) - 1) for v in prof.cpu().tolist()]
    info = plan.info()
    phases = rtcdf.batch_profile_summary(words, info["workers"])
    plan.close()
    del ws
    # The same segments with the metadata in device memory, planned on the
    # device each run (rtcdf_sort_batched_device_ws), replayed from a graph.
    d_o = torch.from_numpy(offs).cuda()
    d_mn = torch.from_numpy(mn.astype(np.int64)).cuda()
    d_mx = torch.from_numpy(mx.astype(np.int64)).cuda()
    max_R = int(R.max())
    dwsb = rtcdf.rtcdf_batch_device_workspace_size(num_segments, total, max_R)
    dws = torch.zeros(dwsb // 4 + 64, dtype=torch.int32, device="cuda")

    def device_planned():
        rc = rtcdf.rtcdf_sort_batched_device_ws(x.data_ptr(), out.data_ptr(), d_o.data_ptr(), d_mn.data_ptr(),
                                                d_mx.data_ptr(), num_segments, total, max_R, dws.data_ptr(),
                                                dwsb, sh)
        if rc != rtcdf.OK:
            raise rtcdf.RtcdfError(rc, "rtcdf_sort_batched_device_ws")
    out.fill_(-1)
    device_planned()
    stream.synchronize()
    same = same and bool(torch.equal(out, ref))
    g3 = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g3, stream=stream):
        device_planned()
    ms_dev_graph = timed(g3.replay, steps)
    rc, bits = rtcdf.rtcdf_batch_status_get(dws.data_ptr(), sh)
    if rc != rtcdf.OK:
        raise rtcdf.RtcdfError(rc, "device-planned status")
    same = same and bool(torch.equal(out, ref))
    del dws, g3
    res = {
        "workload": f"{num_segments} segments: n log-uniform [1e3,1e6], R log-uniform [2^7,2^16], "
                    "minVal uniform [-2^20,2^20], mixed uniform/normal/all-equal",
        "total_keys": total,
        "batched_graph_GKeys_s": round(total / (ms_batched_graph * 1e-3) / 1e9, 2),
        "batched_GKeys_s": round(total / (ms_batched * 1e-3) / 1e9, 2),
        "looped_GKeys_s": round(total / (ms_looped * 1e-3) / 1e9, 2),
        "looped_graph_GKeys_s": round(total / (ms_looped_graph * 1e-3) / 1e9, 2),
        "batched_graph_ms": round(ms_batched_graph, 4), "batched_ms": round(ms_batched, 4),
        "looped_ms": round(ms_looped, 4), "looped_graph_ms": round(ms_looped_graph, 4),
        "speedup_vs_looped_graph": round(ms_looped_graph / ms_batched_graph, 2),
        "device_planned_graph_GKeys_s": round(total / (ms_dev_graph * 1e-3) / 1e9, 2),
        "device_planned_graph_ms": round(ms_dev_graph, 4),
        "device_planned_workspace_GB": round(dwsb / 1e9, 3),
        "frac_8n_roofline": round(8 * total / (ms_batched_graph * 1e-3) / 1e9 / peaks()[0], 4),
        "outputs_equal": same, "plan": info, "phases": phases,
    }
    del x, out, ref
    torch.cuda.empty_cache()
    return res


def sharded_comparison(cases, outs, n, rank, world, stream, steps):
    """The sweep's arrays sorted across the job's ranks: rank r holds the
    slice [r*n/N, (r+1)*n/N) of every array (the same global arrays on every
    rank), counts it (rtcdf_hist_accumulate), takes part in one sum
    all-reduce of the R counts per array (NCCL across GPUs), and writes the
    same window of the sorted array (rtcdf_fill_from_counts).  With one rank
    there is no exchange: the time shows what the split calls cost against
    rtcdf_sort.  Every window is checked against the unsharded sort on rank 0
    with one rank, and the counts' total against n with several."""
    import torch
    from paper_2609_00843_gb300 import dist as rdist, gen, rtcdf
    lo, hi = rdist.slice_bounds(n, world, rank)
    sh = stream.cuda_stream
    srt = rdist.ShardedSorter(max(c["R"] for c in cases), stream=stream)
    ins, wins = [], []
    for c in cases:
        x = torch.empty(hi - lo, dtype=torch.int32, device="cuda")
        gen.keys_device(x.data_ptr(), hi - lo, MIN_SWEEP, c["R"], c["dist"], c["seed"], first=lo, stream=sh)
        ins.append(x)
        wins.append(torch.empty(hi - lo, dtype=torch.int32, device="cuda"))
    stream.synchronize()

    def step():
        for i, c in enumerate(cases):
            srt.sort(ins[i], n, MIN_SWEEP, MIN_SWEEP + c["R"], wins[i], rank=rank, world=world)
    for _ in range(2):
        step()
    torch.cuda.synchronize()
    rdist.barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    rdist.barrier()
    ms = rdist.max_over_ranks(e0.elapsed_time(e1) / steps, device="cuda")
    rc, bits = srt.status()
    ok = rc == rtcdf.OK and bits == 0
    if world == 1 and outs:
        ok = ok and all(bool(torch.equal(wins[i], outs[i])) for i in range(len(cases)))
    del ins, wins
    return {"note": "each array sorted across the ranks: slice counts, one sum all-reduce of R counts, "
                    "own window of the output; 1 rank = no exchange",
            "ranks": world, "ms_per_step": round(ms, 4),
            "GKeys_s": round(n * len(cases) / (ms * 1e-3) / 1e9, 2),
            "exchange": "torch.distributed all_reduce (NCCL)" if world > 1 else "none",
            "windows_ok": bool(ok)}


def serving_comparison(count: int, budget_gb: float = 32.0, max_large: int = 0):
    """Serving workload: a Poisson stream of sort requests, n log-uniform in
    [1e4, 1e8], R log-uniform in [2^7, 2^18], mixed shapes, 32 GB admission
    budget.  The arrival rate is rho x the throughput of sequential
    per-request calls (measured first with every request present at t=0),
    rho in {0.5, 0.9, 1.5}; each trace is served sequentially and by the
    continuous-batching server.  Latency = completion - arrival; a request's
    keys are written into its device slot by the generator (data arrival):
    sequentially right before its sort; in the server on its launch's stream
    right before the sort (and, at rho = 0.5, also at admission for
    comparison)."""
    import numpy as np
    from paper_2609_00843_gb300 import gen, rtcdf
    seed = gen.derive_seed(5)
    n, mn, R, dist, seeds = gen.serving_requests(seed, count)
    mx = mn + R
    fill = gen.fill_function_address()

    def cfg(adaptive=True):
        # The serving policy: keys written on the launch's stream right before
        # its sort, one large launch at a time until four large requests wait
        # (then every stream).  adaptive=False: the previous policy (keys
        # written at admission on separate streams, large launches on every
        # stream), for comparison at rho = 0.5.
        return rtcdf.ServerConfig(budget_bytes=int(budget_gb * (1 << 30)), num_streams=4,
                                  max_batch=256, single_min_keys=1 << 22, fill=fill, digests=0,
                                  max_large_inflight=1 if adaptive else max_large,
                                  fill_at_launch=1 if adaptive else 0,
                                  large_queue_burst=4 if adaptive else 0)
    zero = np.zeros(count)
    r0 = rtcdf.make_requests(n, mn, mx, dist, seeds, zero)
    _, st0 = rtcdf.rtcdf_serve_sequential(cfg(), r0, count)
    _, st1 = rtcdf.rtcdf_serve_trace(cfg(), r0, count)
    seq_rate = count / st0.makespan_s
    out = {"workload": f"{count} requests, Poisson arrivals at rho x sequential throughput "
                       f"(rho in {{0.5, 0.9, 1.5}}), n log-uniform [1e4,1e8], R log-uniform "
                       f"[2^7,2^18], mixed shapes, {budget_gb:g} GB admission budget",
           "total_keys": int(n.sum()), "sequential_rate_per_s": round(seq_rate, 1),
           "saturated": {"note": "every request present at t=0: capacity in keys/s",
                         "sequential_GKeys_s": round(st0.total_keys / st0.makespan_s / 1e9, 2),
                         "server_GKeys_s": round(st1.total_keys / st1.makespan_s / 1e9, 2),
                         "server_vs_sequential": round(st0.makespan_s / st1.makespan_s, 3)},
           "load": {}}
    for rho in (0.5, 0.9, 1.5):
        rate = rho * seq_rate
        arr = gen.poisson_arrivals(seed, count, rate)
        reqs = rtcdf.make_requests(n, mn, mx, dist, seeds, arr)
        row = {"arrival_rate_per_s": round(rate, 1)}
        for name, fn in (("sequential", rtcdf.rtcdf_serve_sequential),
                         ("server", rtcdf.rtcdf_serve_trace)):
            res, st = fn(cfg(), reqs, count)
            lat = np.array([res[i].done_s - arr[i] for i in range(count)])
            ok = all(res[i].status == 0 for i in range(count))
            row[name] = {"GKeys_s": round(st.total_keys / st.makespan_s / 1e9, 2),
                         "makespan_s": round(st.makespan_s, 4),
                         "p50_latency_ms": round(float(np.percentile(lat, 50)) * 1e3, 3),
                         "p99_latency_ms": round(float(np.percentile(lat, 99)) * 1e3, 3),
                         "all_ok": ok, "launches_batched": int(st.launches_batched),
                         "launches_single": int(st.launches_single),
                         "max_inflight": int(st.max_inflight),
                         "peak_GB": round(st.peak_bytes / 1e9, 2)}
        row["p99_ratio_sequential_vs_server"] = round(
            row["sequential"]["p99_latency_ms"] / max(1e-9, row["server"]["p99_latency_ms"]), 3)
        if rho == 0.5:
            # the previous policy: keys written at admission, large launches on every stream
            res, st = rtcdf.rtcdf_serve_trace(cfg(adaptive=False), reqs, count)
            lat = np.array([res[i].done_s - arr[i] for i in range(count)])
            row["server_admission_writes"] = {
                "p50_latency_ms": round(float(np.percentile(lat, 50)) * 1e3, 3),
                "p99_latency_ms": round(float(np.percentile(lat, 99)) * 1e3, 3),
                "all_ok": all(res[i].status == 0 for i in range(count))}
        out["load"][str(rho)] = row
    main = out["load"]["0.9"]
    out["sequential"], out["server"] = main["sequential"], main["server"]
    out["throughput_ratio_server_vs_sequential"] = round(
        out["server"]["GKeys_s"] / max(1e-9, out["sequential"]["GKeys_s"]), 3)
    out["p99_ratio_sequential_vs_server"] = main["p99_ratio_sequential_vs_server"]
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cub", action="store_true", help="skip the CUB radix-sort comparison")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched-vs-looped comparison")
    ap.add_argument("--batched-segments", type=int, default=4096)
    ap.add_argument("--no-serve", action="store_true", help="skip the serving comparison")
    ap.add_argument("--no-sharded", action="store_true",
                    help="skip the sharded sort (each array split across the ranks)")
    ap.add_argument("--serve-requests", type=int, default=20000)
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--streams", type=int, default=12,
                    help="streams the timed step spreads its independent arrays over")
    ap.add_argument("--no-single", action="store_true", help="skip the n=1e6 single-array config")
    ap.add_argument("--no-large", action="store_true", help="skip the n=1e9 configs")
    ap.add_argument("--preheat-s", type=float, default=0.5,
                    help="seconds of untimed load after warm-up so clocks settle")
    ap.add_argument("--only", default="",
                    help="comma list of R:dist (e.g. 16384:normal) to run a subset of the sweep")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    from paper_2609_00843_gb300 import dist as rdist
    rank, world, local_rank = rdist.rank_env()

    if args.impl == "reference":
        return run_reference(args, rank, world)

    import torch
    torch.cuda.set_device(local_rank)
    dist_on = world > 1
    if dist_on:
        rdist.init("nccl", torch.device("cuda", local_rank))
    barrier = rdist.barrier

    from paper_2609_00843_gb300 import _build
    if rank == 0 or not dist_on:
        _build.build()
    barrier()
    from paper_2609_00843_gb300 import gen, rtcdf

    stream = torch.cuda.Stream()
    sh = stream.cuda_stream
    cases = sweep_cases()
    if args.only:
        keep = {tuple(x.split(":")) for x in args.only.split(",")}
        cases = [c for c in cases if (str(c["R"]), c["dist_name"]) in keep]
        if not cases:
            raise SystemExit(f"--only {args.only} selects no sweep array")
    n = N_SWEEP
    ins, outs = [], []
    with torch.cuda.stream(stream):
        for c in cases:
            x = torch.empty(n, dtype=torch.int32, device="cuda")
            seed = rdist.rank_seed(c["seed"], rank)
            gen.keys_device(x.data_ptr(), n, MIN_SWEEP, c["R"], c["dist"], seed, stream=sh)
            ins.append(x)
            outs.append(torch.empty(n, dtype=torch.int32, device="cuda"))
    stream.synchronize()

    R_max = max(SWEEP_R)
    ws_bytes = rtcdf.rtcdf_workspace_size(R_max)
    ws = torch.zeros(ws_bytes // 4 + 64, dtype=torch.int32, device="cuda")
    # Four stage events per sort per timed step, so the timed region has no
    # host synchronisation: before hist, after hist, after scan, after fill.
    nsteps = args.steps
    evs = [[[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in cases]
           for _ in range(nsteps)]
    for per_step in evs:
        for quad in per_step:
            for e in quad:
                e.record(stream)  # creates the underlying cudaEvent_t
    stream.synchronize()
    dbgs = []
    for per_step in evs:
        row = []
        for quad in per_step:
            d = rtcdf.Debug()
            for j in range(4):
                d.stage_events[j] = quad[j].cuda_event
            row.append(d)
        dbgs.append(row)

    def step(dbg_row):
        for i, c in enumerate(cases):
            rc = rtcdf.rtcdf_sort_ex(ins[i].data_ptr(), outs[i].data_ptr(), n, MIN_SWEEP,
                                     MIN_SWEEP + c["R"], None, ws.data_ptr(), ws_bytes,
                                     dbg_row[i] if dbg_row is not None else None, sh)
            if rc != rtcdf.OK:
                raise rtcdf.RtcdfError(rc, "rtcdf_sort_ex")

    # The step's arrays are independent: the timed step sorts them on
    # `--streams` streams (round robin, one workspace each), so one array's
    # latency-bound phases overlap another's memory-bound ones.
    n_streams = max(1, args.streams)
    k_streams = [stream] + [torch.cuda.Stream() for _ in range(n_streams - 1)]
    k_ws = [ws] + [torch.zeros(ws_bytes // 4 + 64, dtype=torch.int32, device="cuda")
                   for _ in range(n_streams - 1)]
    join_ev = [torch.cuda.Event() for _ in range(n_streams)]

    def step_streams():
        start = torch.cuda.Event()
        start.record(stream)
        for k in range(1, n_streams):
            k_streams[k].wait_event(start)
        for i, c in enumerate(cases):
            k = i % n_streams
            rc = rtcdf.rtcdf_sort_ex(ins[i].data_ptr(), outs[i].data_ptr(), n, MIN_SWEEP,
                                     MIN_SWEEP + c["R"], None, k_ws[k].data_ptr(), ws_bytes, None,
                                     k_streams[k].cuda_stream)
            if rc != rtcdf.OK:
                raise rtcdf.RtcdfError(rc, "rtcdf_sort_ex")
        for k in range(1, n_streams):
            join_ev[k].record(k_streams[k])
            stream.wait_event(join_ev[k])

    # Warm-up: W steps plus about half a second of load so clocks settle.
    for _ in range(args.warmup):
        step(None)
        step_streams()
    torch.cuda.synchronize()
    t_end = time.time() + args.preheat_s
    while time.time() < t_end:
        step_streams()
        torch.cuda.synchronize()
    rc, bits = rtcdf.rtcdf_ws_status_get(ws.data_ptr(), sh)
    if rc != rtcdf.OK:
        raise rtcdf.RtcdfError(rc, "device status after warm-up")

    sampler = ClockSampler(local_rank)
    sampler.start()
    time.sleep(0.3)
    # Timed region: K steps back to back, no events between the kernels (an
    # event between two kernels would stop the programmatic dependent launch
    # that overlaps their launch latency).
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.synchronize()
    t0.record(stream)
    for k in range(nsteps):
        step_streams()
    t1.record(stream)
    torch.cuda.synchronize()
    barrier()
    total_ms = t0.elapsed_time(t1)
    # The same steps on one stream, for comparison.
    s0 = torch.cuda.Event(enable_timing=True)
    s1 = torch.cuda.Event(enable_timing=True)
    s0.record(stream)
    for k in range(nsteps):
        step(None)
    s1.record(stream)
    torch.cuda.synchronize()
    serial_ms = s0.elapsed_time(s1) / nsteps
    # Per array: K back-to-back sorts of the same array, uninstrumented, and
    # the paper's protocol (3 runs x 30 event-timed sorts after 10 warm-ups,
    # median of medians).
    solo_ms, proto_ms = [], []
    for i, c in enumerate(cases):
        def sort_once(i=i, c=c):
            rc = rtcdf.rtcdf_sort_ex(ins[i].data_ptr(), outs[i].data_ptr(), n, MIN_SWEEP,
                                     MIN_SWEEP + c["R"], None, ws.data_ptr(), ws_bytes, None, sh)
            if rc != rtcdf.OK:
                raise rtcdf.RtcdfError(rc, "rtcdf_sort_ex")
        a0 = torch.cuda.Event(enable_timing=True)
        a1 = torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        for k in range(nsteps):
            sort_once()
        a1.record(stream)
        stream.synchronize()
        solo_ms.append(a0.elapsed_time(a1) / nsteps)
        proto_ms.append(paper_protocol_ms(sort_once, stream))
    # Instrumented region: the same K steps with CUDA events on the launching
    # stream before and after every kernel, for the per-kernel durations.
    for k in range(nsteps):
        step(dbgs[k])
    torch.cuda.synchronize()
    time.sleep(0.1)
    clocks = sampler.stop()
    total_ms = rdist.max_over_ranks(total_ms, device="cuda")
    rc, bits = rtcdf.rtcdf_ws_status_get(ws.data_ptr(), sh)
    if rc != rtcdf.OK:
        raise rtcdf.RtcdfError(rc, "device status after timed region")

    stage_ms = [[0.0, 0.0, 0.0] for _ in cases]
    per_case_ms = [0.0 for _ in cases]
    for k in range(nsteps):
        for i in range(len(cases)):
            e = evs[k][i]
            for j in range(3):
                stage_ms[i][j] += e[j].elapsed_time(e[j + 1])
            per_case_ms[i] += e[0].elapsed_time(e[3])
    sort_ms = total_ms / nsteps  # whole step, max over ranks
    value = rdist.job_throughput(n * len(cases), world, sort_ms) / 1e9

    hbm, peak_kind = peaks()
    per_config = []
    for i, c in enumerate(cases):
        ms = solo_ms[i]
        pp = rtcdf.rtcdf_plan(n, c["R"])
        per_config.append({"R": c["R"], "dist": c["dist_name"], "ms": round(ms, 5),
                           "GKeys_s": round(n / (ms * 1e-3) / 1e9, 2),
                           "frac_8n_roofline": round(8 * n / (ms * 1e-3) / 1e9 / hbm, 4),
                           "frac_8n_spec": round(8 * n / (ms * 1e-3) / 1e9 / SPEC_HBM_GBS, 4),
                           "ms_paper_protocol": round(proto_ms[i], 5),
                           "launch": {"T": pp.tile_width, "m": -(-c["R"] // pp.tile_width),
                                      "hist_ctas": pp.hist_ctas_per_tile * -(-c["R"] // pp.tile_width),
                                      "hist_threads": pp.hist_threads, "fill_ctas": pp.fill_ctas,
                                      "fill_threads": pp.fill_threads},
                           "ms_instrumented": round(per_case_ms[i] / nsteps, 5),
                           "hist_ms": round(stage_ms[i][0] / nsteps, 5),
                           "scan_ms": round(stage_ms[i][1] / nsteps, 5),
                           "fill_ms": round(stage_ms[i][2] / nsteps, 5)})
    hist_total = sum(s[0] for s in stage_ms)
    fill_total = sum(s[2] for s in stage_ms)
    launches = len(cases) * nsteps
    if hist_total >= fill_total:
        kname, ktime = "hist_kernel", hist_total
        ksrc = ["paper_2609_00843_gb300/csrc/hist.cu", "paper_2609_00843_gb300/csrc/rtcdf_internal.h"]
    else:
        kname, ktime = "fill_kernel", fill_total
        ksrc = ["paper_2609_00843_gb300/csrc/fill.cu", "paper_2609_00843_gb300/csrc/rtcdf_internal.h"]
    avg_launch_s = ktime / launches * 1e-3
    achieved = 4 * n / avg_launch_s / 1e9  # algorithmic: 4n bytes read (hist) or written (fill)
    # The same fraction split by the number of range tiles m of the launch
    # (one tile streams the input once; m > 1 tiles re-read it from L2).
    j = 0 if kname == "hist_kernel" else 2
    by_tiles = {}
    for i, c in enumerate(cases):
        m = -(-c["R"] // rtcdf.rtcdf_plan(n, c["R"]).tile_width)
        by_tiles.setdefault(m, []).append(stage_ms[i][j] / nsteps)
    by_tiles = {str(m): {"launches_per_step": len(t),
                         "frac": round(4 * n / (sum(t) / len(t) * 1e-3) / 1e9 / hbm, 4)}
                for m, t in sorted(by_tiles.items())}
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": hbm, "unit": "GB/s",
                "frac": round(achieved / hbm, 4),
                "traffic": traffic_for(kname, ksrc),
                "kernel": kname, "peak_kind": f"{peak_kind} hbm_gbs (copy)",
                "algorithmic_bytes_per_launch": 4 * n,
                "by_range_tiles": by_tiles}
    whole = {"achieved_8n_GBs": round(8 * n * len(cases) / (sort_ms * 1e-3) / 1e9, 1)}
    whole["frac_8n_roofline"] = round(whole["achieved_8n_GBs"] / hbm, 4)
    whole["frac_8n_spec"] = round(whole["achieved_8n_GBs"] / SPEC_HBM_GBS, 4)
    whole["spec_GBs"] = SPEC_HBM_GBS

    line = {
        "metric": METRIC,
        "value": round(value, 2), "unit": "GKeys/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(sort_ms, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n_per_array": n, "arrays": len(cases),
                   "l2": "inputs larger than L2 (400 MB per array), no flush",
                   "streams": n_streams,
                   "parallelism": f"replicas x{world} (independent arrays per GPU)"},
        "one_stream": {"ms_per_step": round(serial_ms, 4),
                       "GKeys_s": round(n * len(cases) / (serial_ms * 1e-3) / 1e9, 2)},
        "roofline": roofline,
        "whole_sort_roofline": whole,
        "per_config": per_config,
        "clocks": clocks,
        "gpu_launches": 3 * len(cases) * args.steps,
        "timed_region_ms": round(total_ms, 3),
    }

    # End to end through the C ABI with host buffers (rtcdf_sort_host): pinned
    # host input -> chunked upload overlapped with the histogram -> scan and
    # output -> download overlapped with the next array's upload -> host.
    if not args.no_e2e:
        pin_in = [torch.empty(n, dtype=torch.int32, pin_memory=True) for _ in cases]
        for p, x in zip(pin_in, ins):
            p.copy_(x.cpu())
        pin_out = [torch.empty(n, dtype=torch.int32, pin_memory=True) for _ in range(2)]

        def e2e_step():
            for i, c in enumerate(cases):
                rc = rtcdf.rtcdf_sort_host(pin_in[i].data_ptr(), pin_out[i % 2].data_ptr(), n,
                                           MIN_SWEEP, MIN_SWEEP + c["R"], sh)
                if rc != rtcdf.OK:
                    raise rtcdf.RtcdfError(rc, "rtcdf_sort_host")

        e2e_step()
        stream.synchronize()
        # Steps run back to back (each step's uploads overlap the previous
        # step's downloads); an event after each step gives per-step times, and
        # the median is reported (the host link is shared with other tenants of
        # the machine, so single steps can be slowed by traffic not ours).
        evs_e = [torch.cuda.Event(enable_timing=True) for _ in range(args.e2e_steps + 1)]
        evs_e[0].record(stream)
        for k in range(args.e2e_steps):
            e2e_step()
            evs_e[k + 1].record(stream)
        stream.synchronize()
        step_ms = [evs_e[k].elapsed_time(evs_e[k + 1]) for k in range(args.e2e_steps)]
        e_ms = rdist.max_over_ranks(statistics.median(step_ms), device="cuda")
        e_val = n * len(cases) * world / (e_ms * 1e-3) / 1e9
        line["e2e"] = {"value": round(e_val, 3),
                       "unit": "GKeys/s", "h2d_bytes_per_step": 4 * n * len(cases),
                       "d2h_bytes_per_step": 4 * n * len(cases), "ms_per_step": round(e_ms, 3),
                       "step_ms_min_max": [round(min(step_ms), 3), round(max(step_ms), 3)]}
        # The host link's bound: one array's upload and download at the same
        # time (plain copies of the same 400 MB buffers, both directions).
        d_tmp = torch.empty(n, dtype=torch.int32, device="cuda")
        s_up, s_dn = torch.cuda.Stream(), torch.cuda.Stream()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        for rep in range(3):
            torch.cuda.synchronize()
            ev[0].record(s_up)
            s_dn.wait_event(ev[0])
            with torch.cuda.stream(s_up):
                d_tmp.copy_(pin_in[0], non_blocking=True)
            with torch.cuda.stream(s_dn):
                pin_out[0].copy_(outs[0], non_blocking=True)
            s_up.wait_stream(s_dn)
            ev[1].record(s_up)
            torch.cuda.synchronize()
        link_ms = ev[0].elapsed_time(ev[1])
        bound = n / (link_ms * 1e-3) / 1e9
        line["e2e"]["link_bound_GKeys_s"] = round(bound, 2)
        line["e2e"]["link_bidir_GBs"] = round(8 * n / (link_ms * 1e-3) / 1e9, 1)
        line["e2e"]["frac_of_link_bound"] = round(e_val / world / bound, 4)
        del d_tmp
        del pin_in, pin_out

    # Every array split across the job's ranks (one all-reduce of the counts).
    if not args.no_sharded:
        line["sharded"] = sharded_comparison(cases, outs if world == 1 else [], n, rank, world, stream,
                                             max(3, min(args.steps, 10)))

    # On-GPU comparison: CUB DeviceRadixSort restricted to bits [0, ceil(log2 R))
    # on keys normalised to uint32 (normalise / denormalise timed apart).
    if not args.no_cub and rank == 0:
        line["cub_comparison"] = cub_comparison(cases, ins, outs, n, stream, nsteps, solo_ms)

    if not args.no_single and rank == 0:
        line["single"] = single_config(stream)

    if not args.no_batched and rank == 0:
        line["batched"] = batched_comparison(args, stream, args.batched_segments)

    if not args.no_serve and rank == 0:
        line["serve"] = serving_comparison(args.serve_requests)


    if rank == 0 and not args.no_cpu_baseline:
        host = [x.cpu().numpy() for x in ins]
        line["cpu_baseline"] = cpu_baseline_sweep(host, cases)

    if not args.no_large and rank == 0:
        # the sweep arrays are no longer needed: make room for 8 GB
        del ins[:], outs[:]
        torch.cuda.empty_cache()
        line["large"] = large_config(stream)

    if rank == 0:
        print(json.dumps(line), flush=True)
    rdist.finish()
    return 0


if __name__ == "__main__":
    sys.exit(main())
