// Host side of the C ABI (include/rtcdf.h): argument checks, launch planning,
// workspace management and the three-kernel pipeline of Algorithm 4.
//
//   1. hist  -- Algorithm 5 for all m tiles in one launch
//   2. scan  -- local CDFs + tile offsets (Algorithm 6) as one lookback scan
//   3. fill  -- Algorithm 7 for all tiles in one launch
//
// Unlike the paper's host driver there is no device-to-host copy of the tile
// offsets and no per-tile launch loop: every launch size is known from (n, R)
// alone, so a sort is three stream-ordered launches with no host
// synchronisation and can be captured in a CUDA graph.
#include <algorithm>
#include <cstring>
#include <map>
#include <mutex>
#include <utility>

#include "../../include/rtcdf.h"
#include "rtcdf_internal.h"

using namespace rtcdf;

namespace {

struct DeviceInfo {
    int sms = 0;
    size_t smem_optin = 0;
};

std::mutex g_mu;
std::map<int, DeviceInfo> g_dev;

rtcdf_status device_info(DeviceInfo *out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return RTCDF_ERR_CUDA;
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_dev.find(dev);
    if (it == g_dev.end()) {
        DeviceInfo d;
        int v = 0;
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            return RTCDF_ERR_CUDA;
        d.sms = v;
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
            return RTCDF_ERR_CUDA;
        d.smem_optin = (size_t)v;
        try {
            it = g_dev.emplace(dev, d).first;
        } catch (...) {
            return RTCDF_ERR_NO_MEMORY;
        }
    }
    *out = it->second;
    return RTCDF_OK;
}

struct Plan {
    uint32_t R, T, m, g;
    int hist_threads;
    size_t hist_smem;
    bool streaming;
    uint32_t head;
    uint64_t nvec;
    int fill_threads;
    uint32_t fill_ctas;
    uint64_t fill_chunk;
};

rtcdf_status check_range(int64_t minVal, int64_t maxVal, uint32_t *R) {
    if (minVal < INT32_MIN || maxVal > (int64_t)1 << 31) return RTCDF_ERR_RANGE;
    if (maxVal <= minVal) return RTCDF_ERR_RANGE;
    int64_t r = maxVal - minVal;
    if (r > RTCDF_MAX_R) return RTCDF_ERR_RANGE;
    *R = (uint32_t)r;
    return RTCDF_OK;
}

// Choose the launch shape (Section 3.3): tile width T from shared memory, CTAs
// per tile from occupancy, output CTAs from n.
rtcdf_status make_plan_with(uint64_t n, uint32_t R, uintptr_t in_addr, uintptr_t out_addr,
                            const rtcdf_params *p, Plan *pl) {
    DeviceInfo dev;
    rtcdf_status st = device_info(&dev);
    if (st) return st;
    rtcdf_params q;
    memset(&q, 0, sizeof(q));
    if (p) q = *p;

    pl->R = R;
    pl->hist_threads = q.hist_threads ? q.hist_threads : 1024;
    if (pl->hist_threads != 256 && pl->hist_threads != 512 && pl->hist_threads != 1024)
        return RTCDF_ERR_INVALID_ARG;
    // Largest tile whose 32-bit histogram fits the opt-in shared memory.
    const uint32_t t_max = (uint32_t)(dev.smem_optin / 4) & ~1023u;
    uint32_t T = q.tile_width > 0 ? (uint32_t)q.tile_width : 0;
    if (T == 0) {
        // Fewest tiles that fit, then equal widths (rounded up to 1024 values):
        // every tile costs a full input scan, and balanced tiles leave more
        // shared memory per SM for L1.
        const uint32_t m = (R + t_max - 1) / t_max;
        T = m == 1 ? R : std::min(t_max, ((R + m - 1) / m + 1023) & ~1023u);
    }
    if (T > t_max) return RTCDF_ERR_INVALID_ARG;
    if (T > R) T = R;
    pl->T = T;
    pl->m = (R + T - 1) / T;
    pl->streaming = (pl->m == 1);
    // Several tiles: one more word after the tile (out-of-tile keys counted
    // into it, kept to 16 bytes).
    pl->hist_smem = (size_t)T * 4 + (pl->streaming ? 0 : 16);

    // Input split: unaligned head elements, 16-byte vectors, ragged tail.
    uint32_t head_in = (uint32_t)(((16 - (in_addr & 15)) & 15) / 4);
    if (head_in > n) head_in = (uint32_t)n;
    pl->head = head_in;
    pl->nvec = (n - head_in) / 4;

    int occ = 0;
    try {  // the occupancy cache may need memory for a new entry
        if (hist_max_ctas_per_sm(pl->hist_threads, pl->hist_smem, pl->streaming, &occ) != cudaSuccess)
            return RTCDF_ERR_CUDA;
    } catch (...) {
        return RTCDF_ERR_NO_MEMORY;
    }
    if (occ < 1) return RTCDF_ERR_INVALID_ARG;
    // g_hist = min(max(1, floor(a_hist * S / m)), ceil(n / (16 * threads)))
    uint64_t g = std::max<uint64_t>(1, (uint64_t)occ * dev.sms / pl->m);
    uint64_t g_n = std::max<uint64_t>(1, (n + 16ull * pl->hist_threads - 1) / (16ull * pl->hist_threads));
    g = std::min(g, g_n);
    if (q.hist_ctas_per_tile > 0) g = (uint64_t)q.hist_ctas_per_tile;
    pl->g = (uint32_t)g;

    // Output: contiguous position ranges, CTA boundaries on 16-byte vectors of `out`.
    // Not clamped to n: positions below head_out are written one by one, and
    // the vector frame must stay 16-byte aligned.
    const uint32_t head_out = (uint32_t)(((16 - (out_addr & 15)) & 15) / 4);
    pl->fill_threads = q.fill_threads ? q.fill_threads : 512;
    if (pl->fill_threads != 256 && pl->fill_threads != 512 && pl->fill_threads != 1024)
        return RTCDF_ERR_INVALID_ARG;
    // Many more CTAs than fit at once (about 32K positions each, at least four
    // waves' worth): the block scheduler then balances CTAs whose positions
    // cross many short runs against CTAs inside one long run.
    uint64_t body = n > head_out ? n - head_out : 0;
    uint64_t chunk;
    if (q.fill_chunk < 0 || q.fill_ctas < 0) return RTCDF_ERR_INVALID_ARG;
    if (q.fill_chunk > 0) {
        chunk = std::max<uint64_t>((uint64_t)q.fill_chunk,
                                   (body + kMaxFillCtas - 1) / kMaxFillCtas);
        chunk = std::max<uint64_t>(chunk, 4 * (uint64_t)pl->fill_threads);
    } else {
        uint64_t want = q.fill_ctas > 0 ? (uint64_t)q.fill_ctas
                                        : std::max<uint64_t>((uint64_t)dev.sms * 4, body / 32768);
        want = std::min<uint64_t>(want, kMaxFillCtas);
        chunk = std::max<uint64_t>(4 * (uint64_t)pl->fill_threads, (body + want - 1) / want);
    }
    chunk = (chunk + 3) / 4 * 4;
    pl->fill_chunk = chunk;
    pl->fill_ctas = (uint32_t)(1 + (n > head_out ? (n - head_out - 1) / chunk : 0));
    if (pl->fill_ctas > kMaxFillCtas) return RTCDF_ERR_INVALID_ARG;
    pl->head = head_in;
    return RTCDF_OK;
}

// Explicit parameters are used as given; without them the tuning table is
// tried first and the built-in rules cover what it lacks (or what does not fit
// this device).
rtcdf_status make_plan(uint64_t n, uint32_t R, uintptr_t in_addr, uintptr_t out_addr,
                       const rtcdf_params *p, Plan *pl) {
    if (p) return make_plan_with(n, R, in_addr, out_addr, p, pl);
    rtcdf_params t;
    if (tune_lookup(n, R, &t) && make_plan_with(n, R, in_addr, out_addr, &t, pl) == RTCDF_OK)
        return RTCDF_OK;
    return make_plan_with(n, R, in_addr, out_addr, nullptr, pl);
}

bool overlaps(const void *a, const void *b, uint64_t n) {
    uintptr_t x = (uintptr_t)a, y = (uintptr_t)b;
    uint64_t bytes = n * 4;
    return x < y + bytes && y < x + bytes;
}

rtcdf_status check_args(const int32_t *in, int32_t *out, uint64_t n) {
    if (n >= (1ull << 32)) return RTCDF_ERR_INVALID_ARG;
    if (!in || !out) return RTCDF_ERR_INVALID_ARG;
    if (((uintptr_t)in & 3) || ((uintptr_t)out & 3)) return RTCDF_ERR_INVALID_ARG;
    if ((const void *)in != (const void *)out && overlaps(in, out, n)) return RTCDF_ERR_INVALID_ARG;
    return RTCDF_OK;
}

// Algorithm 5 (all tiles) into the workspace's H.  H accumulates, so several
// calls over slices of one array add up to the array's histogram.
rtcdf_status hist_phase(const int32_t *in, uint64_t n, int64_t minVal, uint32_t R, const Plan &pl,
                        const WsLayout &L, char *base, cudaStream_t s) {
    HistArgs h;
    h.in = in; h.n = n; h.nvec = pl.nvec; h.head = pl.head;
    h.min_u = (uint32_t)(int32_t)minVal; h.R = R; h.T = pl.T; h.m = pl.m; h.g = pl.g;
    h.H = (uint32_t *)(base + L.hist);
    h.ctl = (Ctl *)(base + L.ctl);
    if (launch_hist(h, pl.hist_threads, pl.hist_smem, pl.streaming, s) != cudaSuccess)
        return RTCDF_ERR_CUDA;
    return RTCDF_OK;
}

// Local CDFs + offsets (Algorithm 6) and output generation (Algorithm 7)
// for an n-key array whose histogram is in H: positions [pos_base, pos_end)
// of the sorted array are written, position p to out[p - pos_base] (the
// plan's output CTAs are sized for pos_end - pos_base positions).
rtcdf_status finish_phase(int32_t *out, uint64_t n, int64_t minVal, uint32_t R, const Plan &pl,
                          const WsLayout &L, char *base, const rtcdf_debug *dbg,
                          cudaEvent_t ev_scan, cudaEvent_t ev_fill, cudaStream_t s,
                          uint64_t pos_base, uint64_t pos_end) {
    Ctl *ctl = (Ctl *)(base + L.ctl);
    uint64_t *state = (uint64_t *)(base + L.scan_state);
    uint32_t *run_end = (uint32_t *)(base + L.run_end);
    int32_t *run_val = (int32_t *)(base + L.run_val);
    uint32_t *start_run = (uint32_t *)(base + L.start_run);
    const uint32_t head_out = (uint32_t)(((16 - ((uintptr_t)out & 15)) & 15) / 4);
    ScanArgs sc;
    sc.H = (uint32_t *)(base + L.hist); sc.state = state; sc.ctl = ctl; sc.run_end = run_end;
    sc.run_val = run_val; sc.start_run = start_run; sc.n = n; sc.fill_chunk = pl.fill_chunk;
    sc.head = head_out; sc.fill_ctas = pl.fill_ctas; sc.R = R; sc.T = pl.T; sc.chunks = L.scan_chunks;
    sc.pos_base = (uint32_t)pos_base; sc.pos_end = (uint32_t)pos_end;
    sc.minVal = (int32_t)minVal;
    sc.dbg_hist = dbg ? dbg->tile_hist : nullptr;
    sc.dbg_cdf = dbg ? dbg->cdf : nullptr;
    sc.dbg_offset = dbg ? dbg->tile_offset : nullptr;
    if (launch_scan(sc, s) != cudaSuccess) return RTCDF_ERR_CUDA;
    if (ev_scan && cudaEventRecord(ev_scan, s) != cudaSuccess) return RTCDF_ERR_CUDA;

    FillArgs f;
    f.out = out; f.n = pos_end; f.pos_base = (uint32_t)pos_base; f.fill_chunk = pl.fill_chunk;
    f.head = head_out;
    f.fill_ctas = pl.fill_ctas; f.run_end = run_end; f.run_val = run_val;
    f.start_run = start_run; f.ctl = ctl; f.scan_state = state; f.scan_chunks = L.scan_chunks;
    f.R = R;
    if (launch_fill(f, pl.fill_threads, s) != cudaSuccess) return RTCDF_ERR_CUDA;
    if (ev_fill && cudaEventRecord(ev_fill, s) != cudaSuccess) return RTCDF_ERR_CUDA;
    return RTCDF_OK;
}

rtcdf_status run_pipeline(const int32_t *in, int32_t *out, uint64_t n, int64_t minVal,
                          uint32_t R, const Plan &pl, void *ws, size_t ws_bytes,
                          const rtcdf_debug *dbg, cudaStream_t s) {
    const WsLayout L = ws_layout(R, ws_bytes);
    char *base = (char *)ws;
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    if (dbg)
        for (int i = 0; i < 4; i++) ev[i] = (cudaEvent_t)dbg->stage_events[i];
    if (ev[0] && cudaEventRecord(ev[0], s) != cudaSuccess) return RTCDF_ERR_CUDA;
    rtcdf_status st = hist_phase(in, n, minVal, R, pl, L, base, s);
    if (st) return st;
    if (ev[1] && cudaEventRecord(ev[1], s) != cudaSuccess) return RTCDF_ERR_CUDA;
    return finish_phase(out, n, minVal, R, pl, L, base, dbg, ev[2], ev[3], s, 0, n);
}

// ---------------------------------------------------------------- workspace cache
struct CachedWs {
    void *ptr = nullptr;
    size_t bytes = 0;
};
std::map<std::pair<int, cudaStream_t>, CachedWs> g_ws;

rtcdf_status cached_workspace(cudaStream_t s, size_t need, void **ptr, size_t *bytes) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return RTCDF_ERR_CUDA;
    std::lock_guard<std::mutex> lk(g_mu);
    CachedWs *wp = nullptr;
    try {
        wp = &g_ws[std::make_pair(dev, s)];
    } catch (...) {
        return RTCDF_ERR_NO_MEMORY;
    }
    CachedWs &w = *wp;
    if (w.bytes < need) {
        cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(s, &cap) != cudaSuccess) return RTCDF_ERR_CUDA;
        if (cap != cudaStreamCaptureStatusNone) return RTCDF_ERR_NO_MEMORY;
        size_t grow = std::max(need, w.bytes * 2);
        void *p = nullptr;
        if (cudaMallocAsync(&p, grow, s) != cudaSuccess) return RTCDF_ERR_NO_MEMORY;
        if (cudaMemsetAsync(p, 0, grow, s) != cudaSuccess) {
            cudaFreeAsync(p, s);
            return RTCDF_ERR_CUDA;
        }
        void *old = w.ptr;
        w.ptr = p;
        w.bytes = grow;
        if (old && cudaFreeAsync(old, s) != cudaSuccess) return RTCDF_ERR_CUDA;
    }
    *ptr = w.ptr;
    *bytes = w.bytes;
    return RTCDF_OK;
}

// The status code for a status word: a wait that ran out makes every other
// finding unreliable, so it comes first.
rtcdf_status status_of_bits(uint32_t v) {
    if (v & kDevTimeout) return RTCDF_ERR_TIMEOUT;
    if (v & kDevBadSegment) return RTCDF_ERR_INVALID_ARG;
    if (v & kDevKeyOutOfRange) return RTCDF_ERR_KEY_OUT_OF_RANGE;
    return RTCDF_OK;
}

rtcdf_status read_status(void *ws, cudaStream_t s, int32_t *out) {
    uint32_t v = 0;
    Ctl *ctl = (Ctl *)ws;
    if (cudaMemcpyAsync(&v, &ctl->status, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess) return RTCDF_ERR_CUDA;
    if (cudaMemsetAsync(&ctl->status, 0, 4, s) != cudaSuccess) return RTCDF_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return RTCDF_ERR_CUDA;
    if (out) *out = (int32_t)v;
    return status_of_bits(v);
}

}  // namespace

namespace rtcdf {

// Sort in a workspace whose previous contents are unknown: the regions that
// must start at zero (control block, lookback state, histogram) are cleared
// on `s` first.  Used by rtcdf_sort_static.
rtcdf_status sort_with_workspace(const int32_t *in, int32_t *out, uint64_t n, int64_t minVal,
                                 int64_t maxVal, void *ws, size_t ws_bytes, cudaStream_t s) {
    uint32_t R = 0;
    rtcdf_status st = check_range(minVal, maxVal, &R);
    if (st) return st;
    if (n == 0) return RTCDF_OK;
    st = check_args(in, out, n);
    if (st) return st;
    if (!ws || ws_bytes < ws_required(R)) return RTCDF_ERR_NO_MEMORY;
    const WsLayout L = ws_layout(R, ws_bytes);
    if (cudaMemsetAsync(ws, 0, L.zero_bytes, s) != cudaSuccess) return RTCDF_ERR_CUDA;
    Plan pl;
    st = make_plan(n, R, (uintptr_t)in, (uintptr_t)out, nullptr, &pl);
    if (st) return st;
    return run_pipeline(in, out, n, minVal, R, pl, ws, ws_bytes, nullptr, s);
}

// The two halves of a sort, for rtcdf_sort_host: histogram of a slice (may be
// called once per uploaded chunk), then scan + output for the whole array.
rtcdf_status host_pipeline_hist(const int32_t *in, uint64_t n, int64_t minVal, uint32_t R, void *ws,
                                size_t ws_bytes, cudaStream_t s) {
    if (n == 0) return RTCDF_OK;
    Plan pl;
    rtcdf_status st = make_plan(n, R, (uintptr_t)in, 0, nullptr, &pl);
    if (st) return st;
    return hist_phase(in, n, minVal, R, pl, ws_layout(R, ws_bytes), (char *)ws, s);
}

rtcdf_status host_pipeline_finish(int32_t *out, uint64_t n, int64_t minVal, uint32_t R, void *ws,
                                  size_t ws_bytes, cudaStream_t s) {
    Plan pl;
    rtcdf_status st = make_plan(n, R, 0, (uintptr_t)out, nullptr, &pl);
    if (st) return st;
    return finish_phase(out, n, minVal, R, pl, ws_layout(R, ws_bytes), (char *)ws, nullptr,
                        nullptr, nullptr, s, 0, n);
}

}  // namespace rtcdf

extern "C" {

const char *rtcdf_version(void) { return "rtcdf 0.1 (sm_103a)"; }

const char *rtcdf_status_str(rtcdf_status s) {
    switch (s) {
        case RTCDF_OK: return "ok";
        case RTCDF_ERR_INVALID_ARG: return "invalid argument";
        case RTCDF_ERR_RANGE: return "range size outside [1, RTCDF_MAX_R] or outside int32";
        case RTCDF_ERR_KEY_OUT_OF_RANGE: return "a key lies outside [minVal, maxVal)";
        case RTCDF_ERR_CUDA: return "CUDA runtime error";
        case RTCDF_ERR_NO_MEMORY: return "workspace allocation failed or workspace too small";
        case RTCDF_ERR_TIMEOUT: return "a bounded device wait gave up";
    }
    return "unknown status";
}

rtcdf_status rtcdf_workspace_size(int64_t R, size_t *bytes) {
    if (!bytes) return RTCDF_ERR_INVALID_ARG;
    if (R <= 0 || R > RTCDF_MAX_R) return RTCDF_ERR_RANGE;
    *bytes = ws_required((uint64_t)R);
    return RTCDF_OK;
}

rtcdf_status rtcdf_plan(uint64_t n, int64_t R, rtcdf_params *params) {
    if (!params) return RTCDF_ERR_INVALID_ARG;
    if (R <= 0 || R > RTCDF_MAX_R) return RTCDF_ERR_RANGE;
    Plan pl;
    rtcdf_status st = make_plan(n, (uint32_t)R, 0, 0, nullptr, &pl);
    if (st) return st;
    memset(params, 0, sizeof(*params));
    params->tile_width = (int32_t)pl.T;
    params->hist_ctas_per_tile = (int32_t)pl.g;
    params->hist_threads = pl.hist_threads;
    params->fill_ctas = (int32_t)pl.fill_ctas;
    params->fill_threads = pl.fill_threads;
    params->fill_chunk = (int32_t)std::min<uint64_t>(pl.fill_chunk, INT32_MAX);
    return RTCDF_OK;
}

rtcdf_status rtcdf_sort_ex(const int32_t *in, int32_t *out, uint64_t n, int64_t minVal,
                           int64_t maxVal, const rtcdf_params *params, void *workspace,
                           size_t ws_bytes, const rtcdf_debug *debug, rtcdf_stream_t stream) {
    uint32_t R = 0;
    rtcdf_status st = check_range(minVal, maxVal, &R);
    if (st) return st;
    if (n == 0) return RTCDF_OK;
    st = check_args(in, out, n);
    if (st) return st;
    if (!workspace || ((uintptr_t)workspace & 255)) return RTCDF_ERR_INVALID_ARG;
    if (ws_bytes < ws_required(R)) return RTCDF_ERR_NO_MEMORY;
    Plan pl;
    st = make_plan(n, R, (uintptr_t)in, (uintptr_t)out, params, &pl);
    if (st) return st;
    return run_pipeline(in, out, n, minVal, R, pl, workspace, ws_bytes, debug,
                        (cudaStream_t)stream);
}

rtcdf_status rtcdf_sort_ws(const int32_t *in, int32_t *out, uint64_t n, int64_t minVal,
                           int64_t maxVal, void *workspace, size_t ws_bytes,
                           rtcdf_stream_t stream) {
    return rtcdf_sort_ex(in, out, n, minVal, maxVal, nullptr, workspace, ws_bytes, nullptr, stream);
}

rtcdf_status rtcdf_reserve(int64_t max_R, rtcdf_stream_t stream) {
    if (max_R <= 0 || max_R > RTCDF_MAX_R) return RTCDF_ERR_RANGE;
    void *ws = nullptr;
    size_t bytes = 0;
    return cached_workspace((cudaStream_t)stream, ws_required((uint64_t)max_R), &ws, &bytes);
}

rtcdf_status rtcdf_sort(const int32_t *in, int32_t *out, uint64_t n, int64_t minVal,
                        int64_t maxVal, rtcdf_stream_t stream) {
    uint32_t R = 0;
    rtcdf_status st = check_range(minVal, maxVal, &R);
    if (st) return st;
    if (n == 0) return RTCDF_OK;
    st = check_args(in, out, n);
    if (st) return st;
    void *ws = nullptr;
    size_t ws_bytes = 0;
    st = cached_workspace((cudaStream_t)stream, ws_required(R), &ws, &ws_bytes);
    if (st) return st;
    Plan pl;
    st = make_plan(n, R, (uintptr_t)in, (uintptr_t)out, nullptr, &pl);
    if (st) return st;
    return run_pipeline(in, out, n, minVal, R, pl, ws, ws_bytes, nullptr, (cudaStream_t)stream);
}

rtcdf_status rtcdf_hist_accumulate(const int32_t *in, uint64_t n, int64_t minVal, int64_t maxVal,
                                   uint32_t *counts, rtcdf_stream_t stream) {
    uint32_t R = 0;
    rtcdf_status st = check_range(minVal, maxVal, &R);
    if (st) return st;
    if (!counts || ((uintptr_t)counts & 3)) return RTCDF_ERR_INVALID_ARG;
    if (n == 0) return RTCDF_OK;
    if (n >= (1ull << 32) || !in || ((uintptr_t)in & 3)) return RTCDF_ERR_INVALID_ARG;
    {
        const uintptr_t x = (uintptr_t)in, y = (uintptr_t)counts;
        if (x < y + (uint64_t)R * 4 && y < x + n * 4) return RTCDF_ERR_INVALID_ARG;
    }
    Plan pl;
    st = make_plan(n, R, (uintptr_t)in, 0, nullptr, &pl);
    if (st) return st;
    // Algorithm 5 for every tile, added straight into the caller's counts.
    HistArgs h;
    h.in = in; h.n = n; h.nvec = pl.nvec; h.head = pl.head;
    h.min_u = (uint32_t)(int32_t)minVal; h.R = R; h.T = pl.T; h.m = pl.m; h.g = pl.g;
    h.H = counts;
    h.ctl = nullptr;
    if (launch_hist(h, pl.hist_threads, pl.hist_smem, pl.streaming, (cudaStream_t)stream) != cudaSuccess)
        return RTCDF_ERR_CUDA;
    return RTCDF_OK;
}

rtcdf_status rtcdf_fill_from_counts(const uint32_t *counts, uint64_t total_n, int64_t minVal,
                                    int64_t maxVal, uint64_t pos_begin, uint64_t pos_end, int32_t *out,
                                    void *workspace, size_t ws_bytes, rtcdf_stream_t stream) {
    uint32_t R = 0;
    rtcdf_status st = check_range(minVal, maxVal, &R);
    if (st) return st;
    if (total_n >= (1ull << 32) || pos_begin > pos_end || pos_end > total_n) return RTCDF_ERR_INVALID_ARG;
    if (!counts || ((uintptr_t)counts & 3)) return RTCDF_ERR_INVALID_ARG;
    if (pos_end == pos_begin) return RTCDF_OK;
    if (!out || ((uintptr_t)out & 3)) return RTCDF_ERR_INVALID_ARG;
    if (!workspace || ((uintptr_t)workspace & 255)) return RTCDF_ERR_INVALID_ARG;
    if (ws_bytes < ws_required(R)) return RTCDF_ERR_NO_MEMORY;
    const uint64_t len = pos_end - pos_begin;
    {
        const uintptr_t x = (uintptr_t)out, y = (uintptr_t)counts, w = (uintptr_t)workspace;
        if (x < y + (uint64_t)R * 4 && y < x + len * 4) return RTCDF_ERR_INVALID_ARG;
        if (x < w + ws_bytes && w < x + len * 4) return RTCDF_ERR_INVALID_ARG;
    }
    Plan pl;
    st = make_plan(len, R, 0, (uintptr_t)out, nullptr, &pl);
    if (st) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const WsLayout L = ws_layout(R, ws_bytes);
    // The global counts become the workspace's H (zero between sorts; the scan
    // zeroes it again as it reads it).
    if (cudaMemcpyAsync((char *)workspace + L.hist, counts, (size_t)R * 4, cudaMemcpyDeviceToDevice, s) !=
        cudaSuccess)
        return RTCDF_ERR_CUDA;
    return finish_phase(out, total_n, minVal, R, pl, L, (char *)workspace, nullptr, nullptr, nullptr, s,
                        pos_begin, pos_end);
}

rtcdf_status rtcdf_status_get(rtcdf_stream_t stream, int32_t *device_status) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return RTCDF_ERR_CUDA;
    void *ws = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        auto it = g_ws.find(std::make_pair(dev, (cudaStream_t)stream));
        if (it != g_ws.end()) ws = it->second.ptr;
    }
    // The single-array sorts' workspace and the segmented sorts' one (both
    // start with their status word).
    void *bws = batch_stream_workspace((cudaStream_t)stream);
    int32_t bits = 0, b2 = 0;
    if (ws) {
        const rtcdf_status st = read_status(ws, (cudaStream_t)stream, &bits);
        if (st == RTCDF_ERR_CUDA) return st;
    }
    if (bws) {
        const rtcdf_status st = read_status(bws, (cudaStream_t)stream, &b2);
        if (st == RTCDF_ERR_CUDA) return st;
    }
    if (device_status) *device_status = bits | b2;
    return status_of_bits((uint32_t)(bits | b2));
}

rtcdf_status rtcdf_ws_status_get(void *workspace, rtcdf_stream_t stream, int32_t *device_status) {
    if (!workspace) return RTCDF_ERR_INVALID_ARG;
    return read_status(workspace, (cudaStream_t)stream, device_status);
}

}  // extern "C"
