// Host side of the segmented sort: the planner that turns per-segment shapes
// into the work lists of its three launches, and the C entry points
// (rtcdf_batch_* in include/rtcdf.h).
//
// The plan is built once from host-side segment metadata (offsets and ranges)
// and uploaded; running it needs no host work, so it can be captured in a
// CUDA graph and replayed for new keys with the same segment shapes.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "../../include/rtcdf.h"
#include "batched.h"

using namespace rtcdf;

struct rtcdf_batch_plan {
    int device = 0;
    int workers = 0;
    uint32_t num_segs = 0, num_items = 0;
    uint32_t n_first = 0, n_scan = 0, n_small2 = 0, n_fill = 0;
    uint64_t total_keys = 0;
    size_t ws_bytes = 0;          // caller workspace needed
    size_t ctl_off = 0, segctl_off = 0;
    BatchSeg *d_segs = nullptr;
    BatchItem *d_items = nullptr;
    uint32_t small_segs = 0, large_segs = 0;
};

namespace {

size_t words_align(size_t words) { return (words + 63) / 64 * 64; }  // 256-byte units

}  // namespace

namespace rtcdf {

// 0, or the rtcdf_status for the first segment with a bad length or range.
int check_specs(const SegSpec *spec, uint32_t S) {
    for (uint32_t s = 0; s < S; s++) {
        if (spec[s].n >= (1ull << 32)) return 1;
        if (spec[s].minVal < INT32_MIN || spec[s].maxVal > ((int64_t)1 << 31)) return 2;
        if (spec[s].maxVal <= spec[s].minVal || spec[s].maxVal - spec[s].minVal > (int64_t)kBatchMaxR)
            return 2;
    }
    return 0;
}

int build_host_plan(const SegSpec *spec, uint32_t S, HostPlan *P, const BatchTuning &tun) {
    if (const int rc = check_specs(spec, S)) return rc;
    P->segs.assign(S, BatchSeg{});
    P->items.clear();
    P->small_segs = P->large_segs = 0;
    P->total_keys = 0;
    // Workspace (in 32-bit words): control block, per-segment control, then
    // per large segment its histogram (zero between runs), run tables,
    // output-item start runs and lookback state (zero between runs).
    size_t w = 0;
    P->ctl_off = w;     w += words_align(sizeof(BatchCtl) / 4);
    P->segctl_off = w;  w += words_align((size_t)S * sizeof(BatchSegCtl) / 4);
    std::vector<uint32_t> large_ids, small_ids;
    std::vector<uint8_t> in_cta(S, 0);
    uint64_t chunks = 0;
    for (uint32_t s = 0; s < S; s++) {
        BatchSeg &g = P->segs[s];
        memset(&g, 0, sizeof(g));
        g.off = spec[s].in_off;
        g.out_off = spec[s].out_off;
        g.n = (uint32_t)spec[s].n;
        g.R = (uint32_t)(spec[s].maxVal - spec[s].minVal);
        g.minVal = (int32_t)spec[s].minVal;
        P->total_keys += g.n;
        if (g.n == 0) continue;
        if (g.n <= tun.small_max_n && g.R <= kBatchSmallMaxR) in_cta[s] = 1;
        else chunks += (g.R + kBatchScanChunk - 1) / kBatchScanChunk;
    }
    if (tun.small_by_time && chunks > 0) {
        // The second launch's in-CTA segments (R <= small_scan_max_R) start
        // with its scan chunks, and the output launch waits for both: one
        // whose sort is estimated to outlast the launch (its chunks, in waves
        // of six per SM, or the in-CTA sorts spread over all six-per-SM
        // slots) goes the large way instead.  Estimates, measured per item:
        // a 256-thread in-CTA sort 5 us + 1.05 ns per key + 1.9 ns per value,
        // a wave of chunks 10 us.  (On 1024 segments of the benchmark's
        // shapes: 0.336 -> 0.312 ms; on 4096, where the chunks take longer,
        // none is moved.)
        auto small_us = [](const BatchSeg &g) { return 5.0 + 1.05e-3 * g.n + 1.9e-3 * g.R; };
        const double slots = 6.0 * std::max(1u, tun.sms);
        double small_total = 0;
        for (uint32_t s = 0; s < S; s++)
            if (in_cta[s] && P->segs[s].R <= tun.small_scan_max_R) small_total += small_us(P->segs[s]);
        const double launch_us = std::max(10.0 * (1.0 + std::ceil((double)chunks / slots)), small_total / slots);
        for (uint32_t s = 0; s < S; s++)
            if (in_cta[s] && P->segs[s].R <= tun.small_scan_max_R && small_us(P->segs[s]) > launch_us) in_cta[s] = 0;
    }
    for (uint32_t s = 0; s < S; s++) {
        BatchSeg &g = P->segs[s];
        if (g.n == 0) continue;
        if (in_cta[s]) {
            small_ids.push_back(s);
            P->small_segs++;
            continue;
        }
        large_ids.push_back(s);
        P->large_segs++;
        g.m = (g.R + kBatchTileMax - 1) / kBatchTileMax;
        g.T = (g.R + g.m - 1) / g.m;
        const uint64_t chunks = (g.n + tun.hist_chunk - 1) / tun.hist_chunk;
        g.hist_items = (uint32_t)(chunks * g.m);
        g.single_hist = chunks == 1 ? 1u : 0u;
        g.scan_chunks = (g.R + kBatchScanChunk - 1) / kBatchScanChunk;
        g.fill_chunk = tun.fill_chunk;
        g.fill_items = (uint32_t)((g.n + tun.fill_chunk - 1) / tun.fill_chunk);
        g.hist_off = w;      w += words_align((size_t)g.scan_chunks * kBatchScanChunk);
        g.run_end_off = w;   w += words_align(g.R);
        g.run_val_off = w;   w += words_align(g.R);
        g.start_run_off = w; w += words_align(g.fill_items);
        g.state_off = w;     w += words_align((size_t)g.scan_chunks * 2);
    }
    P->ws_words = w;
    const std::vector<BatchSeg> &segs = P->segs;
    auto by_size = [&](uint32_t x, uint32_t y) {
        const uint64_t cx = (uint64_t)segs[x].n + segs[x].R;
        const uint64_t cy = (uint64_t)segs[y].n + segs[y].R;
        return cx != cy ? cx > cy : x < y;
    };
    std::stable_sort(large_ids.begin(), large_ids.end(), by_size);
    std::stable_sort(small_ids.begin(), small_ids.end(), by_size);
    // In-CTA segments with a narrow range run in the scan launch (256-thread
    // CTAs); the others in the first launch.
    std::vector<uint32_t> small2_ids;
    {
        std::vector<uint32_t> keep;
        for (uint32_t s : small_ids) (segs[s].R <= tun.small_scan_max_R ? small2_ids : keep).push_back(s);
        small_ids.swap(keep);
    }
    std::vector<BatchItem> &Q = P->items;
    // First launch: histogram items (largest segments first) with the in-CTA
    // segments (largest first) spread among them in proportion to their keys,
    // so that reads (histograms) and writes (in-CTA sorts) overlap throughout.
    uint64_t large_keys = 0, small_keys = 0, large_done = 0, small_done = 0;
    for (uint32_t s : large_ids) large_keys += (uint64_t)segs[s].n * segs[s].m;
    for (uint32_t s : small_ids) small_keys += segs[s].n;
    size_t si = 0;
    for (uint32_t s : large_ids) {
        const BatchSeg &g = segs[s];
        const uint64_t chunks = g.hist_items / g.m;
        for (uint64_t c = 0; c < chunks; c++) {
            for (uint32_t t = 0; t < g.m; t++) {
                const uint64_t a0 = c * tun.hist_chunk, b0 = std::min<uint64_t>(g.n, (c + 1) * tun.hist_chunk);
                Q.push_back(BatchItem{kItemHist, s, a0, b0, t, 0});
                large_done += b0 - a0;
                // small_done / small_keys keeps up with large_done / large_keys
                while (si < small_ids.size() &&
                       (double)small_done * (double)large_keys < (double)large_done * (double)small_keys) {
                    Q.push_back(BatchItem{kItemSmall, small_ids[si], 0, 0, 0, 0});
                    small_done += segs[small_ids[si]].n;
                    si++;
                }
            }
        }
    }
    for (; si < small_ids.size(); si++) Q.push_back(BatchItem{kItemSmall, small_ids[si], 0, 0, 0, 0});
    P->n_first = (uint32_t)Q.size();
    // Scan launch, in ticket order: each segment's chunks in ascending order
    // (a chunk's lookback only reaches earlier chunks of its segment), the
    // longest chains first.
    std::vector<uint32_t> by_chunks = large_ids;
    std::stable_sort(by_chunks.begin(), by_chunks.end(), [&](uint32_t x, uint32_t y) {
        return segs[x].scan_chunks > segs[y].scan_chunks;
    });
    for (uint32_t s : by_chunks)
        for (uint32_t c = 0; c < segs[s].scan_chunks; c++) Q.push_back(BatchItem{kItemScan, s, c, 0, 0, 0});
    P->n_scan = (uint32_t)Q.size() - P->n_first;
    for (uint32_t s : small2_ids) Q.push_back(BatchItem{kItemSmall, s, 0, 0, 0, 0});
    P->n_small2 = (uint32_t)small2_ids.size();
    // Output launch, most expensive items first, so that cheap ones make the
    // launch's tail.  An item costs its vectors plus the runs it crosses; from
    // the plan alone the runs are estimated as length x min(R, n) / n (every
    // value present: exact for uniform keys, too many for peaked shapes).
    const size_t fill0 = Q.size();
    for (uint32_t s : large_ids) {
        const BatchSeg &g = segs[s];
        for (uint32_t f = 0; f < g.fill_items; f++)
            Q.push_back(BatchItem{kItemFill, s, (uint64_t)f * g.fill_chunk,
                                  std::min<uint64_t>(g.n, (uint64_t)(f + 1) * g.fill_chunk), 0, f});
    }
    auto fill_cost = [&](const BatchItem &x) {
        const BatchSeg &g = segs[x.seg];
        return (double)(x.b - x.a) * (0.25 + (double)std::min(g.R, g.n) / (double)g.n);
    };
    std::stable_sort(Q.begin() + fill0, Q.end(), [&](const BatchItem &x, const BatchItem &y) {
        return fill_cost(x) > fill_cost(y);
    });
    P->n_fill = (uint32_t)Q.size() - P->n_first - P->n_scan - P->n_small2;
    return 0;
}

}  // namespace rtcdf

extern "C" {

rtcdf_status rtcdf_batch_plan_create(const int64_t *seg_offsets, const int64_t *seg_minVal,
                                     const int64_t *seg_maxVal, int32_t num_segments,
                                     rtcdf_batch_plan **plan_out) {
    return rtcdf_batch_plan_create_ex(seg_offsets, seg_minVal, seg_maxVal, num_segments, nullptr,
                                      plan_out);
}

rtcdf_status rtcdf_batch_plan_create_ex(const int64_t *seg_offsets, const int64_t *seg_minVal,
                                        const int64_t *seg_maxVal, int32_t num_segments,
                                        const rtcdf_batch_params *params,
                                        rtcdf_batch_plan **plan_out) try {
    if (!plan_out || num_segments < 0) return RTCDF_ERR_INVALID_ARG;
    BatchTuning tun;
    if (params) {
        if (params->hist_chunk < 0 || (params->hist_chunk > 0 && params->hist_chunk < 4096) ||
            params->fill_chunk < 0 || (params->fill_chunk > 0 && params->fill_chunk < 4096) ||
            params->small_max_n < 0 || params->small_max_n > (int32_t)kBatchSmallMaxN ||
            params->small_scan_max_R < 0 || params->small_scan_max_R > (int32_t)kSmallInScanCapR ||
            params->small_by_time < -1 || params->small_by_time > 1)
            return RTCDF_ERR_INVALID_ARG;
        if (params->hist_chunk) tun.hist_chunk = (uint64_t)params->hist_chunk;
        if (params->fill_chunk) tun.fill_chunk = (uint32_t)params->fill_chunk;
        if (params->small_max_n) tun.small_max_n = (uint32_t)params->small_max_n;
        if (params->small_scan_max_R) tun.small_scan_max_R = (uint32_t)params->small_scan_max_R;
        if (params->small_by_time < 0) tun.small_by_time = 0;
    }
    *plan_out = nullptr;
    if (num_segments > 0 && (!seg_offsets || !seg_minVal || !seg_maxVal)) return RTCDF_ERR_INVALID_ARG;
    const uint32_t S = (uint32_t)num_segments;
    if (S > 0 && seg_offsets[0] < 0) return RTCDF_ERR_INVALID_ARG;
    std::vector<SegSpec> spec(S);
    for (uint32_t s = 0; s < S; s++) {
        if (seg_offsets[s + 1] < seg_offsets[s]) return RTCDF_ERR_INVALID_ARG;
        spec[s] = SegSpec{(uint64_t)seg_offsets[s], (uint64_t)seg_offsets[s],
                          (uint64_t)(seg_offsets[s + 1] - seg_offsets[s]), seg_minVal[s], seg_maxVal[s]};
    }
    if (const int rc = check_specs(spec.data(), S)) return (rtcdf_status)rc;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return RTCDF_ERR_CUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return RTCDF_ERR_CUDA;
    tun.sms = (uint32_t)sms;
    HostPlan hp;
    const int rc = build_host_plan(spec.data(), S, &hp, tun);
    if (rc) return (rtcdf_status)rc;

    rtcdf_batch_plan *p = new rtcdf_batch_plan();
    p->device = dev;
    p->workers = sms;  // resident 1024-thread CTAs of the first launch (one per SM)
    p->num_segs = S;
    p->num_items = (uint32_t)hp.items.size();
    p->n_first = hp.n_first;
    p->n_scan = hp.n_scan;
    p->n_small2 = hp.n_small2;
    p->n_fill = hp.n_fill;
    p->total_keys = hp.total_keys;
    p->ws_bytes = hp.ws_words * 4;
    p->ctl_off = hp.ctl_off;
    p->segctl_off = hp.segctl_off;
    p->small_segs = hp.small_segs;
    p->large_segs = hp.large_segs;
    if (S > 0 && cudaMalloc(&p->d_segs, sizeof(BatchSeg) * S) != cudaSuccess) {
        delete p;
        return RTCDF_ERR_NO_MEMORY;
    }
    if (!hp.items.empty() && cudaMalloc(&p->d_items, sizeof(BatchItem) * hp.items.size()) != cudaSuccess) {
        cudaFree(p->d_segs);
        delete p;
        return RTCDF_ERR_NO_MEMORY;
    }
    if ((S > 0 && cudaMemcpy(p->d_segs, hp.segs.data(), sizeof(BatchSeg) * S,
                             cudaMemcpyHostToDevice) != cudaSuccess) ||
        (!hp.items.empty() && cudaMemcpy(p->d_items, hp.items.data(), sizeof(BatchItem) * hp.items.size(),
                                         cudaMemcpyHostToDevice) != cudaSuccess)) {
        cudaFree(p->d_segs);
        cudaFree(p->d_items);
        delete p;
        return RTCDF_ERR_CUDA;
    }
    *plan_out = p;
    return RTCDF_OK;
} catch (...) {  // an allocation failed (std::bad_alloc and the like)
    return RTCDF_ERR_NO_MEMORY;
}

rtcdf_status rtcdf_batch_plan_destroy(rtcdf_batch_plan *plan) {
    if (!plan) return RTCDF_OK;
    cudaFree(plan->d_segs);
    cudaFree(plan->d_items);
    delete plan;
    return RTCDF_OK;
}

rtcdf_status rtcdf_batch_workspace_size(const rtcdf_batch_plan *plan, size_t *bytes) {
    if (!plan || !bytes) return RTCDF_ERR_INVALID_ARG;
    *bytes = plan->ws_bytes;
    return RTCDF_OK;
}

rtcdf_status rtcdf_batch_plan_info(const rtcdf_batch_plan *plan, rtcdf_batch_info *info) {
    if (!plan || !info) return RTCDF_ERR_INVALID_ARG;
    memset(info, 0, sizeof(*info));
    info->num_segments = plan->num_segs;
    info->total_keys = plan->total_keys;
    info->small_segments = plan->small_segs;
    info->large_segments = plan->large_segs;
    info->work_items = plan->num_items;
    info->workers = (uint32_t)plan->workers;
    info->workspace_bytes = plan->ws_bytes;
    return RTCDF_OK;
}

rtcdf_status rtcdf_sort_batched_ws(const rtcdf_batch_plan *plan, const int32_t *in, int32_t *out,
                                   void *workspace, size_t ws_bytes, rtcdf_stream_t stream) {
    return rtcdf_sort_batched_profiled(plan, in, out, workspace, ws_bytes, nullptr, stream);
}

rtcdf_status rtcdf_sort_batched_profiled(const rtcdf_batch_plan *plan, const int32_t *in,
                                         int32_t *out, void *workspace, size_t ws_bytes,
                                         uint64_t *profile, rtcdf_stream_t stream) {
    if (profile && ((uintptr_t)profile & 7)) return RTCDF_ERR_INVALID_ARG;
    if (!plan) return RTCDF_ERR_INVALID_ARG;
    if (plan->num_items == 0) return RTCDF_OK;
    if (!in || !out || !workspace) return RTCDF_ERR_INVALID_ARG;
    if (((uintptr_t)in & 3) || ((uintptr_t)out & 3) || ((uintptr_t)workspace & 255))
        return RTCDF_ERR_INVALID_ARG;
    if ((const void *)in != (const void *)out) {
        const uintptr_t x = (uintptr_t)in, y = (uintptr_t)out, b = plan->total_keys * 4;
        if (x < y + b && y < x + b) return RTCDF_ERR_INVALID_ARG;
    }
    if (ws_bytes < plan->ws_bytes) return RTCDF_ERR_NO_MEMORY;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return RTCDF_ERR_CUDA;
    if (dev != plan->device) return RTCDF_ERR_INVALID_ARG;
    uint32_t *ws = (uint32_t *)workspace;
    BatchArgs a;
    a.in = in;
    a.out = out;
    a.segs = plan->d_segs;
    a.items = plan->d_items;
    a.n_first = plan->n_first;
    a.n_scan = plan->n_scan;
    a.n_small2 = plan->n_small2;
    a.n_fill = plan->n_fill;
    a.num_segs = plan->num_segs;
    a.ws_u32 = ws;
    a.ctl = (BatchCtl *)(ws + plan->ctl_off);
    a.seg_ctl = (BatchSegCtl *)(ws + plan->segctl_off);
    a.prof = reinterpret_cast<unsigned long long *>(profile);
    if (launch_batched(a, (cudaStream_t)stream) != cudaSuccess) return RTCDF_ERR_CUDA;
    return RTCDF_OK;
}

rtcdf_status rtcdf_batch_status_get(void *workspace, rtcdf_stream_t stream, int32_t *device_status) {
    if (!workspace) return RTCDF_ERR_INVALID_ARG;
    BatchCtl *ctl = (BatchCtl *)workspace;  // the control block is first
    uint32_t v = 0;
    if (cudaMemcpyAsync(&v, &ctl->status, 4, cudaMemcpyDeviceToHost, (cudaStream_t)stream) != cudaSuccess)
        return RTCDF_ERR_CUDA;
    if (cudaMemsetAsync(&ctl->status, 0, 4, (cudaStream_t)stream) != cudaSuccess) return RTCDF_ERR_CUDA;
    if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return RTCDF_ERR_CUDA;
    if (device_status) *device_status = (int32_t)v;
    // A wait that ran out makes every other finding unreliable: report it first.
    if (v & kDevTimeout) return RTCDF_ERR_TIMEOUT;
    if (v & kDevBadSegment) return RTCDF_ERR_INVALID_ARG;
    if (v & kDevKeyOutOfRange) return RTCDF_ERR_KEY_OUT_OF_RANGE;
    return RTCDF_OK;
}

rtcdf_status rtcdf_sort_batched_host(const int32_t *in, int32_t *out, const int64_t *seg_offsets,
                                     const int64_t *seg_minVal, const int64_t *seg_maxVal,
                                     int32_t num_segments, rtcdf_stream_t stream) {
    rtcdf_batch_plan *plan = nullptr;
    rtcdf_status st = rtcdf_batch_plan_create(seg_offsets, seg_minVal, seg_maxVal, num_segments, &plan);
    if (st) return st;
    void *ws = nullptr;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t bytes = std::max<size_t>(plan->ws_bytes, 256);
    if (cudaMallocAsync(&ws, bytes, s) != cudaSuccess) {
        rtcdf_batch_plan_destroy(plan);
        return RTCDF_ERR_NO_MEMORY;
    }
    st = RTCDF_OK;
    if (cudaMemsetAsync(ws, 0, bytes, s) != cudaSuccess) st = RTCDF_ERR_CUDA;
    if (!st) st = rtcdf_sort_batched_ws(plan, in, out, ws, bytes, stream);
    int32_t bits = 0;
    const rtcdf_status dst = rtcdf_batch_status_get(ws, stream, &bits);  // synchronises `stream`
    const bool freed = cudaFreeAsync(ws, s) == cudaSuccess && cudaStreamSynchronize(s) == cudaSuccess;
    rtcdf_batch_plan_destroy(plan);
    return st ? st : dst ? dst : freed ? RTCDF_OK : RTCDF_ERR_CUDA;
}

}  // extern "C"
