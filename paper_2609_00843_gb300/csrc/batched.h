// Internal declarations of the segmented (batched) RT-CDF pipeline.
#pragma once

#include <climits>
#include <vector>

#include "rtcdf_internal.h"

namespace rtcdf {

// Three launches per plan:
//   1. histogram items of the large segments and whole in-CTA sorts of the
//      small ones (1024 threads, 112 KB of shared memory each, one per SM);
//   2. local CDFs + offsets: one 256-thread CTA per 4096-bin chunk of a large
//      segment's histogram, chained within the segment by a decoupled lookback,
//      plus the in-CTA sorts of the small segments with R <= kSmallInScanMaxR
//      (these do not wait for the first launch, so they overlap its tail and
//      the latency-bound scan chunks);
//   3. output items of the large segments (512-thread CTAs).
constexpr int kSegThreads = 1024;
constexpr size_t kSegSmemBytes = 112 * 1024;          // first launch, per CTA
constexpr uint32_t kBatchSmallMaxN = 65535;           // 16-bit counters are exact below 2^16
constexpr uint32_t kBatchSmallMaxR = 55296;           // 16-bit counters in 108 KB
constexpr uint32_t kBatchTileMax = 28672;             // 32-bit tile histogram in 112 KB
constexpr uint32_t kBatchScanChunk = 4096;            // bins per scan CTA (4 per thread)
constexpr uint32_t kSegFillRuns = 4096;               // run window of an output CTA
constexpr uint32_t kSmallInScanMaxR = 16000;          // default: in-CTA segments run by scan-launch CTAs
// Shared memory of a scan-launch CTA (words): the chunk's staged runs (end and
// value, one padding word per 32), reused for an in-CTA segment's counters and
// its block-scan scratch (the last 64 words).
constexpr uint32_t kScanStageWords = kBatchScanChunk + kBatchScanChunk / 32;
constexpr uint32_t kScanSmemWords = 2 * kScanStageWords;
constexpr uint32_t kSmallInScanCapR = 2 * (kScanSmemWords - 64);  // 16-bit counters
constexpr uint64_t kBatchMaxR = 1ull << 20;

enum : uint32_t { kItemHist = 0, kItemSmall = 1, kItemScan = 2, kItemFill = 3 };

// One segment (all offsets in 32-bit words of the workspace).
struct BatchSeg {
    uint64_t off;          // first element of the segment in `in`
    uint64_t out_off;      // first element of the segment in `out`
    uint32_t n, R;
    int32_t minVal;
    uint32_t T, m;         // tile width and tiles (large segments; m = 0 for small ones)
    uint32_t hist_items;   // HIST items per tile times tiles
    uint32_t fill_items, fill_chunk;
    uint32_t scan_chunks;  // ceil(R / kBatchScanChunk)
    uint32_t single_hist;  // 1: one HIST item per tile, so it stores its counts
    uint64_t hist_off, run_end_off, run_val_off, start_run_off, state_off;
};

struct BatchItem {
    uint32_t kind, seg;
    uint64_t a, b;         // HIST: key range; SCAN: chunk index; FILL: position range
    uint32_t tile;         // HIST: range tile
    uint32_t aux;          // FILL: index among the segment's FILL items
};

struct BatchSegCtl {
    uint32_t num_runs;     // written by the segment's last scan chunk
    uint32_t pad[3];
};

struct BatchCtl {
    uint32_t status;
    uint32_t scan_ticket;   // dynamic order of the scan CTAs (reset by the output launch)
    uint32_t first_ticket;  // device-built lists: items of the first launch taken so far
                            // (reset by the planner before the first launch)
    uint32_t plan_ticket;   // device planner: CTAs in start order (reset by the output launch)
    uint32_t pad[60];
};

struct BatchArgs {
    const int32_t *in;
    int32_t *out;
    const BatchSeg *segs;
    const BatchItem *items;          // [first launch | scan chunks | in-CTA segments of the
                                     //  scan launch | output launch]
    uint32_t n_first, n_scan, n_small2, n_fill;
    uint32_t num_segs;
    uint32_t *ws_u32;                // workspace base
    BatchCtl *ctl;
    BatchSegCtl *seg_ctl;
    // Optional phase profile (device, RTCDF_BATCH_PROFILE_WORDS u64), or null:
    // per item kind busy ns, items, first start, last end, dependency-wait ns.
    unsigned long long *prof = nullptr;
    // Lists built on the device: their lengths (n_first, n_scan, n_small2,
    // n_fill, n_hist, n_small1, then the lengths of the histogram, scan and
    // output lists by class) in device memory; null for a host-built plan.
    // The lists then sit at fixed offsets given by their bounds
    // (devplan_pos).
    const uint32_t *dev_counts = nullptr;
    uint64_t dev_bounds[5] = {0, 0, 0, 0, 0};  // DevListBounds: hist, first, scan, small2, fill
    // The device planner's lookback records, zeroed by the output launch.
    uint32_t *plan_look = nullptr;
    uint32_t plan_look_words = 0;
};

cudaError_t launch_batched(const BatchArgs &a, cudaStream_t s);
// The three launches over device-built lists with fixed grids.
cudaError_t launch_batched_dev(const BatchArgs &a, uint32_t first_ctas, uint32_t scan_ctas, uint32_t fill_ctas,
                               cudaStream_t s);

// Host planner shared by the plan API and the server: segment s reads
// n[s] keys at in_off[s] and writes them sorted at out_off[s].
struct SegSpec {
    uint64_t in_off, out_off, n;
    int64_t minVal, maxVal;
};
struct HostPlan {
    std::vector<BatchSeg> segs;
    std::vector<BatchItem> items;    // [first launch | scan chunks | in-CTA segments of the
                                     //  scan launch | output launch]
    uint32_t n_first = 0, n_scan = 0, n_small2 = 0, n_fill = 0;
    size_t ws_words = 0, ctl_off = 0, segctl_off = 0;
    uint32_t small_segs = 0, large_segs = 0;
    uint64_t total_keys = 0;
};

// Work-item sizes of a plan (rtcdf_batch_params with the defaults filled in).
struct BatchTuning {
    uint64_t hist_chunk = 1ull << 19;   // keys per HIST item
    uint32_t fill_chunk = 1u << 16;     // positions per FILL item
    uint32_t small_max_n = kBatchSmallMaxN;
    uint32_t small_scan_max_R = kSmallInScanMaxR;
    uint32_t small_by_time = 1;         // host plan: in-CTA segments that would outlast the second launch go large
    uint32_t sms = 152;                 // SMs of the device the plan is for
};

// 0, or the rtcdf_status for the first segment with a bad length or range
// (n >= 2^32, R outside [1, kBatchMaxR], range outside int32).
int check_specs(const SegSpec *segs, uint32_t S);
int build_host_plan(const SegSpec *segs, uint32_t S, HostPlan *plan,
                    const BatchTuning &tuning = BatchTuning());

// ---------------------------------------------------------------- device planner
// A segmented sort whose segment metadata lives in device memory is planned
// on the device (devplan.cu) into a workspace sized from host-known bounds.
// The per-segment and per-item rules below are shared by the planner kernels
// and a host emulation of them (for checks on the CPU).
struct DevBounds {
    uint32_t S;                 // segments
    uint32_t max_R;             // every R_s <= max_R <= kBatchMaxR
    uint64_t max_total_keys;    // seg_offsets[S] <= max_total_keys
};

// The lists, in items-array order.  Each kind of item comes in lists by
// size, which the launches take largest first, so that a launch ends on
// short items (in segment order, the last long histogram items made a tail
// of about 0.1 ms, measured): histogram items by keys (>= hist_chunk / 2,
// >= hist_chunk / 4, fewer), scan chunks by their segment's chain (at least
// kLongChain chunks first), output items by estimated cost (length x (1/4 +
// min(R, n) / n) at least fill_chunk / 2 first).
enum : uint32_t {
    kListHist0 = 0, kListHist1 = 1, kListHist2 = 2,
    kListSmall1 = 3,
    kListScan0 = 4, kListScan1 = 5,
    kListSmall2 = 6,
    kListFill0 = 7, kListFill1 = 8,
    kNumLists = 9
};
constexpr uint32_t kHistClasses = 3;
constexpr uint32_t kLongChain = 8;

// Items of one segment in each list.
struct DevSegCount {
    uint32_t v[kNumLists];
};

// Exclusive prefixes of DevSegCount over the segments before s.
struct DevPfx {
    uint32_t v[kNumLists];
    uint32_t pad[16 - kNumLists];
};

// Lengths of the lists (the first four are BatchArgs::dev_counts[0..3]).
struct DevPlanHdr {
    uint32_t n_first, n_scan, n_small2, n_fill, n_hist, n_small1;
    uint32_t n_hist_class[kHistClasses];   // dev_counts[6..8]
    uint32_t n_scan_class[2];              // dev_counts[9..10]
    uint32_t n_fill_class[2];              // dev_counts[11..12]
    uint32_t pad[51];
};

// Bounds of the lists (each list of a kind has the kind's bound).
struct DevListBounds {
    uint64_t hist, first, scan, small2, fill;  // first = 3 * hist + (in-CTA segments: S)
};

// Workspace layout of the device-planned sort (32-bit word offsets).  Every
// segment owns a fixed slot [H | lookback state | run ends | run keys] sized
// for max_R, so H and the state, zero between runs, stay where the next run
// of any layout expects them.
struct DevLayout {
    size_t ctl, hdr, segctl, segs, look, items, start, slots, slot_words, total_words;
    size_t slot_state, slot_run_end, slot_run_val;  // offsets inside a slot
    DevListBounds lb;
    uint64_t item_bound;
    uint32_t look_blocks;  // planner CTAs (1024 segments each)
};

// Position in the items array of list `list`'s element k (its base is the
// bound-sum of the lists before it).
__host__ __device__ inline uint64_t devplan_pos(const DevListBounds &b, uint32_t list, uint64_t k) {
    if (list < kHistClasses) return list * b.hist + k;
    switch (list) {
        case kListSmall1: return kHistClasses * b.hist + k;
        case kListScan0: return b.first + k;
        case kListScan1: return b.first + b.scan + k;
        case kListSmall2: return b.first + 2 * b.scan + k;
        case kListFill0: return b.first + 2 * b.scan + b.small2 + k;
        default: return b.first + 2 * b.scan + b.small2 + b.fill + k;
    }
}

// The h-th item over `nl` consecutive lists (first list `list0`, lengths n):
// the lists taken one after another.
__host__ __device__ inline uint64_t devplan_chain_pos(const DevListBounds &b, uint32_t list0, const uint32_t *n,
                                                      uint32_t nl, uint64_t h) {
    uint32_t c = 0;
    while (c + 1 < nl && h >= n[c]) h -= n[c++];
    return devplan_pos(b, list0 + c, h);
}

// The first launch's k-th ticket (k < nh + ns, nh = the histogram lists'
// lengths nc[0..2] summed): the histogram lists one after another (largest
// items first), and the in-CTA segments spread evenly among them --
// in-CTA segment j at ticket floor(j * (nh + ns) / ns) -- so that reads
// (histograms) and writes (in-CTA sorts) overlap throughout.  Returns the
// items-array position.
__host__ __device__ inline uint64_t devplan_first_pos(uint64_t k, const uint32_t *nc, uint64_t ns,
                                                      const DevListBounds &b) {
    const uint64_t nh = (uint64_t)nc[0] + nc[1] + nc[2], T = nh + ns;
    uint64_t h = k;
    if (ns > 0) {
        const uint64_t j = (k * ns + T - 1) / T;  // in-CTA slots before ticket k: ceil(k * ns / T)
        if (j < ns && j * T / ns == k) return devplan_pos(b, kListSmall1, j);
        h = k - j;
    }
    return devplan_chain_pos(b, kListHist0, nc, kHistClasses, h);
}
// 0, or RTCDF_ERR_RANGE / RTCDF_ERR_INVALID_ARG for bounds out of range.
int devplan_layout(const DevBounds &b, const BatchTuning &t, DevLayout *L);

// List (0 or 1 of its kind) of an output item of `len` positions.
__host__ __device__ inline uint32_t devplan_fill_class(uint64_t len, const BatchSeg &g) {
    const uint32_t d = g.R < g.n ? g.R : g.n;  // min(R, n)
    // len * (1/4 + d / n) >= fill_chunk / 2, in integers
    return (uint64_t)len * ((uint64_t)g.n + 4ull * d) >= 2ull * g.fill_chunk * g.n ? 0u : 1u;
}

// Size class of a histogram item of `keys` keys.
__host__ __device__ inline uint32_t devplan_hist_class(uint64_t keys, uint64_t hist_chunk) {
    return keys >= hist_chunk / 2 ? 0u : keys >= hist_chunk / 4 ? 1u : 2u;
}

// Segment s from its metadata: its descriptor (workspace offsets left to the
// caller) and its items per list, as build_host_plan classifies it; false
// when it breaks the bounds or the limits of a segmented sort.
__host__ __device__ inline bool devplan_segment(int64_t o0, int64_t o1, int64_t mn, int64_t mx, const DevBounds &b,
                                                const BatchTuning &t, BatchSeg *g, DevSegCount *c) {
    for (uint32_t i = 0; i < kNumLists; i++) c->v[i] = 0;
    *g = BatchSeg{};
    if (o0 < 0 || o1 < o0 || (uint64_t)o1 > b.max_total_keys) return false;
    const uint64_t n = (uint64_t)(o1 - o0);
    if (n >= (1ull << 32)) return false;
    if (mn < INT32_MIN || mx > ((int64_t)1 << 31) || mx <= mn || mx - mn > (int64_t)b.max_R) return false;
    g->off = g->out_off = (uint64_t)o0;
    g->n = (uint32_t)n;
    g->R = (uint32_t)(mx - mn);
    g->minVal = (int32_t)mn;
    if (n == 0) return true;
    if (g->n <= t.small_max_n && g->R <= kBatchSmallMaxR) {
        if (g->R <= t.small_scan_max_R) c->v[kListSmall2] = 1;
        else c->v[kListSmall1] = 1;
        return true;
    }
    g->m = (g->R + kBatchTileMax - 1) / kBatchTileMax;
    g->T = (g->R + g->m - 1) / g->m;
    const uint64_t chunks = (n + t.hist_chunk - 1) / t.hist_chunk;
    g->hist_items = (uint32_t)(chunks * g->m);
    g->single_hist = chunks == 1 ? 1u : 0u;
    g->scan_chunks = (g->R + kBatchScanChunk - 1) / kBatchScanChunk;
    g->fill_chunk = t.fill_chunk;
    g->fill_items = (uint32_t)((n + t.fill_chunk - 1) / t.fill_chunk);
    // Whole histogram chunks are class 0; the last chunk, when shorter, goes
    // by its keys.  Output items likewise: the whole ones share a class, the
    // last one goes by its length.
    const uint64_t whole = n / t.hist_chunk, rest = n - whole * t.hist_chunk;
    c->v[kListHist0] = (uint32_t)(whole * g->m);
    if (rest) c->v[devplan_hist_class(rest, t.hist_chunk)] += g->m;
    c->v[g->scan_chunks >= kLongChain ? kListScan0 : kListScan1] = g->scan_chunks;
    const uint64_t fwhole = n / t.fill_chunk, frest = n - fwhole * t.fill_chunk;
    c->v[kListFill0 + devplan_fill_class(t.fill_chunk, *g)] = (uint32_t)fwhole;
    if (frest) c->v[kListFill0 + devplan_fill_class(frest, *g)] += 1;
    return true;
}

// The k-th item of list `list` that belongs to segment s (k counted within the
// segment): histogram items chunk-major over tiles (class 0: the whole chunks,
// then the last chunk if it is in that class; classes 1 and 2: the last
// chunk), scan chunks ascending, output items ascending (the whole ones in
// their class, then the last one in its class).
__host__ __device__ inline BatchItem devplan_item(uint32_t list, uint32_t s, uint32_t k, const BatchSeg &g,
                                                  const BatchTuning &t) {
    BatchItem it{};
    it.seg = s;
    if (list < kHistClasses) {
        const uint32_t whole_items = list == kListHist0 ? (uint32_t)(g.n / t.hist_chunk) * g.m : 0u;
        const uint32_t c = k < whole_items ? k / g.m : (uint32_t)(g.n / t.hist_chunk);
        it.kind = kItemHist;
        it.a = (uint64_t)c * t.hist_chunk;
        it.b = ((uint64_t)c + 1) * t.hist_chunk < g.n ? ((uint64_t)c + 1) * t.hist_chunk : g.n;
        it.tile = k < whole_items ? k % g.m : k - whole_items;
        return it;
    }
    switch (list) {
        case kListScan0:
        case kListScan1:
            it.kind = kItemScan;
            it.a = k;
            break;
        case kListFill0:
        case kListFill1: {
            const uint32_t fwhole = g.n / g.fill_chunk;
            const uint32_t in_list = devplan_fill_class(g.fill_chunk, g) == list - kListFill0 ? fwhole : 0u;
            const uint32_t f = k < in_list ? k : fwhole;  // else the last (shorter) item
            it.kind = kItemFill;
            it.a = (uint64_t)f * g.fill_chunk;
            it.b = ((uint64_t)f + 1) * g.fill_chunk < g.n ? ((uint64_t)f + 1) * g.fill_chunk : g.n;
            it.aux = f;
            break;
        }
        default:
            it.kind = kItemSmall;
            break;
    }
    return it;
}

// Host emulation of the device planner: the descriptors, prefixes, list
// lengths and items the planner kernels write (workspace offsets per the
// layout), or a nonzero rtcdf_status for metadata that breaks the bounds.
int devplan_host(const int64_t *offs, const int64_t *mn, const int64_t *mx, const DevBounds &b,
                 const BatchTuning &t, const DevLayout &L, std::vector<BatchSeg> *segs,
                 std::vector<DevPfx> *pfx, DevPlanHdr *hdr, std::vector<BatchItem> *items);

}  // namespace rtcdf
