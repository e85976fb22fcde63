// Internal declarations of the segmented (batched) RT-CDF pipeline.
#pragma once

#include <vector>

#include "rtcdf_internal.h"

namespace rtcdf {

// Three launches per plan:
//   1. histogram items of the large segments and whole in-CTA sorts of the
//      small ones (1024 threads, 112 KB of shared memory each, two per SM);
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
    uint32_t scan_ticket;  // dynamic order of the scan CTAs (reset by the output launch)
    uint32_t pad[62];
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
};

cudaError_t launch_batched(const BatchArgs &a, cudaStream_t s);

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
};

// 0, or the rtcdf_status for the first segment with a bad length or range
// (n >= 2^32, R outside [1, kBatchMaxR], range outside int32).
int check_specs(const SegSpec *segs, uint32_t S);
int build_host_plan(const SegSpec *segs, uint32_t S, HostPlan *plan,
                    const BatchTuning &tuning = BatchTuning());

}  // namespace rtcdf
