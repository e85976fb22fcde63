// Internal declarations of the segmented (batched) RT-CDF launch.
#pragma once

#include <vector>

#include "rtcdf_internal.h"

namespace rtcdf {

constexpr int kBatchThreads = 512;
constexpr int kBatchWorkersPerSM = 2;                // one worker's stalls overlap the other's work
constexpr size_t kBatchSmemBytes = 112 * 1024;       // per worker CTA
constexpr uint32_t kBatchSmallMaxN = 65535;          // 16-bit counters are exact below 2^16
constexpr uint32_t kBatchSmallMaxR = 55296;          // 16-bit counters in 108 KB
constexpr uint32_t kBatchTileMax = 27648;            // 32-bit tile histogram in 108 KB
constexpr uint32_t kBatchScanChunk = 4096;           // bins per pass of a segment scan
constexpr uint64_t kBatchMaxR = 1ull << 20;

enum : uint32_t { kItemHist = 0, kItemSmall = 1, kItemScan = 2, kItemFill = 3 };

// One segment (all offsets in 32-bit words of the workspace).
struct BatchSeg {
    uint64_t off;          // first element of the segment in `in`
    uint64_t out_off;      // first element of the segment in `out`
    uint32_t n, R;
    int32_t minVal;
    uint32_t T, m;         // tile width and tiles (large segments)
    uint32_t hist_items;   // HIST items the SCAN waits for
    uint32_t fill_items, fill_chunk;
    uint64_t hist_off, run_end_off, run_val_off, start_run_off;
};

struct BatchItem {
    uint32_t kind, seg;
    uint64_t a, b;         // HIST: key range; FILL: position range (segment-relative)
    uint32_t tile;         // HIST: range tile
    uint32_t aux;          // FILL: index among the segment's FILL items
};

struct BatchSegCtl {
    uint32_t hist_done;    // HIST items finished
    uint32_t scan_done;    // 1 once the SCAN has published the run table
    uint32_t num_runs;
    uint32_t pad;
};

struct BatchCtl {
    uint32_t status;
    uint32_t queue_head;
    uint32_t workers_done;
    uint32_t pad[61];
};

struct BatchArgs {
    const int32_t *in;
    int32_t *out;
    const BatchSeg *segs;
    const BatchItem *items;
    uint32_t num_items, num_segs;
    uint32_t *ws_u32;       // workspace base
    BatchCtl *ctl;
    BatchSegCtl *seg_ctl;
    // Optional phase profile (device, RTCDF_BATCH_PROFILE_WORDS u64), or null:
    // per item kind busy ns, items, first start, last end, dependency-wait ns.
    unsigned long long *prof = nullptr;
};

cudaError_t launch_batched(const BatchArgs &a, int workers, cudaStream_t s);

// Host planner shared by the plan API and the server: segment s reads
// n[s] keys at in_off[s] and writes them sorted at out_off[s].
struct SegSpec {
    uint64_t in_off, out_off, n;
    int64_t minVal, maxVal;
};
struct HostPlan {
    std::vector<BatchSeg> segs;
    std::vector<BatchItem> items;
    size_t ws_words = 0, ctl_off = 0, segctl_off = 0;
    uint32_t small_segs = 0, large_segs = 0;
    uint64_t total_keys = 0;
};
// Validates ranges (R in [1, kBatchMaxR], inside int32) and n < 2^32;
// returns RTCDF-style codes (0 ok, 1 invalid argument, 2 range).
// Work-item sizes of a plan (rtcdf_batch_params with the defaults filled in).
struct BatchTuning {
    uint64_t hist_chunk = 1ull << 19;   // keys per HIST item (tuned on GB300)
    uint32_t fill_chunk = 1u << 16;     // positions per FILL item
    uint32_t small_max_n = kBatchSmallMaxN;
    int64_t lag_items = -1;             // queue distance HIST -> SCAN -> FILL; < 0: phase order
};

int build_host_plan(const SegSpec *segs, uint32_t S, HostPlan *plan,
                    const BatchTuning &tuning = BatchTuning());

}  // namespace rtcdf
