// Internal declarations shared by the RT-CDF kernels and the C-ABI host code.
// Not installed; the public interface is include/rtcdf.h.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/rtcdf.h"

namespace rtcdf {

// Launch parameters of the tuning table for (n, R), if it has an entry
// (tune.cu).
bool tune_lookup(uint64_t n, uint32_t R, rtcdf_params *out);

// Device status bits (mirror RTCDF_DEV_* in rtcdf.h).
constexpr uint32_t kDevKeyOutOfRange = 0x1;
constexpr uint32_t kDevTimeout = 0x2;
constexpr uint32_t kDevBadSegment = 0x4;

// The library-owned workspace of rtcdf_sort_batched for `s` on the current
// device, or null (devplan.cu).
void *batch_stream_workspace(cudaStream_t s);

// Local-CDF scan: one CTA of kScanThreads threads scans kScanChunk histogram
// bins (kScanItems per thread); chunks are chained by a decoupled lookback.
constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanChunk = kScanThreads * kScanItems;

// Upper bound on output-generation CTAs (the start-run table has this many slots).
constexpr int kMaxFillCtas = 4096;

// Iteration cap of every device-side wait; a wait that runs out records
// kDevTimeout and the kernel carries on without hanging.
constexpr uint32_t kMaxSpin = 1u << 21;

// Control block at the start of every workspace.
struct Ctl {
    uint32_t status;       // RTCDF_DEV_* bits, sticky until read
    uint32_t scan_ticket;  // dynamic chunk index of the lookback scan
    uint32_t num_runs;     // number of values with c_v > 0 (written by the scan)
    uint32_t pad[61];
};
static_assert(sizeof(Ctl) == 256, "control block is 256 bytes");

// Most lookback chunks any sort can use (RTCDF_MAX_R / kScanChunk).
constexpr uint32_t kMaxScanChunks = (1u << 24) / kScanChunk;

// Byte offsets of the workspace regions for a sort with range size R in a
// workspace of `total` bytes.  Regions that must be zero when a sort starts
// (control block, lookback state, histogram H) sit at fixed offsets from the
// bottom, so they stay zero whatever R the previous sort had; regions that
// each sort writes before reading (run table, start-run table) are anchored
// at the top and may overlap what a previous sort left behind.
struct WsLayout {
    size_t ctl, scan_state, hist, run_end, run_val, start_run, total;
    uint32_t scan_chunks;
    size_t zero_bytes;  // [0, zero_bytes) must be zero when a sort starts
};

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

constexpr size_t kWsHistOffset = 256 + (size_t)kMaxScanChunks * 8;

// H is padded to whole scan chunks.  Its size never decreases as R grows, so a
// sort's run table (anchored at the top) never reaches the part of H
// (anchored at the bottom) that a sort with a smaller range expects zeroed.
inline size_t hist_region_bytes(uint64_t R) {
    return (size_t)((R + kScanChunk - 1) / kScanChunk) * kScanChunk * 4;
}

inline size_t ws_required(uint64_t R) {
    return kWsHistOffset + hist_region_bytes(R) + align_up((size_t)kMaxFillCtas * 4, 256) +
           2 * align_up((size_t)R * 4, 256);
}

inline WsLayout ws_layout(uint64_t R, size_t total) {
    WsLayout L;
    L.scan_chunks = (uint32_t)((R + kScanChunk - 1) / kScanChunk);
    L.ctl = 0;
    L.scan_state = 256;
    L.hist = kWsHistOffset;
    L.zero_bytes = L.hist + hist_region_bytes(R);
    size_t top = total / 256 * 256;
    L.run_val = top - align_up((size_t)R * 4, 256);
    L.run_end = L.run_val - align_up((size_t)R * 4, 256);
    L.start_run = L.run_end - align_up((size_t)kMaxFillCtas * 4, 256);
    L.total = total;
    return L;
}

// ---------------------------------------------------------------- histogram
struct HistArgs {
    const int32_t *in;
    uint64_t n;
    uint64_t nvec;         // 16-byte vectors after the unaligned head
    uint32_t head;         // elements before the first 16-byte aligned address
    uint32_t min_u;        // (uint32_t)minVal
    uint32_t R, T, m, g;   // range size, tile width, tiles, CTAs per tile
    uint32_t *H;           // global histogram, R entries (zero on entry)
    Ctl *ctl;
};
cudaError_t launch_hist(const HistArgs &a, int threads, size_t smem, bool streaming,
                        cudaStream_t s);
cudaError_t hist_max_ctas_per_sm(int threads, size_t smem, bool streaming, int *ctas);

// ---------------------------------------------------------------- scan
struct ScanArgs {
    uint32_t *H;           // histogram, zeroed as it is consumed
    uint64_t *state;       // lookback state per chunk (zero on entry)
    Ctl *ctl;
    uint32_t *run_end;     // inclusive CDF at each non-empty value (exclusive end of its run)
    int32_t *run_val;      // the key of each non-empty value
    uint32_t *start_run;   // per output CTA: run containing its first position
    uint64_t n;            // keys of the whole array (the counts must add up to it)
    uint64_t fill_chunk;   // positions per output CTA (multiple of 4)
    uint32_t head;         // first output CTA boundary is pos_base + head + fill_chunk
    uint32_t fill_ctas;
    uint32_t pos_base;     // the output CTAs cover positions [pos_base, pos_end) of
    uint32_t pos_end;      // the sorted array (0 and n for a whole sort)
    uint32_t R, T, chunks;
    int32_t minVal;
    uint32_t *dbg_hist, *dbg_cdf, *dbg_offset;  // optional exports
};
cudaError_t launch_scan(const ScanArgs &a, cudaStream_t s);

// ---------------------------------------------------------------- output
struct FillArgs {
    int32_t *out;          // out[0] holds position pos_base of the sorted array
    uint64_t n;            // end of the positions written (pos_end)
    uint32_t pos_base;     // first position written (0 for a whole sort)
    uint64_t fill_chunk;
    uint32_t head;
    uint32_t fill_ctas;
    const uint32_t *run_end;
    const int32_t *run_val;
    const uint32_t *start_run;
    Ctl *ctl;
    uint64_t *scan_state;  // reset here for the next call
    uint32_t scan_chunks;
    uint32_t R;            // entries of run_end / run_val
};
cudaError_t launch_fill(const FillArgs &a, int threads, cudaStream_t s);

}  // namespace rtcdf
