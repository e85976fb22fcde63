/*
 * rtcdf.h -- C ABI of librtcdf, a GB300 (sm_103a) implementation of
 * Range-Tiled CDF sort (RT-CDF) from "Shared-Memory Range-Tiled CDF Sort for
 * Small-Range Integer Keys on GPUs" (Ando, Takase, Fujimoto, Wada).
 *
 * Problem (Section 2.1): sort n int32 keys that all lie in a known range
 * [minVal, maxVal) of size R = maxVal - minVal into nondecreasing order.  The
 * sort is unstable; for keys alone every correct output is the same array, so
 * results are bit-exact.
 *
 * Method (Section 3, Algorithms 4-7): the value range is cut into tiles of at
 * most T values; each tile's histogram is built in shared memory (Algorithm 5),
 * prefix-summed into a local CDF, offset by the number of smaller keys
 * (Algorithm 6), and the output is generated from the local CDFs alone
 * (Algorithm 7) -- the input is never rescanned after the histogram.
 *
 * Conventions for every entry point
 *  - Pointers named `in`, `out`, `workspace` are DEVICE pointers (cudaMalloc,
 *    torch CUDA tensors, ...) on the current CUDA device; the caller owns them.
 *  - `in` and `out` must be 4-byte aligned; any further alignment is handled.
 *    `in == out` (in-place) is allowed because output generation never reads
 *    the input; any other overlap is rejected with RTCDF_ERR_INVALID_ARG.
 *  - Calls are asynchronous and ordered on `stream` (0 = legacy default
 *    stream).  Errors detectable on the host return immediately and enqueue
 *    nothing.  Errors found by the device (a key outside [minVal, maxVal), a
 *    bounded wait that ran out) are recorded in a device status word that
 *    rtcdf_status_get / rtcdf_ws_status_get read; `out` is then unspecified.
 *    The status word is sticky: once a bounded wait has run out, sorts on
 *    that workspace write no output until the status has been read.
 *  - minVal >= INT32_MIN and maxVal <= 2^31 (the range lies in the int32 key
 *    space), 1 <= R <= RTCDF_MAX_R, n < 2^32.  n == 0 returns RTCDF_OK.
 *  - No entry point synchronizes the device except rtcdf_status_get /
 *    rtcdf_ws_status_get and first-use workspace growth outside stream
 *    capture (which only orders on `stream`).
 *  - No C++ exception leaves the library: a failed host allocation is
 *    returned as RTCDF_ERR_NO_MEMORY.
 */
#ifndef RTCDF_H
#define RTCDF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *rtcdf_stream_t; /* same handle as cudaStream_t */

typedef enum {
    RTCDF_OK = 0,
    RTCDF_ERR_INVALID_ARG = 1,      /* null pointer, misalignment, overlap, bad size */
    RTCDF_ERR_RANGE = 2,            /* R <= 0, R > RTCDF_MAX_R, or range outside int32 */
    RTCDF_ERR_KEY_OUT_OF_RANGE = 3, /* device status: a key outside [minVal, maxVal) */
    RTCDF_ERR_CUDA = 4,             /* a CUDA runtime call failed */
    RTCDF_ERR_NO_MEMORY = 5,        /* device or host allocation failed, or workspace too small */
    RTCDF_ERR_TIMEOUT = 6           /* device status: a bounded wait gave up */
} rtcdf_status;

/* Device status bits reported by rtcdf_status_get / rtcdf_ws_status_get
 * (and RTCDF_DEV_BAD_SEGMENT, below, for segmented sorts planned on the
 * device). */
#define RTCDF_DEV_KEY_OUT_OF_RANGE 0x1
#define RTCDF_DEV_TIMEOUT 0x2

/* Largest supported range size.  Ranges wider than one shared-memory tile are
 * handled by several tiles (Algorithm 4, m = ceil(R / T) > 1). */
#define RTCDF_MAX_R (1LL << 24)

/*
 * rtcdf_sort -- sort n keys of `in` into `out` (Algorithm 4 end to end).
 * Uses a workspace owned by the library, cached per (device, stream) and grown
 * on demand (stream-ordered allocation; inside CUDA graph capture it must
 * already be large enough, see rtcdf_reserve).  Calls on the same stream reuse
 * one workspace; calls on different streams never share one.
 */
rtcdf_status rtcdf_sort(const int32_t *in, int32_t *out, uint64_t n, int64_t minVal,
                        int64_t maxVal, rtcdf_stream_t stream);

/*
 * rtcdf_reserve -- grow the library-owned workspace of `stream` so that any
 * later rtcdf_sort with range size <= max_R runs without allocating (needed
 * before capturing rtcdf_sort into a CUDA graph).
 */
rtcdf_status rtcdf_reserve(int64_t max_R, rtcdf_stream_t stream);

/*
 * Workspace sizing for the caller-owned variant.  The workspace holds the
 * histogram H[0..R-1] (Algorithm 5), the run table derived from the local CDFs
 * and tile offsets (Algorithm 6), the scan's lookback state and the status
 * word: O(R) bytes, independent of n (Section 3.2: workspace O(R + m)).
 */
rtcdf_status rtcdf_workspace_size(int64_t R, size_t *bytes);

/*
 * rtcdf_sort_ws -- rtcdf_sort with a caller-owned device workspace of
 * `ws_bytes` >= rtcdf_workspace_size(R).  No allocation happens inside, so the
 * call can be captured in a CUDA graph.  The workspace must be zero-filled
 * before its first use (cudaMemsetAsync(workspace, 0, ws_bytes, stream)).
 * Every call leaves the parts that must start at zero (control block, lookback
 * state, histogram) zeroed again -- the run tables it also holds are written
 * before they are read -- so one workspace serves any sequence of sorts whose
 * ranges it is large enough for; the status word is sticky until read.  Calls
 * that share one workspace must be ordered (same stream or events).
 */
rtcdf_status rtcdf_sort_ws(const int32_t *in, int32_t *out, uint64_t n, int64_t minVal,
                           int64_t maxVal, void *workspace, size_t ws_bytes,
                           rtcdf_stream_t stream);

/*
 * rtcdf_status_get -- wait for `stream`, then return in *device_status the
 * RTCDF_DEV_* bits recorded by sorts on the library-owned workspaces of
 * `stream` (rtcdf_sort's and rtcdf_sort_batched's) since the last read, and
 * clear them.  Returns RTCDF_ERR_TIMEOUT when a bounded wait ran out (checked
 * first: the other findings of that sort are then unreliable), else
 * RTCDF_ERR_INVALID_ARG for segment metadata that broke its bounds, else
 * RTCDF_ERR_KEY_OUT_OF_RANGE when a key lay outside its range.
 */
rtcdf_status rtcdf_status_get(rtcdf_stream_t stream, int32_t *device_status);

/* Same for a caller-owned workspace. */
rtcdf_status rtcdf_ws_status_get(void *workspace, rtcdf_stream_t stream,
                                 int32_t *device_status);

/* Human-readable name of a status code (static string). */
const char *rtcdf_status_str(rtcdf_status status);

/*
 * Launch parameters of one sort (Section 3.3, Table "Kernel launch
 * configurations"): tile width T (values per range tile, m = ceil(R / T)),
 * histogram CTAs per tile (g_hist), threads per histogram CTA, output CTAs.
 * Zero in a field means "choose automatically".
 */
typedef struct {
    int32_t tile_width;      /* T; 0 = largest that fits shared memory */
    int32_t hist_ctas_per_tile;
    int32_t hist_threads;    /* 256, 512 or 1024 */
    int32_t fill_ctas;
    int32_t fill_threads;    /* 256, 512 or 1024 */
    int32_t fill_chunk;      /* output positions per output CTA; when > 0 it
                                replaces fill_ctas (the count then follows n) */
    int32_t reserved[2];
} rtcdf_params;

/* The parameters rtcdf_sort would use for (n, R) on the current device
 * (tuning table first, then the built-in rules). */
rtcdf_status rtcdf_plan(uint64_t n, int64_t R, rtcdf_params *params);

/*
 * Tuning table.  rtcdf_sort, rtcdf_sort_ws, rtcdf_sort_host and
 * rtcdf_sort_static take their launch parameters from a per-process table
 * keyed by the range class ceil(log2 R) and the input-size class of n; a
 * range/size pair with no entry, or an entry whose parameters do not fit the
 * current device, falls back to the built-in rules (zero fields of an entry
 * also keep the built-in choice).  The table starts as the one compiled into
 * the library (measured on GB300 with rtcdf_autotune); rtcdf_tune_set replaces
 * it, rtcdf_tune_reset restores the compiled-in one.  The input distribution
 * is not a key: the sort cannot know it before its histogram, so the tuner
 * ranks candidates over several distributions (Section 4.1's rule).
 */
#define RTCDF_TUNE_N_SMALL 0   /* n < 2^20 */
#define RTCDF_TUNE_N_MEDIUM 1  /* 2^20 <= n < 2^26 */
#define RTCDF_TUNE_N_LARGE 2   /* n >= 2^26 */

typedef struct {
    int32_t log2_R;        /* ceil(log2 R): 0 for R = 1, up to 24 */
    int32_t n_class;       /* RTCDF_TUNE_N_* */
    rtcdf_params params;
} rtcdf_tune_entry;

/* The size class of n (RTCDF_TUNE_N_*). */
int32_t rtcdf_tune_n_class(uint64_t n);
/* Replace the table (count == 0 empties it: built-in rules only).  Entries are
 * copied; a later entry with the same key wins.  Thread-safe. */
rtcdf_status rtcdf_tune_set(const rtcdf_tune_entry *entries, int32_t count);
/* Restore the table compiled into the library. */
rtcdf_status rtcdf_tune_reset(void);
/* Copy up to `capacity` entries of the current table; *count = table size. */
rtcdf_status rtcdf_tune_get(rtcdf_tune_entry *entries, int32_t capacity, int32_t *count);

/*
 * rtcdf_autotune -- time candidate launch parameters and pick one by the
 * paper's rule (Section 4.1): for every condition (case) c and candidate k the
 * median of `reps` sorts t(c, k) is measured with CUDA events on `stream`;
 * r(c, k) = t(c, k) / min_k' t(c, k') is its time normalised to the fastest
 * candidate for that condition, and the candidate with the smallest geometric
 * mean of r over all conditions wins.
 *
 * cases[i].in / .out are device arrays of .n keys in [.minVal, .maxVal);
 * `workspace` (256-byte aligned, zero-filled before first use, then kept as
 * rtcdf_sort_ws keeps it) holds at least rtcdf_workspace_size(max R) bytes.  Host outputs:
 * times_ms[c * num_candidates + k] (median ms; -1 if candidate k cannot run
 * case c on this device), geomean[k] (HUGE_VAL for a candidate that cannot
 * run every case), *best.  Synchronises `stream`; not capturable.  Returns
 * RTCDF_ERR_INVALID_ARG if no candidate runs every case, and the device
 * status (e.g. RTCDF_ERR_KEY_OUT_OF_RANGE) if a sort recorded one.
 */
typedef struct {
    const int32_t *in;
    int32_t *out;
    uint64_t n;
    int64_t minVal;
    int64_t maxVal;
} rtcdf_tune_case;

rtcdf_status rtcdf_autotune(const rtcdf_tune_case *cases, int32_t num_cases,
                            const rtcdf_params *candidates, int32_t num_candidates, int32_t reps,
                            void *workspace, size_t ws_bytes, float *times_ms, double *geomean,
                            int32_t *best, rtcdf_stream_t stream);

/*
 * rtcdf_sort_ex -- rtcdf_sort_ws with explicit launch parameters (for tuning
 * and tests).  `params` may be NULL (tuning table, then built-in rules); when
 * given it is used as is (its zero fields take the built-in rules, the tuning
 * table is not consulted).  When `debug` is non-NULL it receives
 * device copies of the intermediates (device pointers, caller-owned):
 *   debug->tile_hist[0..R-1]  H after the histogram step (Algorithm 5)
 *   debug->cdf[0..R-1]        O[t] + local CDF, i.e. the inclusive CDF
 *   debug->tile_offset[0..m-1] O (Algorithm 6)
 * Any of the three may be NULL, as may each stage event.
 */
typedef struct {
    uint32_t *tile_hist;
    uint32_t *cdf;
    uint32_t *tile_offset;
    /* Optional cudaEvent_t handles (caller-created, may be NULL) recorded on
     * `stream` before the histogram kernel, after it, after the scan and after
     * the output kernel: per-stage CUDA-event timing on the launching stream. */
    void *stage_events[4];
} rtcdf_debug;

rtcdf_status rtcdf_sort_ex(const int32_t *in, int32_t *out, uint64_t n, int64_t minVal,
                           int64_t maxVal, const rtcdf_params *params, void *workspace,
                           size_t ws_bytes, const rtcdf_debug *debug,
                           rtcdf_stream_t stream);

/*
 * Sharded sort of one array over several GPUs (or several slices on one).
 * The sorted output depends on the global histogram alone (Section 3.1,
 * Algorithms 4 and 7; Section 3.2, Lemma 3: value v occupies positions
 * [sum_{u<v} c_u, sum_{u<=v} c_u)), so P ranks that each hold a contiguous
 * slice of the input run:
 *   1. rtcdf_hist_accumulate on their slice into a counts array zeroed
 *      beforehand (Algorithm 5 for every tile);
 *   2. one sum all-reduce of the R counts over the ranks (the caller's
 *      collective, e.g. NCCL on uint32/int32: sums wrap identically);
 *   3. rtcdf_fill_from_counts for their own window [pos_begin, pos_end) of
 *      the sorted array (Algorithm 6's offsets and Algorithm 7's output for
 *      those positions only).
 * No keys cross ranks.  Both calls are asynchronous and stream-ordered, and
 * allocate nothing.
 *
 * rtcdf_hist_accumulate -- counts[x] += #{i : in[i] - minVal == x} for the n
 * keys of `in` (device), x in [0, R).  `counts` is a DEVICE array of R uint32
 * (4-byte aligned) that the caller zeroes before the first slice; calls on
 * several slices add up.  Keys outside [minVal, maxVal) are counted nowhere
 * (the shortfall is found by rtcdf_fill_from_counts).  Errors:
 * RTCDF_ERR_RANGE as for rtcdf_sort; RTCDF_ERR_INVALID_ARG for a null or
 * misaligned pointer, n >= 2^32, or `in` overlapping `counts`.
 */
rtcdf_status rtcdf_hist_accumulate(const int32_t *in, uint64_t n, int64_t minVal, int64_t maxVal,
                                   uint32_t *counts, rtcdf_stream_t stream);

/*
 * rtcdf_fill_from_counts -- write positions [pos_begin, pos_end) of the sorted
 * array whose global counts are `counts` (device, R uint32 adding up to
 * total_n): out[p - pos_begin] = minVal + min{v : sum_{u<=v} c_u > p}.
 * `counts` is only read.  `workspace` is as for rtcdf_sort_ws (at least
 * rtcdf_workspace_size(R) bytes, 256-byte aligned, zero-filled before its
 * first use, left ready for the next call; calls sharing it must be
 * ordered).  Counts that do not add up to total_n (a key outside the range
 * on some rank) set RTCDF_DEV_KEY_OUT_OF_RANGE in the workspace's status word
 * (rtcdf_ws_status_get), and `out` is then unspecified.  Errors:
 * RTCDF_ERR_RANGE as for rtcdf_sort; RTCDF_ERR_INVALID_ARG for total_n >=
 * 2^32, pos_begin > pos_end, pos_end > total_n, a null or misaligned pointer,
 * or `out` overlapping `counts` or the workspace; RTCDF_ERR_NO_MEMORY for a
 * workspace that is too small.  An empty window returns RTCDF_OK at once.
 */
rtcdf_status rtcdf_fill_from_counts(const uint32_t *counts, uint64_t total_n, int64_t minVal,
                                    int64_t maxVal, uint64_t pos_begin, uint64_t pos_end, int32_t *out,
                                    void *workspace, size_t ws_bytes, rtcdf_stream_t stream);

/*
 * rtcdf_sort_host -- rtcdf_sort with HOST buffers: `in` and `out` point to
 * host memory (page-locked for the transfers to overlap anything; pageable
 * works but copies synchronously).  The keys are uploaded in 16 MB chunks on
 * a library-owned copy stream, the histogram of each chunk runs on a
 * library-owned compute stream as soon as it has landed, the scan and output
 * follow, and the result is downloaded on a second copy stream, which
 * overlaps the next call's upload and histogram.  Device buffers are
 * library-owned (two sets per device and stream, used in turn).  `in` is read
 * as of the call (the host must have finished writing it; the upload is not
 * ordered after earlier work on `stream`).  When `stream` completes, `out`
 * holds the result; `in` must not be modified before then.  Device status:
 * rtcdf_status_get does not cover these calls; keys outside [minVal, maxVal)
 * leave `out` unspecified.  The library-owned buffers (sized for the largest
 * n seen), streams and events live until the process exits.  Errors:
 * RTCDF_ERR_RANGE and RTCDF_ERR_INVALID_ARG as for rtcdf_sort (checked
 * before any CUDA call); RTCDF_ERR_NO_MEMORY when device buffers cannot be
 * allocated; RTCDF_ERR_CUDA when creating the streams or events, a copy, an
 * event record or a stream wait fails.
 */
rtcdf_status rtcdf_sort_host(const int32_t *in, int32_t *out, uint64_t n, int64_t minVal,
                             int64_t maxVal, rtcdf_stream_t stream);

/*
 * Segmented sort: many independent arrays ("segments") sorted by three
 * launches whatever their number.  Segment s is
 * in[seg_offsets[s] .. seg_offsets[s+1]), its keys lie in
 * [seg_minVal[s], seg_maxVal[s]) (R_s <= 2^20), and it is written sorted to
 * the same positions of `out`.  The method per segment is Algorithms 4-7
 * unchanged; segments with fewer than 65536 keys (and R_s <= 55296) are
 * sorted entirely inside one CTA -- of the second launch when R_s is at most
 * rtcdf_batch_params.small_scan_max_R (default 16000), else of the first --
 * and larger ones are split into histogram items (first launch), 4096-bin
 * scan chunks (second launch) and output items (third launch).
 *
 * rtcdf_batch_plan_create builds the work list from HOST arrays
 * (seg_offsets: S+1 entries, nondecreasing; seg_minVal / seg_maxVal: S) and
 * uploads it (this allocates and synchronises; do it once per segment layout).
 * rtcdf_sort_batched_ws then runs it with no host work and no allocation
 * (capturable in a CUDA graph; replay with new keys of the same shapes); its
 * workspace (rtcdf_batch_workspace_size bytes, 256-byte aligned) belongs to
 * one plan: zero-fill it before its first use with that plan; every run leaves
 * the parts that must start at zero (histograms, lookback state, control
 * block) zeroed again, so the plan can be replayed on it, but its other parts
 * hold per-run tables, so zero-fill it again before using it with another
 * plan.  The status word is sticky until read with rtcdf_batch_status_get.
 * rtcdf_sort_batched_host is the one-shot form over host arrays: plan,
 * allocate, run, read the status, free -- it synchronises.
 *
 * rtcdf_sort_batched (below the plan API) takes the metadata in DEVICE memory
 * and plans on the device: asynchronous and stream-ordered, no host
 * synchronisation.
 */
typedef struct rtcdf_batch_plan rtcdf_batch_plan;

typedef struct {
    uint32_t num_segments;
    uint32_t small_segments;   /* sorted inside one CTA */
    uint32_t large_segments;   /* split into work items */
    uint32_t work_items;       /* CTAs over the three launches */
    uint32_t workers;          /* CTAs of the first launch resident at once (one per SM) */
    uint32_t reserved;
    uint64_t total_keys;
    uint64_t workspace_bytes;
} rtcdf_batch_info;

rtcdf_status rtcdf_batch_plan_create(const int64_t *seg_offsets, const int64_t *seg_minVal,
                                     const int64_t *seg_maxVal, int32_t num_segments,
                                     rtcdf_batch_plan **plan);
/* Work-item sizes of a segmented sort (zero = built-in choice). */
typedef struct {
    int32_t hist_chunk;   /* keys per histogram item of a large segment (>= 4096; default 524288) */
    int32_t fill_chunk;   /* output positions per output item (>= 4096; default 65536) */
    int32_t small_max_n;  /* longest segment sorted inside one CTA (<= 65535; default 65535) */
    int32_t small_scan_max_R; /* in-CTA segments with R up to this are sorted by 256-thread CTAs
                                 of the scan launch, wider ones by 1024-thread CTAs of the first
                                 launch (1 .. 16768; default 16000) */
    int32_t small_by_time;    /* 0 or 1 (default): a segment the two limits above would sort
                                 inside one CTA of the scan launch is split into work items
                                 instead when its estimated in-CTA sort time exceeds the scan
                                 launch's (only when the plan has large segments); -1: the
                                 limits alone decide */
    int32_t reserved[3];
} rtcdf_batch_params;

/* rtcdf_batch_plan_create with explicit work-item sizes (`params` may be NULL). */
rtcdf_status rtcdf_batch_plan_create_ex(const int64_t *seg_offsets, const int64_t *seg_minVal,
                                        const int64_t *seg_maxVal, int32_t num_segments,
                                        const rtcdf_batch_params *params,
                                        rtcdf_batch_plan **plan);
rtcdf_status rtcdf_batch_plan_destroy(rtcdf_batch_plan *plan);
rtcdf_status rtcdf_batch_workspace_size(const rtcdf_batch_plan *plan, size_t *bytes);
rtcdf_status rtcdf_batch_plan_info(const rtcdf_batch_plan *plan, rtcdf_batch_info *info);
rtcdf_status rtcdf_sort_batched_ws(const rtcdf_batch_plan *plan, const int32_t *in, int32_t *out,
                                   void *workspace, size_t ws_bytes, rtcdf_stream_t stream);
rtcdf_status rtcdf_batch_status_get(void *workspace, rtcdf_stream_t stream,
                                    int32_t *device_status);

/*
 * rtcdf_sort_batched_profiled -- rtcdf_sort_batched_ws that also records where
 * the launches spend their time, per work-item kind k (0 histogram, 1 in-CTA
 * segment, 2 scan chunk, 3 output): `profile` is a device array of
 * RTCDF_BATCH_PROFILE_WORDS uint64, initialised by the caller to zero except
 * words 8..11, initialised to UINT64_MAX; afterwards
 *   profile[k]      sum over items (CTAs) of their duration (ns)
 *   profile[4 + k]  items processed
 *   profile[8 + k]  earliest item start   (device global timer, ns)
 *   profile[12 + k] latest item end       (device global timer, ns)
 *   profile[16 + k] ns spent waiting for other items (scan chunks: the
 *                   lookback over earlier chunks), included in profile[k].
 * The instrumentation adds a few timer reads and atomics per item.
 */
#define RTCDF_BATCH_PROFILE_WORDS 20
rtcdf_status rtcdf_sort_batched_profiled(const rtcdf_batch_plan *plan, const int32_t *in,
                                         int32_t *out, void *workspace, size_t ws_bytes,
                                         uint64_t *profile, rtcdf_stream_t stream);
/* One-shot segmented sort over HOST metadata (the plan API's arrays):
 * plans on the host, allocates, runs, reads the status and frees; it
 * synchronises `stream` and returns the device status. */
rtcdf_status rtcdf_sort_batched_host(const int32_t *in, int32_t *out, const int64_t *seg_offsets,
                                     const int64_t *seg_minVal, const int64_t *seg_maxVal,
                                     int32_t num_segments, rtcdf_stream_t stream);

/*
 * rtcdf_sort_batched -- segmented sort with the segment metadata in DEVICE
 * memory (e.g. written by earlier kernels on `stream`): int64 seg_offsets
 * (S+1 entries, nondecreasing, seg_offsets[0] >= 0), seg_minVal and
 * seg_maxVal (S entries), 8-byte aligned.  Each segment s is sorted as in the
 * plan API (Section 2.1's problem per segment, Algorithms 4-7).  The work
 * lists are built on the device by two planner kernels, so the call enqueues
 * five launches and returns: asynchronous, stream-ordered, no host
 * synchronisation.
 *
 * The caller states bounds the metadata must keep: num_segments (S),
 * max_total_keys (>= seg_offsets[S]; also the length checked for in/out
 * overlap) and max_R (every R_s <= max_R <= 2^20).  The workspace is sized
 * from them (rtcdf_batch_device_workspace_size): about 12 bytes x max_R per
 * segment plus O(S + max_total_keys / 65536) -- every segment owns a slot for
 * a range of max_R.  Metadata that breaks a bound (or a limit of the
 * segmented sort) sets RTCDF_DEV_BAD_SEGMENT in the device status word and
 * nothing is written; the status calls then return RTCDF_ERR_INVALID_ARG.
 *
 * rtcdf_sort_batched uses a library-owned workspace per (device, stream),
 * grown on demand by stream-ordered allocation (inside CUDA graph capture it
 * must already be large enough: rtcdf_batch_reserve); rtcdf_status_get reads
 * its status.  rtcdf_sort_batched_device_ws takes a caller workspace
 * (256-byte aligned, zero-filled before its first use, left ready for the
 * next call of any layout within the same bounds; calls sharing it must be
 * ordered): no allocation, so it can be captured in a CUDA graph and replayed
 * with new keys AND new segment metadata.  Its status: rtcdf_batch_status_get.
 * Host-side errors (returned at once, nothing enqueued): RTCDF_ERR_INVALID_ARG
 * for S < 0, max_total_keys >= 2^40, null or misaligned pointers, in/out
 * partial overlap; RTCDF_ERR_RANGE for max_R outside 1..2^20;
 * RTCDF_ERR_NO_MEMORY for a workspace that is too small (or cannot grow).
 */
#define RTCDF_DEV_BAD_SEGMENT 0x4
rtcdf_status rtcdf_batch_device_workspace_size(int32_t num_segments, uint64_t max_total_keys, int64_t max_R,
                                               size_t *bytes);
rtcdf_status rtcdf_sort_batched_device_ws(const int32_t *in, int32_t *out, const int64_t *seg_offsets,
                                          const int64_t *seg_minVal, const int64_t *seg_maxVal,
                                          int32_t num_segments, uint64_t max_total_keys, int64_t max_R,
                                          void *workspace, size_t ws_bytes, rtcdf_stream_t stream);
rtcdf_status rtcdf_sort_batched(const int32_t *in, int32_t *out, const int64_t *seg_offsets,
                                const int64_t *seg_minVal, const int64_t *seg_maxVal, int32_t num_segments,
                                uint64_t max_total_keys, int64_t max_R, rtcdf_stream_t stream);
/* Grow the library-owned workspace of `stream` for these bounds (needed
 * before capturing rtcdf_sort_batched in a CUDA graph). */
rtcdf_status rtcdf_batch_reserve(int32_t num_segments, uint64_t max_total_keys, int64_t max_R,
                                 rtcdf_stream_t stream);

/*
 * Continuous-batching server.  A trace of sort requests (arrival times
 * relative to its start) is served from one device slab of `budget_bytes`:
 * requests are admitted in arrival order when their slot (input + output,
 * 8n bytes) fits, their keys are written into the slot by `fill` (for
 * synthetic traces: rtcdf_gen_keys has this signature), and admitted requests
 * are launched as soon as one of `num_streams` streams is free -- a request of
 * at least `single_min_keys` keys alone through the single-array pipeline, all
 * other pending requests together in one segmented launch (at most
 * `max_batch`; a lone pending request takes the single-array pipeline).  Arrivals keep being admitted while launches run, and a
 * request's memory is released when its launch completes.  With `digests`
 * set, each result carries an order-dependent 64-bit digest of its sorted
 * output (sum over positions i of SplitMix64's finaliser applied to
 * (i << 32 | out[i]), mod 2^64).  Times are seconds from the trace start.
 * rtcdf_serve_sequential serves the same trace one request at a time
 * (rtcdf_sort_ws on one stream, waiting for each) as the comparison.
 * Both allocate, synchronise and return when every request is done.
 *
 * Errors: RTCDF_ERR_INVALID_ARG for a null config or fill function or a null
 * array with count > 0 (rtcdf_serve_trace also: num_streams outside 1..16,
 * max_batch < 1); RTCDF_ERR_RANGE for a request with R outside 1..2^20 or
 * n >= 2^32 (rtcdf_serve_sequential: R outside 1..RTCDF_MAX_R);
 * RTCDF_ERR_NO_MEMORY when the slab, the digests or the pinned staging cannot
 * be allocated; RTCDF_ERR_CUDA when a CUDA call fails or `fill` returns
 * nonzero.  On an error the trace stops: requests not yet served keep status
 * -1, and every resource the call created is released.  A request that can
 * never fit the budget gets status RTCDF_ERR_NO_MEMORY and the trace goes on.
 */
typedef int (*rtcdf_fill_fn)(int32_t *dev_out, uint64_t n, uint64_t first, int64_t minVal,
                             int64_t R, int dist, uint64_t seed, rtcdf_stream_t stream);

typedef struct {
    uint64_t budget_bytes;
    int32_t num_streams;        /* 1..16 */
    int32_t max_batch;          /* requests per segmented launch */
    uint64_t single_min_keys;   /* requests this large run alone */
    rtcdf_fill_fn fill;
    int32_t digests;            /* nonzero: compute result digests */
    int32_t max_large_inflight; /* launches of requests with at least single_min_keys
                                   keys in flight at once (0 = num_streams): large
                                   sorts are bandwidth-bound, so running them one
                                   after another keeps their latency while small
                                   batches still overlap them */
    int32_t *const *outputs;    /* NULL, or `count` HOST pointers (entries may be
                                   NULL): request i's sorted keys are copied to
                                   outputs[i] (n int32) once its launch has
                                   completed, before its memory is released.  The
                                   copy is synchronous and holds up the serving
                                   loop: leave this NULL when timing. */
    int32_t large_priority;     /* nonzero: requests of at least single_min_keys
                                   keys are written and sorted on streams of the
                                   device's highest stream priority (batches keep
                                   the default priority), so a large sort runs
                                   about as fast as alone while batches fill in */
    int32_t reserved2;
    int32_t fill_at_launch;     /* nonzero: a request's keys are written by `fill`
                                   on its launch's stream right before the sort
                                   (as rtcdf_serve_sequential does); 0: at
                                   admission, on separate streams, overlapping
                                   the sorts in flight */
    int32_t large_queue_burst;  /* > 0: max_large_inflight applies only while fewer
                                   than this many large requests wait; with more
                                   waiting, large launches may use every stream */
} rtcdf_server_config;

typedef struct {
    uint64_t n;
    int64_t minVal, maxVal;     /* R <= 2^20 */
    int32_t dist;               /* passed to fill */
    int32_t reserved;
    uint64_t seed;              /* passed to fill */
    double arrival_s;           /* nondecreasing along the trace */
} rtcdf_request;

typedef struct {
    double admit_s, launch_s, done_s;
    uint64_t digest;
    int32_t status;             /* 0 done, -1 not served (the call failed), else an rtcdf_status */
    int32_t batch_id;           /* launch that served the request */
} rtcdf_result;

typedef struct {
    double makespan_s;
    uint64_t total_keys;
    uint64_t launches_batched, launches_single, batched_requests;
    uint64_t peak_bytes;
    int32_t max_inflight;
    int32_t reserved;
} rtcdf_serve_stats;

rtcdf_status rtcdf_serve_trace(const rtcdf_server_config *cfg, const rtcdf_request *reqs,
                               int64_t count, rtcdf_result *results, rtcdf_serve_stats *stats);
rtcdf_status rtcdf_serve_sequential(const rtcdf_server_config *cfg, const rtcdf_request *reqs,
                                    int64_t count, rtcdf_result *results, rtcdf_serve_stats *stats);

/*
 * rtcdf_sort_static -- the sort without any allocation, for callers that
 * cannot allocate device memory: code running under another framework's
 * memory manager that owns all device memory, serving loops whose memory
 * budget is fixed up front, and hot paths that cannot afford the implicit
 * synchronisation of an allocation.  The paper has no counterpart; this is an
 * integration entry point.
 *
 * The caller passes `in` and `out` as for rtcdf_sort.  The scratch the sort
 * needs beyond them lives in one array of RTCDF_STATIC_WS_BYTES bytes compiled
 * into the library; every GPU that loads the library holds that array until
 * the process exits.  Ranges wider than RTCDF_STATIC_MAX_R return
 * RTCDF_ERR_RANGE.  Nothing is allocated and no allocating routine is called.
 *
 * The first call on a device looks up the array's device address (once per
 * device, on the current device).  All calls on a device share the array and
 * it keeps what the last call left, so each call clears the part that must
 * start at zero; calls that overlap on the GPU (unordered streams) race and
 * must not be issued.  This
 * entry point reports no device-detected error: neither a key outside
 * [minVal, maxVal) nor a bounded wait that ran out (which only overlapping
 * calls can cause) reaches the caller, and `out` is then unspecified.  The
 * caller guarantees that every key lies in [minVal, maxVal) and that calls on
 * one device are ordered.
 */
#define RTCDF_STATIC_MAX_R (1LL << 16)
#define RTCDF_STATIC_WS_BYTES (1u << 20)
rtcdf_status rtcdf_sort_static(const int32_t *in, int32_t *out, uint64_t n, int64_t minVal,
                               int64_t maxVal, rtcdf_stream_t stream);

/* Library version string. */
const char *rtcdf_version(void);

#ifdef __cplusplus
}
#endif

#endif /* RTCDF_H */
