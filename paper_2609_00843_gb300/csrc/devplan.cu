// Segmented sort with the segment metadata in device memory, planned on the
// device: asynchronous, stream-ordered, no host synchronisation and no
// allocation, so a caller whose segment layout is produced by earlier kernels
// can enqueue the sort -- or capture it in a CUDA graph and replay it with new
// layouts -- without a round trip through the host.
//
// Each segment is still sorted by Algorithms 4-7 (Section 3); the plan is the
// same three work lists as the host planner's (batch_api.cu), built by one
// kernel: each CTA classifies 1024 segments (the rules of devplan_segment,
// batched.h), scans their item counts per list, gets the counts of the
// segments before its own from the CTAs before it (a decoupled lookback over
// CTAs taken in start order, every wait bounded), and writes its segments'
// descriptors and items.  The lists sit at fixed offsets (the bounds of the
// lists before them), so no CTA needs the totals to place its items; the
// last CTA writes the lists' lengths.
// The three launches then run over these lists (seg_*_kernel<true>); their
// lengths are known only on the device, so the launches take items by
// ticket: the first launch from a fixed grid of one CTA per SM looping
// over the three histogram lists (largest items first) with the in-CTA
// segments spread evenly among them; the scan launch one item per CTA (the
// narrow in-CTA segments by CTA index, then the chunks by ticket) and the
// output launch one CTA per item, from grids sized by the lists' bounds, the
// CTAs past a list's length exiting at once (about half a microsecond per
// thousand, measured).
//
// The workspace is sized from host-known bounds (segment count, total keys,
// widest range).  Every segment owns a fixed slot for its histogram, lookback
// state and run tables, so the regions that must be zero when a run starts
// (histogram, lookback state) are where the next run expects them whatever
// its layout.  Metadata that breaks the bounds sets RTCDF_DEV_BAD_SEGMENT and
// the lists are left empty: nothing is written.
#include <algorithm>
#include <cstring>
#include <map>
#include <mutex>
#include <utility>

#include "../../include/rtcdf.h"
#include "batched.h"

namespace rtcdf {

namespace {

size_t align64(uint64_t words) { return (size_t)((words + 63) / 64 * 64); }

// Largest scan-launch grid: its CTAs past the lists only exit, about half a
// microsecond per thousand (so at most about 35 us of them).
constexpr uint64_t kScanGridCap = 1u << 16;

struct DevPlanArgs {
    const int64_t *offs, *mn, *mx;
    DevBounds b;
    BatchTuning t;
    uint32_t *ws;
    DevLayout L;
};

// Lookback record of a planner CTA: state (0 none, 1 its own counts
// published, 2 the counts of every segment up to its last published), its own
// counts and the inclusive ones -- per list, and the number of segments that
// broke the bounds.  Each array is written once, before the state that
// announces it, so a reader never sees one being overwritten.
constexpr uint32_t kLookCounts = kNumLists + 1;  // every list, and the segments that broke the bounds
struct DevLook {
    uint32_t flag;
    uint32_t own[kLookCounts];
    uint32_t incl[kLookCounts];
    uint32_t pad[32 - 1 - 2 * kLookCounts];
};
static_assert(sizeof(DevLook) == 128, "lookback record is 32 words");
constexpr uint32_t kLookWords = sizeof(DevLook) / 4;

__device__ __forceinline__ void st_release_u32(uint32_t *p, uint32_t v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ uint32_t ld_acquire_u32(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__global__ void __launch_bounds__(1024) devplan_kernel(DevPlanArgs p) {
    __shared__ uint32_t s_ex[kNumLists][1024];  // exclusive prefix of each list's counts within the CTA
    __shared__ uint32_t s_warp[kNumLists][32];
    __shared__ uint32_t s_tot[kLookCounts], s_base[kLookCounts];
    __shared__ uint32_t s_blk;
    __shared__ int s_bad;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    BatchCtl *ctl = reinterpret_cast<BatchCtl *>(p.ws + p.L.ctl);
    BatchSeg *segs = reinterpret_cast<BatchSeg *>(p.ws + p.L.segs);
    BatchItem *items = reinterpret_cast<BatchItem *>(p.ws + p.L.items);
    DevLook *look = reinterpret_cast<DevLook *>(p.ws + p.L.look);
    // CTAs in start order, so a CTA only waits for CTAs already running.
    if (tid == 0) {
        s_blk = atomicAdd(&ctl->plan_ticket, 1u);
        s_bad = 0;
    }
    __syncthreads();
    const uint32_t blk = s_blk;
    if (blk >= p.L.look_blocks) {
        // Only with a workspace whose ticket was not zero: the lists of this
        // run are incomplete, so the output launch must not trust them.
        if (tid == 0) atomicOr(&ctl->status, kDevTimeout);
        return;
    }
    if (blk == 0 && tid == 0) {  // the previous run has finished (stream order)
        ctl->first_ticket = 0;
        ctl->scan_ticket = 0;
    }
    const uint32_t S = p.b.S, s = blk * 1024 + tid;
    DevSegCount c{};
    BatchSeg g{};
    if (s < S && !devplan_segment(p.offs[s], p.offs[s + 1], p.mn[s], p.mx[s], p.b, p.t, &g, &c)) s_bad = 1;
    const uint32_t *v = c.v;
    uint32_t inc[kNumLists];
#pragma unroll
    for (int f = 0; f < kNumLists; f++) {
        inc[f] = v[f];
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, inc[f], d);
            if (lane >= d) inc[f] += y;
        }
        if (lane == 31) s_warp[f][warp] = inc[f];
    }
    __syncthreads();
    if (warp < kNumLists) {
        const uint32_t x = s_warp[warp][lane];
        uint32_t xi = x;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, xi, d);
            if (lane >= d) xi += y;
        }
        s_warp[warp][lane] = xi - x;
        if (lane == 31) s_tot[warp] = xi;
    }
    __syncthreads();
#pragma unroll
    for (int f = 0; f < kNumLists; f++) s_ex[f][tid] = s_warp[f][warp] + inc[f] - v[f];
    if (tid == 0) {
        s_tot[kNumLists] = s_bad ? 1u : 0u;
        // Counts of the segments before this CTA's: publish its own, then
        // add the predecessors' until one has published its inclusive counts.
        uint32_t pre[kLookCounts] = {};
        if (blk > 0) {
            for (int i = 0; i < kLookCounts; i++) look[blk].own[i] = s_tot[i];
            st_release_u32(&look[blk].flag, 1u);
            int64_t j = (int64_t)blk - 1;
            uint32_t spins = 0;
            while (j >= 0) {
                uint32_t f = ld_acquire_u32(&look[j].flag);
                while (f == 0) {
                    if (++spins > kMaxSpin) break;
                    __nanosleep(64);
                    f = ld_acquire_u32(&look[j].flag);
                }
                if (f == 0) {  // the wait ran out: mark the plan unusable
                    atomicOr(&ctl->status, kDevTimeout);
                    pre[kNumLists] += 1;
                    break;
                }
                const uint32_t *src = f == 2 ? look[j].incl : look[j].own;
                for (int i = 0; i < kLookCounts; i++) pre[i] += src[i];
                if (f == 2) break;
                j--;
            }
        }
        for (int i = 0; i < kLookCounts; i++) {
            s_base[i] = pre[i];
            look[blk].incl[i] = pre[i] + s_tot[i];
        }
        st_release_u32(&look[blk].flag, 2u);
    }
    __syncthreads();
    if (s < S) {
        if (g.m > 0) {
            const size_t slot = p.L.slots + (size_t)s * p.L.slot_words;
            g.hist_off = slot;
            g.state_off = slot + p.L.slot_state;
            g.run_end_off = slot + p.L.slot_run_end;
            g.run_val_off = slot + p.L.slot_run_val;
            // the segment's output items, both lists: consecutive start-run slots
            g.start_run_off = p.L.start + s_base[kListFill0] + s_ex[kListFill0][tid] + s_base[kListFill1] +
                              s_ex[kListFill1][tid];
        }
        segs[s] = g;
    }
    __syncthreads();  // the descriptors are read back below, by other threads of the CTA
    // This CTA's items of every list, all threads together: the owner of the
    // k-th is the last segment whose prefix is at most k.
    const uint32_t nseg = min(1024u, S - blk * 1024);
    for (uint32_t f = 0; f < kNumLists; f++) {
        for (uint32_t k = tid; k < s_tot[f]; k += 1024) {
            uint32_t lo = 0, hi = nseg;
            while (hi - lo > 1) {
                const uint32_t mid = (lo + hi) >> 1;
                if (s_ex[f][mid] <= k) lo = mid;
                else hi = mid;
            }
            const uint32_t sg = blk * 1024 + lo;
            items[devplan_pos(p.L.lb, f, (uint64_t)s_base[f] + k)] = devplan_item(f, sg, k - s_ex[f][lo], segs[sg], p.t);
        }
    }
    if (blk == p.L.look_blocks - 1 && tid == 0) {
        uint32_t t[kLookCounts];
        for (int i = 0; i < kLookCounts; i++) t[i] = s_base[i] + s_tot[i];
        DevPlanHdr *h = reinterpret_cast<DevPlanHdr *>(p.ws + p.L.hdr);
        const uint64_t nh = (uint64_t)t[kListHist0] + t[kListHist1] + t[kListHist2];
        const uint64_t ns = (uint64_t)t[kListScan0] + t[kListScan1], nf = (uint64_t)t[kListFill0] + t[kListFill1];
        // The bounds hold by construction; checked anyway, so that a list
        // never outgrows its region.
        const DevListBounds &lb = p.L.lb;
        bool bad = t[kNumLists] > 0 || nh > lb.hist || t[kListSmall1] > p.b.S || ns > lb.scan ||
                   t[kListSmall2] > lb.small2 || nf > lb.fill;
        h->n_hist = bad ? 0 : (uint32_t)nh;
        h->n_small1 = bad ? 0 : t[kListSmall1];
        h->n_first = bad ? 0 : (uint32_t)nh + t[kListSmall1];
        h->n_scan = bad ? 0 : (uint32_t)ns;
        h->n_small2 = bad ? 0 : t[kListSmall2];
        h->n_fill = bad ? 0 : (uint32_t)nf;
        for (uint32_t c = 0; c < kHistClasses; c++) h->n_hist_class[c] = bad ? 0 : t[kListHist0 + c];
        for (uint32_t c = 0; c < 2; c++) {
            h->n_scan_class[c] = bad ? 0 : t[kListScan0 + c];
            h->n_fill_class[c] = bad ? 0 : t[kListFill0 + c];
        }
        if (bad) atomicOr(&ctl->status, kDevBadSegment);
    }
}

// Library-owned workspaces of rtcdf_sort_batched, per (device, stream).
struct BatchCache {
    void *ptr = nullptr;
    size_t bytes = 0;
};
std::mutex g_bmu;
std::map<std::pair<int, cudaStream_t>, BatchCache> g_bws;

rtcdf_status check_bounds(int32_t S, uint64_t N, int64_t max_R, DevBounds *b) {
    if (S < 0) return RTCDF_ERR_INVALID_ARG;
    if (max_R < 1 || max_R > (int64_t)kBatchMaxR) return RTCDF_ERR_RANGE;
    if (N >= (1ull << 40)) return RTCDF_ERR_INVALID_ARG;
    *b = DevBounds{(uint32_t)S, (uint32_t)max_R, N};
    return RTCDF_OK;
}

rtcdf_status grow_cache(cudaStream_t s, size_t need, void **ptr, size_t *bytes) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return RTCDF_ERR_CUDA;
    std::lock_guard<std::mutex> lk(g_bmu);
    BatchCache *c = nullptr;
    try {
        c = &g_bws[std::make_pair(dev, s)];
    } catch (...) {
        return RTCDF_ERR_NO_MEMORY;
    }
    if (c->bytes < need) {
        cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(s, &cap) != cudaSuccess) return RTCDF_ERR_CUDA;
        if (cap != cudaStreamCaptureStatusNone) return RTCDF_ERR_NO_MEMORY;
        void *p = nullptr;
        if (cudaMallocAsync(&p, need, s) != cudaSuccess) return RTCDF_ERR_NO_MEMORY;
        if (cudaMemsetAsync(p, 0, need, s) != cudaSuccess) {
            cudaFreeAsync(p, s);
            return RTCDF_ERR_CUDA;
        }
        void *old = c->ptr;
        c->ptr = p;
        c->bytes = need;
        if (old && cudaFreeAsync(old, s) != cudaSuccess) return RTCDF_ERR_CUDA;
    }
    *ptr = c->ptr;
    *bytes = c->bytes;
    return RTCDF_OK;
}

}  // namespace

int devplan_layout(const DevBounds &b, const BatchTuning &t, DevLayout *L) {
    if (b.max_R < 1 || b.max_R > kBatchMaxR) return RTCDF_ERR_RANGE;
    const uint64_t S = b.S, N = b.max_total_keys;
    const uint64_t cpr = (b.max_R + kBatchScanChunk - 1) / kBatchScanChunk;  // scan chunks per segment
    const uint64_t m_max = (b.max_R + kBatchTileMax - 1) / kBatchTileMax;
    DevListBounds &lb = L->lb;
    lb.hist = (N / t.hist_chunk + S) * m_max;
    lb.first = kHistClasses * lb.hist + S;
    lb.scan = S * cpr;
    lb.small2 = S;
    lb.fill = N / t.fill_chunk + S;
    L->item_bound = lb.first + 2 * lb.scan + lb.small2 + 2 * lb.fill;
    size_t w = 0;
    L->ctl = w;      w += 64;
    L->hdr = w;      w += 64;
    L->segctl = w;   w += align64(S * sizeof(BatchSegCtl) / 4);
    L->segs = w;     w += align64(S * sizeof(BatchSeg) / 4);
    L->look_blocks = (uint32_t)((S + 1023) / 1024);
    L->look = w;     w += align64((uint64_t)L->look_blocks * kLookWords);
    L->items = w;    w += align64(L->item_bound * sizeof(BatchItem) / 4);
    L->start = w;    w += align64(lb.fill);
    L->slots = w;
    L->slot_state = align64(cpr * kBatchScanChunk);
    L->slot_run_end = L->slot_state + align64(2 * cpr);
    L->slot_run_val = L->slot_run_end + align64(b.max_R);
    L->slot_words = L->slot_run_val + align64(b.max_R);
    w += S * L->slot_words;
    L->total_words = w;
    return 0;
}

int devplan_host(const int64_t *offs, const int64_t *mn, const int64_t *mx, const DevBounds &b,
                 const BatchTuning &t, const DevLayout &L, std::vector<BatchSeg> *segs,
                 std::vector<DevPfx> *pfx, DevPlanHdr *hdr, std::vector<BatchItem> *items) {
    const uint32_t S = b.S;
    segs->assign(S, BatchSeg{});
    pfx->assign((size_t)S + 1, DevPfx{});
    memset(hdr, 0, sizeof(*hdr));
    items->clear();
    DevPfx run{};
    for (uint32_t s = 0; s < S; s++) {
        DevSegCount c;
        BatchSeg g;
        if (!devplan_segment(offs[s], offs[s + 1], mn[s], mx[s], b, t, &g, &c)) return RTCDF_ERR_INVALID_ARG;
        (*pfx)[s] = run;
        if (g.m > 0) {
            const size_t slot = L.slots + (size_t)s * L.slot_words;
            g.hist_off = slot;
            g.state_off = slot + L.slot_state;
            g.run_end_off = slot + L.slot_run_end;
            g.run_val_off = slot + L.slot_run_val;
            g.start_run_off = L.start + run.v[kListFill0] + run.v[kListFill1];
        }
        (*segs)[s] = g;
        for (uint32_t f = 0; f < kNumLists; f++) run.v[f] += c.v[f];
    }
    (*pfx)[S] = run;
    hdr->n_hist = run.v[kListHist0] + run.v[kListHist1] + run.v[kListHist2];
    for (uint32_t c = 0; c < kHistClasses; c++) hdr->n_hist_class[c] = run.v[kListHist0 + c];
    for (uint32_t c = 0; c < 2; c++) {
        hdr->n_scan_class[c] = run.v[kListScan0 + c];
        hdr->n_fill_class[c] = run.v[kListFill0 + c];
    }
    hdr->n_small1 = run.v[kListSmall1];
    hdr->n_first = hdr->n_hist + hdr->n_small1;
    hdr->n_scan = run.v[kListScan0] + run.v[kListScan1];
    hdr->n_small2 = run.v[kListSmall2];
    hdr->n_fill = run.v[kListFill0] + run.v[kListFill1];
    if (hdr->n_hist > L.lb.hist || hdr->n_small1 > S || hdr->n_scan > L.lb.scan || hdr->n_small2 > L.lb.small2 ||
        hdr->n_fill > L.lb.fill)
        return RTCDF_ERR_INVALID_ARG;
    // The items at the positions the planner writes them: each list in
    // segment order from its own base (devplan_pos); unused positions stay
    // zero here.
    items->assign(L.item_bound, BatchItem{});
    for (uint32_t list = 0; list < kNumLists; list++)
        for (uint32_t s = 0; s < S; s++)
            for (uint32_t k = (*pfx)[s].v[list]; k < (*pfx)[s + 1].v[list]; k++)
                (*items)[devplan_pos(L.lb, list, k)] = devplan_item(list, s, k - (*pfx)[s].v[list], (*segs)[s], t);
    return 0;
}

// The batch workspace of `stream` on the current device, if rtcdf_sort_batched
// made one (for rtcdf_status_get).
void *batch_stream_workspace(cudaStream_t s) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
    std::lock_guard<std::mutex> lk(g_bmu);
    auto it = g_bws.find(std::make_pair(dev, s));
    return it == g_bws.end() ? nullptr : it->second.ptr;
}

}  // namespace rtcdf

using namespace rtcdf;

extern "C" {

rtcdf_status rtcdf_batch_device_workspace_size(int32_t num_segments, uint64_t max_total_keys, int64_t max_R,
                                               size_t *bytes) {
    if (!bytes) return RTCDF_ERR_INVALID_ARG;
    DevBounds b;
    rtcdf_status st = check_bounds(num_segments, max_total_keys, max_R, &b);
    if (st) return st;
    DevLayout L;
    if (const int rc = devplan_layout(b, BatchTuning(), &L)) return (rtcdf_status)rc;
    *bytes = L.total_words * 4;
    return RTCDF_OK;
}

rtcdf_status rtcdf_sort_batched_device_ws(const int32_t *in, int32_t *out, const int64_t *seg_offsets,
                                          const int64_t *seg_minVal, const int64_t *seg_maxVal,
                                          int32_t num_segments, uint64_t max_total_keys, int64_t max_R,
                                          void *workspace, size_t ws_bytes, rtcdf_stream_t stream) {
    DevBounds b;
    rtcdf_status st = check_bounds(num_segments, max_total_keys, max_R, &b);
    if (st) return st;
    if (num_segments == 0 || max_total_keys == 0) return RTCDF_OK;
    if (!in || !out || !seg_offsets || !seg_minVal || !seg_maxVal || !workspace) return RTCDF_ERR_INVALID_ARG;
    if (((uintptr_t)in & 3) || ((uintptr_t)out & 3) || ((uintptr_t)workspace & 255) ||
        ((uintptr_t)seg_offsets & 7) || ((uintptr_t)seg_minVal & 7) || ((uintptr_t)seg_maxVal & 7))
        return RTCDF_ERR_INVALID_ARG;
    if ((const void *)in != (const void *)out) {
        const uintptr_t x = (uintptr_t)in, y = (uintptr_t)out, n = max_total_keys * 4;
        if (x < y + n && y < x + n) return RTCDF_ERR_INVALID_ARG;
    }
    const BatchTuning tun;
    DevLayout L;
    if (const int rc = devplan_layout(b, tun, &L)) return (rtcdf_status)rc;
    if (ws_bytes < L.total_words * 4) return RTCDF_ERR_NO_MEMORY;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return RTCDF_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    uint32_t *ws = (uint32_t *)workspace;
    DevPlanArgs p;
    p.offs = seg_offsets;
    p.mn = seg_minVal;
    p.mx = seg_maxVal;
    p.b = b;
    p.t = tun;
    p.ws = ws;
    p.L = L;
    devplan_kernel<<<L.look_blocks, 1024, 0, s>>>(p);
    if (cudaGetLastError() != cudaSuccess) return RTCDF_ERR_CUDA;
    BatchArgs a;
    a.in = in;
    a.out = out;
    a.segs = reinterpret_cast<const BatchSeg *>(ws + L.segs);
    a.items = reinterpret_cast<const BatchItem *>(ws + L.items);
    // (the n_* of a device-built plan are unused: the lengths are on the
    // device, the positions come from dev_bounds)
    a.n_first = a.n_scan = a.n_small2 = a.n_fill = 0;
    a.num_segs = b.S;
    a.ws_u32 = ws;
    a.ctl = reinterpret_cast<BatchCtl *>(ws + L.ctl);
    a.seg_ctl = reinterpret_cast<BatchSegCtl *>(ws + L.segctl);
    a.dev_counts = ws + L.hdr;  // n_first, n_scan, n_small2, n_fill, n_hist, n_small1, n_hist_class[3]
    a.dev_bounds[0] = L.lb.hist;
    a.dev_bounds[1] = L.lb.first;
    a.dev_bounds[2] = L.lb.scan;
    a.dev_bounds[3] = L.lb.small2;
    a.dev_bounds[4] = L.lb.fill;
    a.plan_look = ws + L.look;
    a.plan_look_words = L.look_blocks * kLookWords;
    // The first launch: one resident CTA per SM taking items by ticket; the
    // scan launch: one CTA per item of the lists' bounds, at most
    // kScanGridCap (CTAs loop when the lists are longer); the output launch:
    // one CTA per item of the list's bound.
    if (L.lb.fill > 0x7fffffffull) return RTCDF_ERR_INVALID_ARG;
    const uint32_t first = (uint32_t)std::min<uint64_t>(L.lb.first, (uint64_t)sms);
    const uint32_t scan = (uint32_t)std::min<uint64_t>(L.lb.scan + L.lb.small2, kScanGridCap);
    const uint32_t fill = (uint32_t)L.lb.fill;
    if (launch_batched_dev(a, std::max(first, 1u), std::max(scan, 1u), std::max(fill, 1u), s) != cudaSuccess)
        return RTCDF_ERR_CUDA;
    return RTCDF_OK;
}

rtcdf_status rtcdf_batch_reserve(int32_t num_segments, uint64_t max_total_keys, int64_t max_R,
                                 rtcdf_stream_t stream) try {
    size_t need = 0;
    rtcdf_status st = rtcdf_batch_device_workspace_size(num_segments, max_total_keys, max_R, &need);
    if (st) return st;
    void *ws = nullptr;
    size_t bytes = 0;
    return grow_cache((cudaStream_t)stream, std::max<size_t>(need, 256), &ws, &bytes);
} catch (...) {
    return RTCDF_ERR_NO_MEMORY;
}

rtcdf_status rtcdf_sort_batched(const int32_t *in, int32_t *out, const int64_t *seg_offsets,
                                const int64_t *seg_minVal, const int64_t *seg_maxVal, int32_t num_segments,
                                uint64_t max_total_keys, int64_t max_R, rtcdf_stream_t stream) try {
    size_t need = 0;
    rtcdf_status st = rtcdf_batch_device_workspace_size(num_segments, max_total_keys, max_R, &need);
    if (st) return st;
    if (num_segments == 0 || max_total_keys == 0) return RTCDF_OK;
    if (!in || !out || !seg_offsets || !seg_minVal || !seg_maxVal) return RTCDF_ERR_INVALID_ARG;
    void *ws = nullptr;
    size_t bytes = 0;
    st = grow_cache((cudaStream_t)stream, std::max<size_t>(need, 256), &ws, &bytes);
    if (st) return st;
    return rtcdf_sort_batched_device_ws(in, out, seg_offsets, seg_minVal, seg_maxVal, num_segments,
                                        max_total_keys, max_R, ws, bytes, stream);
} catch (...) {
    return RTCDF_ERR_NO_MEMORY;
}

}  // extern "C"
