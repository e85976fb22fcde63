// rtcdf_sort_host: the sort with HOST input and output buffers.
//
// Keys cross to the device in chunks on a copy stream; the histogram of each
// chunk (Algorithm 5) runs on a library-owned compute stream as soon as the
// chunk has landed, so the transfer and the histogram overlap.  The local-CDF
// scan and the output generation (Algorithms 6-7) follow, and the sorted keys
// go back on a second copy stream.  The caller's stream only waits for that
// download: the next call's upload and histogram do not wait for it, so a
// sequence of calls keeps both directions of the host link busy at once
// (uploads of call i + 1 under the download of call i).  Device buffers are
// owned by the library: two sets per (device, stream), used alternately and
// guarded by events.
#include <algorithm>
#include <map>
#include <mutex>

#include "../../include/rtcdf.h"
#include "rtcdf_internal.h"

namespace rtcdf {
// rtcdf_api.cu
rtcdf_status host_pipeline_hist(const int32_t *in, uint64_t n, int64_t minVal, uint32_t R, void *ws,
                                size_t ws_bytes, cudaStream_t s);
rtcdf_status host_pipeline_finish(int32_t *out, uint64_t n, int64_t minVal, uint32_t R, void *ws,
                                  size_t ws_bytes, cudaStream_t s);
}  // namespace rtcdf

using namespace rtcdf;

namespace {

struct BufSet {
    int32_t *in = nullptr, *out = nullptr;
    uint64_t cap = 0;
    cudaEvent_t in_free = nullptr;   // the histogram that last read `in` is done
    cudaEvent_t out_free = nullptr;  // the download that last read `out` is done
};

struct HostCtx {
    bool ready = false;              // streams and events below all exist
    BufSet set[2];
    int next = 0;
    void *ws = nullptr;
    size_t ws_bytes = 0;
    cudaStream_t up = nullptr, down = nullptr, comp = nullptr;
    cudaEvent_t ev_done = nullptr;   // sort finished on the compute stream
    cudaEvent_t ev_chunk = nullptr;  // a chunk has landed (re-recorded per chunk)
};

std::mutex g_host_mu;
std::map<std::pair<int, cudaStream_t>, HostCtx> g_host;

constexpr uint64_t kChunk = 1ull << 22;  // keys per uploaded chunk (16 MB)

// Creates the context's streams and events, all or none.
bool init_ctx(HostCtx &c) {
    cudaStream_t *streams[3] = {&c.up, &c.down, &c.comp};
    cudaEvent_t *events[6] = {&c.ev_done, &c.ev_chunk, &c.set[0].in_free, &c.set[0].out_free,
                              &c.set[1].in_free, &c.set[1].out_free};
    bool ok = true;
    for (cudaStream_t *p : streams)
        ok = ok && cudaStreamCreateWithFlags(p, cudaStreamNonBlocking) == cudaSuccess;
    for (cudaEvent_t *p : events) ok = ok && cudaEventCreateWithFlags(p, cudaEventDisableTiming) == cudaSuccess;
    // Both sets start free: their events complete with the (empty) compute stream.
    for (BufSet &b : c.set)
        ok = ok && cudaEventRecord(b.in_free, c.comp) == cudaSuccess &&
             cudaEventRecord(b.out_free, c.comp) == cudaSuccess;
    if (!ok) {
        for (cudaEvent_t *p : events)
            if (*p) cudaEventDestroy(*p), *p = nullptr;
        for (cudaStream_t *p : streams)
            if (*p) cudaStreamDestroy(*p), *p = nullptr;
    }
    return c.ready = ok;
}

}  // namespace

extern "C" rtcdf_status rtcdf_sort_host(const int32_t *h_in, int32_t *h_out, uint64_t n, int64_t minVal,
                                        int64_t maxVal, rtcdf_stream_t stream) {
    if (minVal < INT32_MIN || maxVal > ((int64_t)1 << 31) || maxVal <= minVal ||
        maxVal - minVal > RTCDF_MAX_R)
        return RTCDF_ERR_RANGE;
    if (n == 0) return RTCDF_OK;
    if (!h_in || !h_out || n >= (1ull << 32)) return RTCDF_ERR_INVALID_ARG;
    if (((uintptr_t)h_in & 3) || ((uintptr_t)h_out & 3)) return RTCDF_ERR_INVALID_ARG;
    const uint32_t R = (uint32_t)(maxVal - minVal);
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return RTCDF_ERR_CUDA;
    std::lock_guard<std::mutex> lk(g_host_mu);
    HostCtx *cp = nullptr;
    try {
        cp = &g_host[std::make_pair(dev, s)];
    } catch (...) {
        return RTCDF_ERR_NO_MEMORY;
    }
    HostCtx &c = *cp;
    if (!c.ready && !init_ctx(c)) return RTCDF_ERR_CUDA;
    cudaStream_t cs = c.comp;
    // Every record and wait below orders a buffer's reuse: one that fails
    // ends the call with RTCDF_ERR_CUDA.
    auto rec = [](cudaEvent_t e, cudaStream_t st) { return cudaEventRecord(e, st) == cudaSuccess; };
    auto wait = [](cudaStream_t st, cudaEvent_t e) { return cudaStreamWaitEvent(st, e, 0) == cudaSuccess; };
    // Workspace (shared by both sets: the sorts themselves are ordered on the
    // compute stream).
    const size_t need_ws = ws_required(R);
    if (c.ws_bytes < need_ws) {
        void *p = nullptr;
        if (cudaMallocAsync(&p, need_ws, cs) != cudaSuccess) return RTCDF_ERR_NO_MEMORY;
        if (cudaMemsetAsync(p, 0, need_ws, cs) != cudaSuccess) {
            cudaFreeAsync(p, cs);
            return RTCDF_ERR_CUDA;
        }
        void *old = c.ws;
        c.ws = p;
        c.ws_bytes = need_ws;
        if (old && cudaFreeAsync(old, cs) != cudaSuccess) return RTCDF_ERR_CUDA;
    }
    BufSet &b = c.set[c.next];
    c.next ^= 1;
    if (b.cap < n) {
        // Growing: wait until nothing uses the old buffers, then replace them.
        if (!wait(cs, b.in_free) || !wait(cs, b.out_free)) return RTCDF_ERR_CUDA;
        if (b.in) cudaFreeAsync(b.in, cs);
        if (b.out) cudaFreeAsync(b.out, cs);
        b.in = b.out = nullptr;
        b.cap = 0;
        if (cudaMallocAsync((void **)&b.in, n * 4, cs) != cudaSuccess ||
            cudaMallocAsync((void **)&b.out, n * 4, cs) != cudaSuccess)
            return RTCDF_ERR_NO_MEMORY;
        b.cap = n;
        if (!rec(b.in_free, cs) || !rec(b.out_free, cs)) return RTCDF_ERR_CUDA;
    }
    // Upload in chunks; the histogram of chunk k waits only for chunk k (the
    // wait takes the event as last recorded, so one event serves every chunk).
    if (!wait(c.up, b.in_free)) return RTCDF_ERR_CUDA;
    for (uint64_t k0 = 0; k0 < n; k0 += kChunk) {
        const uint64_t k1 = std::min(n, k0 + kChunk);
        if (cudaMemcpyAsync(b.in + k0, h_in + k0, (k1 - k0) * 4, cudaMemcpyHostToDevice, c.up) != cudaSuccess)
            return RTCDF_ERR_CUDA;
        if (!rec(c.ev_chunk, c.up) || !wait(cs, c.ev_chunk)) return RTCDF_ERR_CUDA;
        rtcdf_status st = host_pipeline_hist(b.in + k0, k1 - k0, minVal, R, c.ws, c.ws_bytes, cs);
        if (st) return st;
    }
    // Scan and output, once the previous download from this set is done.
    if (!rec(b.in_free, cs) || !wait(cs, b.out_free)) return RTCDF_ERR_CUDA;
    // Nobody reads this workspace's status word; clear it so that a wait that
    // ran out in an earlier call does not stop this call's output kernel.
    if (cudaMemsetAsync(c.ws, 0, 4, cs) != cudaSuccess) return RTCDF_ERR_CUDA;
    rtcdf_status st = host_pipeline_finish(b.out, n, minVal, R, c.ws, c.ws_bytes, cs);
    if (st) return st;
    if (!rec(c.ev_done, cs) || !wait(c.down, c.ev_done)) return RTCDF_ERR_CUDA;
    if (cudaMemcpyAsync(h_out, b.out, n * 4, cudaMemcpyDeviceToHost, c.down) != cudaSuccess)
        return RTCDF_ERR_CUDA;
    // The caller's stream completes only when the download has.
    if (!rec(b.out_free, c.down) || !wait(s, b.out_free)) return RTCDF_ERR_CUDA;
    return RTCDF_OK;
}
