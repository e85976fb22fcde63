// rtcdf_sort_static: the sort with a fixed scratch area compiled into the
// library, for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc (or any allocator): code that runs under
// another framework's memory manager that owns all device memory, serving
// loops with a fixed memory budget decided up front, and hot paths where the
// implicit synchronisation of an allocation is not acceptable.  They pass their
// input and output buffers; the scratch this sort needs beyond them (histogram,
// lookback state, run table) lives in one file-scope __device__ array.
//
// The array is RTCDF_STATIC_WS_BYTES bytes, enough for range sizes up to
// RTCDF_STATIC_MAX_R; every GPU that loads the library holds it until the
// process exits.  All calls on a device share it: calls that overlap on the
// GPU (different streams without ordering) race, and the array keeps whatever
// the last call left.  Each call therefore clears the part that must start at
// zero before using it.
#include <mutex>

#include "../../include/rtcdf.h"
#include "rtcdf_internal.h"

namespace rtcdf {
// Declared in rtcdf_api.cu.
rtcdf_status sort_with_workspace(const int32_t *in, int32_t *out, uint64_t n, int64_t minVal,
                                 int64_t maxVal, void *ws, size_t ws_bytes, cudaStream_t s);
}  // namespace rtcdf

using namespace rtcdf;

namespace {

constexpr size_t kStaticBytes = RTCDF_STATIC_WS_BYTES;
static_assert(kStaticBytes % 256 == 0, "static scratch is a multiple of 256 bytes");

static __device__ __align__(256) unsigned char g_static_scratch[kStaticBytes];

constexpr int kMaxDevices = 64;
std::mutex g_static_mu;
void *g_static_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device, looked up once
// per device.  In host code the array's name is only a host-side stand-in.
rtcdf_status static_scratch(void **ptr) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return RTCDF_ERR_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return RTCDF_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(g_static_mu);
    if (!g_static_ptr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || !p) return RTCDF_ERR_CUDA;
        g_static_ptr[dev] = p;
    }
    *ptr = g_static_ptr[dev];
    return RTCDF_OK;
}

}  // namespace

extern "C" rtcdf_status rtcdf_sort_static(const int32_t *in, int32_t *out, uint64_t n,
                                          int64_t minVal, int64_t maxVal, rtcdf_stream_t stream) {
    if (maxVal > minVal && (uint64_t)maxVal - (uint64_t)minVal > (uint64_t)RTCDF_STATIC_MAX_R)
        return RTCDF_ERR_RANGE;  // wider than the fixed scratch can serve
    static_assert(RTCDF_STATIC_MAX_R <= RTCDF_MAX_R, "static range limit within the general one");
    if (ws_required(RTCDF_STATIC_MAX_R) > kStaticBytes) return RTCDF_ERR_NO_MEMORY;
    void *ws = nullptr;
    rtcdf_status st = static_scratch(&ws);
    if (st) return st;
    return sort_with_workspace(in, out, n, minVal, maxVal, ws, kStaticBytes,
                               (cudaStream_t)stream);
}
