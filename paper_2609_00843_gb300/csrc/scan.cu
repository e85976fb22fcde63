// Local CDFs and tile offsets (Section 3.1 and Algorithm 6) in one pass.
//
// The paper scans each tile's slice of H in place (one CTA per tile), then a
// single thread accumulates the tile totals into O[t].  Here one decoupled
// lookback scan over H[0..R-1] produces, for every value v,
//     O[t] + C_t[v - b_t] = sum_{u<=v} c_u,
// i.e. the tile offset plus the local CDF (Lemmas 1-2), which is exactly the
// exclusive end of v's output interval (Lemma 3).  In the same pass each value
// with c_v > 0 is given a run index k (a second prefix count packed in the
// high half of the same 64-bit scan word) and the run table
//     run_end[k] = sum_{u<=v} c_u,   run_val[k] = minVal + v
// is written, so that output generation never walks empty values.  The value
// containing the first position of every output CTA is recorded in start_run.
// H is zeroed as it is read, leaving the workspace ready for the next sort.
//
// Chunks of kScanChunk bins are handed out by an atomic ticket so that a chunk
// only ever waits for chunks already owned by running CTAs; every wait is
// bounded by kMaxSpin and records kDevTimeout when it gives up.
#include "rtcdf_internal.h"

namespace rtcdf {

// Lookback word: bits 0..31 count prefix, bits 32..56 run-count prefix,
// bits 62..63 state.
constexpr uint64_t kStateAgg = 1ull << 62;
constexpr uint64_t kStateIncl = 2ull << 62;
constexpr uint64_t kValueMask = (1ull << 62) - 1;

__device__ __forceinline__ void store_release(uint64_t *p, uint64_t v) {
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ uint64_t load_acquire(const uint64_t *p) {
    uint64_t v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ uint64_t warp_incl_scan(uint64_t x, int lane) {
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        uint64_t y = __shfl_up_sync(0xffffffffu, x, d);
        if (lane >= d) x += y;
    }
    return x;
}

__device__ __forceinline__ uint64_t warp_sum(uint64_t x) {
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) x += __shfl_xor_sync(0xffffffffu, x, d);
    return x;
}

__global__ void __launch_bounds__(kScanThreads) scan_kernel(ScanArgs a) {
    __shared__ uint32_t s_chunk;
    __shared__ uint64_t s_warp[kScanThreads / 32];
    __shared__ uint64_t s_prefix;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    if (tid == 0) s_chunk = atomicAdd(&a.ctl->scan_ticket, 1u);
    __syncthreads();
    const uint32_t chunk = s_chunk;
    const uint32_t base = chunk * kScanChunk + tid * kScanItems;

    // Load four counts (H is padded to whole chunks) and zero them behind us.
    uint4 h4 = *reinterpret_cast<const uint4 *>(a.H + base);
    *reinterpret_cast<uint4 *>(a.H + base) = make_uint4(0, 0, 0, 0);
    uint32_t c[kScanItems] = {h4.x, h4.y, h4.z, h4.w};
    if (a.dbg_hist) {
#pragma unroll
        for (int i = 0; i < kScanItems; i++)
            if (base + i < a.R) a.dbg_hist[base + i] = c[i];
    }

    // Thread-local inclusive scan of (run flag, count) pairs.
    uint64_t incl[kScanItems];
    uint64_t run = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; i++) {
        run += ((uint64_t)(c[i] > 0) << 32) | c[i];
        incl[i] = run;
    }
    // Block scan of the thread totals.
    uint64_t winc = warp_incl_scan(run, lane);
    if (lane == 31) s_warp[warp] = winc;
    __syncthreads();
    if (warp == 0) {
        uint64_t wt = s_warp[lane];
        uint64_t wi = warp_incl_scan(wt, lane);
        s_warp[lane] = wi - wt;  // exclusive prefix of each warp
        uint64_t total = __shfl_sync(0xffffffffu, wi, 31);

        // Decoupled lookback across chunks (warp 0 only).
        uint64_t prefix = 0;
        if (chunk == 0) {
            if (lane == 0) store_release(&a.state[0], kStateIncl | total);
        } else {
            if (lane == 0) store_release(&a.state[chunk], kStateAgg | total);
            int64_t look = (int64_t)chunk - 1;
            uint32_t spins = 0;
            bool timed_out = false;
            while (true) {
                int64_t idx = look - lane;
                uint64_t st = (idx >= 0) ? load_acquire(&a.state[idx]) : (kStateIncl | 0ull);
                // Wait until every lane's predecessor has published something.
                while (!__all_sync(0xffffffffu, (st >> 62) != 0)) {
                    if (++spins > kMaxSpin) { timed_out = true; break; }
                    __nanosleep(64);
                    if ((st >> 62) == 0) st = load_acquire(&a.state[idx]);
                }
                if (timed_out) break;
                unsigned incl_mask = __ballot_sync(0xffffffffu, (st >> 62) == 2);
                if (incl_mask) {
                    int first = __ffs(incl_mask) - 1;  // nearest inclusive predecessor
                    uint64_t v = (lane <= first) ? (st & kValueMask) : 0;
                    prefix += warp_sum(v);
                    break;
                }
                prefix += warp_sum(st & kValueMask);
                look -= 32;
            }
            if (timed_out && lane == 0) atomicOr(&a.ctl->status, kDevTimeout);
            if (lane == 0) store_release(&a.state[chunk], kStateIncl | (prefix + total));
        }
        if (lane == 0) s_prefix = prefix;
    }
    __syncthreads();

    const uint64_t texcl = s_prefix + s_warp[warp] + (winc - run);
#pragma unroll
    for (int i = 0; i < kScanItems; i++) {
        const uint32_t v = base + i;
        if (v >= a.R) break;
        const uint64_t p = texcl + incl[i];
        const uint32_t cnt_end = (uint32_t)p;           // sum_{u<=v} c_u
        const uint32_t runs = (uint32_t)(p >> 32);      // values u<=v with c_u > 0
        if (a.dbg_cdf) a.dbg_cdf[v] = cnt_end;
        if (a.dbg_offset && (v % a.T) == 0) a.dbg_offset[v / a.T] = cnt_end - c[i];
        if (v == a.R - 1) a.ctl->num_runs = runs;
        if (c[i] == 0) continue;
        const uint32_t k = runs - 1;
        a.run_end[k] = cnt_end;
        a.run_val[k] = (int32_t)((uint32_t)a.minVal + v);
        // Output CTAs whose first position lies in [cnt_end - c, cnt_end):
        // CTA 0 starts at 0, CTA j >= 1 at head + j * fill_chunk.
        const uint64_t s = cnt_end - c[i], e = cnt_end;
        if (s == 0) a.start_run[0] = k;
        if (e > a.head) {
            uint64_t lo = (s > a.head) ? (s - a.head + a.fill_chunk - 1) / a.fill_chunk : 1;
            if (lo < 1) lo = 1;
            uint64_t hi = (e - a.head + a.fill_chunk - 1) / a.fill_chunk;
            if (hi > a.fill_ctas) hi = a.fill_ctas;
            for (uint64_t j = lo; j < hi; j++) a.start_run[j] = k;
        }
    }
}

cudaError_t launch_scan(const ScanArgs &a, cudaStream_t s) {
    scan_kernel<<<a.chunks, kScanThreads, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace rtcdf
