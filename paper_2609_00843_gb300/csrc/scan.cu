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
// is written, so that output generation never walks empty values.
//
// Each output CTA needs the run holding its first position.  Every scan CTA
// keeps its chunk's CDF in shared memory and, for the output CTAs whose first
// position falls inside the chunk's positions, finds that run with the rule of
// Algorithm 7 (smallest value whose CDF exceeds the position) by binary
// search -- a handful of steps per output CTA whatever the distribution.
//
// H is zeroed as it is read, leaving the workspace ready for the next sort.
// Chunks of kScanChunk bins are handed out by an atomic ticket so that a chunk
// only ever waits for chunks already owned by running CTAs; every wait is
// bounded by kMaxSpin and records kDevTimeout when it gives up.  The total
// count is compared with n: every in-range key is counted by exactly one tile,
// so a shortfall means some key lies outside [minVal, maxVal).
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

// Exclusive prefix of the chunks before `chunk` (decoupled lookback, warp 0).
__device__ uint64_t lookback(uint64_t *state, uint32_t chunk, uint64_t total, int lane, Ctl *ctl) {
    if (chunk == 0) {
        if (lane == 0) store_release(&state[0], kStateIncl | total);
        return 0;
    }
    if (lane == 0) store_release(&state[chunk], kStateAgg | total);
    uint64_t prefix = 0;
    int64_t look = (int64_t)chunk - 1;
    uint32_t spins = 0;
    bool timed_out = false;
    while (true) {
        const int64_t idx = look - lane;
        uint64_t st = (idx >= 0) ? load_acquire(&state[idx]) : kStateIncl;
        // Wait until every lane's predecessor has published something.
        while (!__all_sync(0xffffffffu, (st >> 62) != 0)) {
            if (++spins > kMaxSpin) { timed_out = true; break; }
            __nanosleep(64);
            if ((st >> 62) == 0) st = load_acquire(&state[idx]);
        }
        if (timed_out) break;
        const unsigned incl_mask = __ballot_sync(0xffffffffu, (st >> 62) == 2);
        if (incl_mask) {
            const int first = __ffs(incl_mask) - 1;  // nearest inclusive predecessor
            prefix += warp_sum((lane <= first) ? (st & kValueMask) : 0);
            break;
        }
        prefix += warp_sum(st & kValueMask);
        look -= 32;
    }
    if (timed_out && lane == 0) atomicOr(&ctl->status, kDevTimeout);
    if (lane == 0) store_release(&state[chunk], kStateIncl | (prefix + total));
    return prefix;
}

__global__ void __launch_bounds__(kScanThreads) scan_kernel(ScanArgs a) {
    __shared__ uint32_t s_chunk;
    __shared__ uint64_t s_warp[kScanThreads / 32];
    __shared__ uint64_t s_prefix;
    __shared__ uint32_t s_cdf[kScanChunk];   // sum_{u<=v} c_u for the chunk's values
    __shared__ uint32_t s_runs[kScanChunk];  // non-empty values u <= v
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    // Launched as a programmatic dependent of the histogram.  The chunk ticket
    // does not depend on it (the counter was reset by the previous sort's
    // output kernel, which finished before this sort's histogram began), so
    // it is taken first; then wait until the histogram grid has finished and
    // its writes are visible, and let the output kernel be scheduled (it
    // waits for this grid in the same way).
    const bool single = (a.chunks == 1);  // R <= kScanChunk: no lookback at all
    if (!single) {
        if (tid == 0) s_chunk = atomicAdd(&a.ctl->scan_ticket, 1u);
        __syncthreads();
    }
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;");
    const uint32_t chunk = single ? 0u : s_chunk;
    // A ticket past the last chunk only happens with a workspace whose ticket
    // was not zero (not cleared, or shared by unordered calls): take no chunk
    // and record kDevTimeout, since the chunk that ticket stood for is never
    // published (its successor's lookback would run out too) and the output
    // kernel must not trust this sort's run table.
    if (chunk >= a.chunks) {
        if (tid == 0) atomicOr(&a.ctl->status, kDevTimeout);
        return;
    }
    const uint32_t cbase = chunk * kScanChunk;
    const uint32_t base = cbase + tid * kScanItems;

    // Four counts (H is padded to whole chunks), zeroed behind us.
    uint4 *h4p = reinterpret_cast<uint4 *>(a.H + base);
    const uint4 h4 = *h4p;
    *h4p = make_uint4(0, 0, 0, 0);
    const uint32_t c[kScanItems] = {h4.x, h4.y, h4.z, h4.w};
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
    // Block scan of the thread totals, then the chunk prefix.
    const uint64_t winc = warp_incl_scan(run, lane);
    if (lane == 31) s_warp[warp] = winc;
    __syncthreads();
    if (warp == 0) {
        const uint64_t wt = s_warp[lane];
        const uint64_t wi = warp_incl_scan(wt, lane);
        s_warp[lane] = wi - wt;  // exclusive prefix of each warp
        const uint64_t total = __shfl_sync(0xffffffffu, wi, 31);
        const uint64_t prefix = single ? 0 : lookback(a.state, chunk, total, lane, a.ctl);
        if (lane == 0) s_prefix = prefix;
    }
    __syncthreads();

    const uint64_t chunk_prefix = s_prefix;
    const uint64_t texcl = chunk_prefix + s_warp[warp] + (winc - run);
#pragma unroll
    for (int i = 0; i < kScanItems; i++) {
        const uint32_t v = base + i;
        const uint64_t p = texcl + incl[i];
        const uint32_t cnt_end = (uint32_t)p;       // sum_{u<=v} c_u
        const uint32_t runs = (uint32_t)(p >> 32);  // values u<=v with c_u > 0
        s_cdf[tid * kScanItems + i] = cnt_end;
        s_runs[tid * kScanItems + i] = runs;
        if (v >= a.R) continue;
        if (a.dbg_cdf) a.dbg_cdf[v] = cnt_end;
        if (a.dbg_offset && (v % a.T) == 0) a.dbg_offset[v / a.T] = cnt_end - c[i];
        if (v == a.R - 1) {
            a.ctl->num_runs = runs;
            if (cnt_end != (uint32_t)a.n) atomicOr(&a.ctl->status, kDevKeyOutOfRange);
        }
        if (c[i] > 0) {
            a.run_end[runs - 1] = cnt_end;
            a.run_val[runs - 1] = (int32_t)((uint32_t)a.minVal + v);
        }
    }
    __syncthreads();

    // Output CTA j starts at P0(j): P0(0) = pos_base, P0(j) = pos_base + head
    // + j * fill_chunk, all inside [pos_base, pos_end).  The chunk's values
    // cover positions [pos_lo, pos_hi); only the part inside the written
    // window can hold a CTA's first position.
    const uint32_t pos_lo = max((uint32_t)chunk_prefix, a.pos_base);
    const uint32_t pos_hi = min(s_cdf[kScanChunk - 1], a.pos_end);
    if (pos_hi > pos_lo) {
        const uint32_t fc = (uint32_t)a.fill_chunk, head = a.head, pb = a.pos_base;
        // First CTA j with P0(j) >= pb + l (P0 is increasing in j).
        auto first_cta_at_or_after = [&](uint32_t l) -> uint32_t {
            if (l == 0) return 0u;
            if ((uint64_t)l <= (uint64_t)head + fc) return 1u;
            return (uint32_t)(((uint64_t)l - head + fc - 1) / fc);
        };
        const uint32_t j_lo = first_cta_at_or_after(pos_lo - pb);
        const uint32_t j_hi = min(first_cta_at_or_after(pos_hi - pb), a.fill_ctas);
        for (uint32_t j = j_lo + tid; j < j_hi; j += kScanThreads) {
            const uint32_t p0 = pb + ((j == 0) ? 0u : head + j * fc);
            // Smallest value of the chunk whose CDF exceeds p0 (Algorithm 7's rule).
            int lo = 0, hi = kScanChunk - 1;
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (s_cdf[mid] > p0) hi = mid; else lo = mid + 1;
            }
            a.start_run[j] = s_runs[lo] - 1;
        }
    }
}

cudaError_t launch_scan(const ScanArgs &a, cudaStream_t s) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(a.chunks);
    cfg.blockDim = dim3(kScanThreads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, scan_kernel, a);
}

}  // namespace rtcdf
