// Segmented RT-CDF: many independent arrays (segments) of uneven length n_s
// and range size R_s, each with its own [minVal_s, maxVal_s), sorted by three
// launches whatever the number of segments.  The method per segment is
// unchanged (Algorithms 4-7: tile histogram, local CDF + offsets, output from
// the CDF); what is new is the schedule:
//
//   first launch   one CTA per work item, two kinds mixed in one grid:
//                  HIST  (large segments) the histogram of a chunk of keys for
//                        one range tile (Algorithm 5), added into the
//                        segment's H -- or stored, when the tile has only one
//                        chunk;
//                  SMALL (n_s < 65536) the whole sort of the segment in one
//                        CTA: 16-bit shared-memory counters (a count never
//                        exceeds n_s < 2^16), in-place CDF, output by
//                        Algorithm 7's rule;
//   scan launch    one 256-thread CTA per 4096-bin chunk of a large
//                  segment's H: local CDF + offsets (Algorithm 6) by a
//                  decoupled lookback chained within the segment, the run
//                  table and the first run of each output item;
//   output launch  one CTA per output item: positions from the run table
//                  (Algorithm 7's rule), as in the single-array output kernel.
//
// The second and third launches are programmatic dependents of the one before
// (their launch latency overlaps its tail).  Every phase runs at full
// occupancy, and nothing waits on another CTA except the scan's lookback,
// whose chunks are handed out by a ticket in segment/chunk order (a chunk only
// waits for chunks owned by running CTAs; every wait is bounded).  The output
// launch resets the lookback state and the ticket, and the scan zeroes H as it
// reads it, so a plan can be replayed (e.g. from a CUDA graph) with no host
// work.
#include "batched.h"

namespace rtcdf {

namespace {

// Lookback word: bits 0..31 count prefix, bits 32..56 run-count prefix,
// bits 62..63 state (as in the single-array scan).
constexpr uint64_t kStAgg = 1ull << 62;
constexpr uint64_t kStIncl = 2ull << 62;
constexpr uint64_t kStValue = (1ull << 62) - 1;

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void st_release_u64(uint64_t *p, uint64_t v) {
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ uint64_t ld_acquire_u64(const uint64_t *p) {
    uint64_t v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ uint64_t warp_incl_scan_u64(uint64_t x, int lane) {
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint64_t y = __shfl_up_sync(0xffffffffu, x, d);
        if (lane >= d) x += y;
    }
    return x;
}

__device__ __forceinline__ uint64_t warp_sum_u64(uint64_t x) {
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) x += __shfl_xor_sync(0xffffffffu, x, d);
    return x;
}

// Exclusive block scan of one u32 per thread (1024 threads); s_tmp holds 33 words.
__device__ __forceinline__ uint32_t block_excl_scan_u32(uint32_t x, uint32_t *s_tmp, uint32_t *total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    uint32_t inc = x;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, inc, d);
        if (lane >= d) inc += y;
    }
    if (lane == 31) s_tmp[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        const uint32_t t = lane < nw ? s_tmp[lane] : 0u;
        uint32_t ti = t;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, ti, d);
            if (lane >= d) ti += y;
        }
        if (lane < nw) s_tmp[lane] = ti - t;
        if (lane == 31) s_tmp[nw] = ti;
    }
    __syncthreads();
    const uint32_t r = s_tmp[warp] + inc - x;
    *total = s_tmp[nw];
    __syncthreads();
    return r;
}

// S[word] += 1 (low half) or += 65536 (high half) when pred, as a predicated
// shared-memory reduction with an immediate increment: lanes that hit one
// address are combined by the hardware, so a segment of one repeated key
// costs no more than any other.
__device__ __forceinline__ void red_lo(uint32_t addr, bool pred) {
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %1, 0;\n\t@p red.shared.add.u32 [%0], 1;\n\t}"
                 ::"r"(addr), "r"((uint32_t)pred));
}
__device__ __forceinline__ void red_hi(uint32_t addr, bool pred) {
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %1, 0;\n\t@p red.shared.add.u32 [%0], 65536;\n\t}"
                 ::"r"(addr), "r"((uint32_t)pred));
}
__device__ __forceinline__ void count_key_pred(uint32_t s_base, uint32_t y, uint32_t w) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.lt.u32 p, %0, %1;\n\t"
        "@p red.shared.add.u32 [%2], 1;\n\t}"
        ::"r"(y), "r"(w), "r"(s_base + 4u * y));
}

// ---------------------------------------------------------------- SMALL
// One segment, n < 65536 keys, R <= kBatchSmallMaxR values, in one CTA.
// WIDE: one 32-bit counter per value (R words).  Otherwise 16-bit counters,
// W = ceil(R / 2) words: value v < W counts in the low half of word v, value
// v >= W in the high half of word v - W.
// `sm` holds the counters, `s_tmp` the block scan's scratch (blockDim / 32 + 1
// words).
template <bool WIDE>
__device__ void do_small_impl(const BatchArgs &a, const BatchSeg &g, uint32_t *sm, uint32_t *s_tmp) {
    const uint32_t R = g.R, n = g.n, nt = blockDim.x, tid = threadIdx.x;
    const uint32_t W = WIDE ? R : (R + 1) / 2;
    uint32_t *cnt = sm;
    for (uint32_t i = tid; i < W; i += nt) cnt[i] = 0;
    __syncthreads();
    const int32_t *in = a.in + g.off;
    const uint32_t min_u = (uint32_t)g.minVal;
    const uint32_t s_base = (uint32_t)__cvta_generic_to_shared(cnt);
    auto count1 = [&](int32_t key) {
        const uint32_t x = (uint32_t)key - min_u;
        if (WIDE) {
            count_key_pred(s_base, x, R);
        } else {
            const bool lo = x < W, hi = !lo && x < R;
            const uint32_t wv = lo ? x : x - W;
            red_lo(s_base + 4u * wv, lo);
            red_hi(s_base + 4u * wv, hi);
        }
    };
    const uint32_t lead_a = (uint32_t)(((16 - ((uintptr_t)in & 15)) & 15) / 4);
    const uint32_t lead = lead_a < n ? lead_a : n;
    const uint32_t nv = (n - lead) / 4;
    const int4 *vin = reinterpret_cast<const int4 *>(in + lead);
    uint32_t iv = tid;
    for (; iv + 3 * nt < nv; iv += 4 * nt) {
        int4 k[4];
#pragma unroll
        for (int u = 0; u < 4; u++) k[u] = __ldcs(vin + iv + u * nt);
#pragma unroll
        for (int u = 0; u < 4; u++) { count1(k[u].x); count1(k[u].y); count1(k[u].z); count1(k[u].w); }
    }
    for (; iv < nv; iv += nt) {
        const int4 k = __ldcs(vin + iv);
        count1(k.x); count1(k.y); count1(k.z); count1(k.w);
    }
    if (tid < lead) count1(in[tid]);
    for (uint32_t i = lead + 4 * nv + tid; i < n; i += nt) count1(in[i]);
    __syncthreads();
    // In-place inclusive CDF over the counters (values <= n < 2^16).  Each
    // thread takes an odd number of consecutive values, so that the 32 lanes
    // of a warp step through 32 distinct banks.
    uint16_t *c16 = reinterpret_cast<uint16_t *>(cnt);
    auto slot = [&](uint32_t v) -> uint32_t { return v < W ? 2u * v : 2u * (v - W) + 1u; };
    auto get = [&](uint32_t v) -> uint32_t { return WIDE ? cnt[v] : (uint32_t)c16[slot(v)]; };
    auto put = [&](uint32_t v, uint32_t x) {
        if (WIDE) cnt[v] = x; else c16[slot(v)] = (uint16_t)x;
    };
    const uint32_t per = ((R + nt - 1) / nt) | 1u;
    const uint32_t b0 = min(R, tid * per), b1 = min(R, b0 + per);
    uint32_t local = 0;
    for (uint32_t v = b0; v < b1; v++) local += get(v);
    uint32_t total = 0;
    const uint32_t ex = block_excl_scan_u32(local, s_tmp, &total);
    uint32_t run = ex;
    for (uint32_t v = b0; v < b1; v++) {
        run += get(v);
        put(v, run);
    }
    if (tid == 0 && total != n) atomicOr(&a.ctl->status, kDevKeyOutOfRange);
    __syncthreads();
    // Output: position p holds minVal + min{v : CDF[v] >= p + 1} (Algorithm 7).
    // 16-byte vectors: each warp takes a contiguous share, lanes interleaved
    // (one coalesced store per step); a lane's value index only moves forward
    // (a galloping search from the current value).  The positions before the
    // first whole vector and after the last are written one by one.
    int32_t *out = a.out + g.out_off;
    const uint32_t lim = min(n, total);
    const uint32_t head = min(lim, (uint32_t)(((16 - ((uintptr_t)out & 15)) & 15) / 4));
    const uint32_t nvec = (lim - head) / 4;
    int4 *vout = reinterpret_cast<int4 *>(out + head);
    auto cdf = [&](uint32_t v) -> uint32_t { return get(v); };
    auto first_above = [&](uint32_t lo, uint32_t p) -> uint32_t {  // min{v >= lo : cdf(v) > p}
        uint32_t hi = R - 1;
        while (lo < hi) {
            const uint32_t mid = (lo + hi) >> 1;
            if (cdf(mid) > p) hi = mid; else lo = mid + 1;
        }
        return lo;
    };
    // The same from a value known to be close: steps of 1, 2, 4, ... until the
    // CDF exceeds p, then a binary search inside the last step -- O(log gap),
    // so sparse stretches of the range (the tails of a peaked shape, n << R)
    // are crossed in a few reads.
    auto next_above = [&](uint32_t lo, uint32_t p) -> uint32_t {
        uint32_t hi = lo, step = 1;
        while (cdf(hi) <= p) {  // cdf(R - 1) = total > p ends it
            lo = hi + 1;
            hi = min(R - 1, hi + step);
            step <<= 1;
        }
        while (lo < hi) {
            const uint32_t mid = (lo + hi) >> 1;
            if (cdf(mid) > p) hi = mid; else lo = mid + 1;
        }
        return lo;
    };
    const uint32_t lane = tid & 31, warp = tid >> 5, nwarps = nt >> 5;
    const uint32_t per_warp = ((nvec + nwarps - 1) / nwarps + 31) & ~31u;
    const uint32_t wb = warp * per_warp, we = min(nvec, wb + per_warp);
    uint32_t v = 0;
    bool first = true;
    for (uint32_t w = wb + lane; w < we; w += 32) {
        const uint32_t q = head + 4 * w;
        if (first) {
            v = first_above(0u, q);
            first = false;
        } else if (cdf(v) <= q) {
            v = next_above(v + 1, q);
        }
        if (cdf(v) >= q + 4) {
            const int32_t val = (int32_t)(min_u + v);
            vout[w] = make_int4(val, val, val, val);
        } else {
            int32_t r[4];
            uint32_t vv = v;
#pragma unroll
            for (int e = 0; e < 4; e++) {
                if (cdf(vv) <= q + e) vv = next_above(vv + 1, q + e);
                r[e] = (int32_t)(min_u + vv);
            }
            vout[w] = make_int4(r[0], r[1], r[2], r[3]);
        }
    }
    if (tid < 8) {
        const uint32_t p = tid < head ? tid : head + 4 * nvec + (tid - head);
        if ((tid < head || tid - head < 4) && p < lim) out[p] = (int32_t)(min_u + first_above(0u, p));
    }
}

// 32-bit counters when R of them fit in the `cap` words before s_tmp.
__device__ __forceinline__ void do_small(const BatchArgs &a, const BatchSeg &g, uint32_t *sm, uint32_t cap,
                                         uint32_t *s_tmp) {
    if (g.R <= cap) do_small_impl<true>(a, g, sm, s_tmp);
    else do_small_impl<false>(a, g, sm, s_tmp);
}

// ---------------------------------------------------------------- HIST
// Software pipelined: each thread has the next six 16-byte vectors in flight
// while it counts the six before them (the first launch's CTAs have 64
// registers each).  Measured on the benchmark's segments: four vectors
// loaded then counted 0.969 ms, eight 0.944 ms, sixteen spilled (1.09 ms),
// pipelined four 0.939 ms, pipelined six 0.930 ms.
__device__ void do_hist(const BatchArgs &a, const BatchSeg &g, const BatchItem &it, uint32_t *S) {
    const uint32_t tid = threadIdx.x, nt = blockDim.x;
    const uint32_t b = it.tile * g.T;
    const uint32_t w = min(g.T, g.R - b);
    for (uint32_t i = tid; i < w; i += nt) S[i] = 0;
    __syncthreads();
    const uint32_t base = (uint32_t)g.minVal + b;
    const uint32_t s_base = (uint32_t)__cvta_generic_to_shared(S);
    const int32_t *in = a.in + g.off;
    const uint64_t k0 = it.a, k1 = it.b;
    // 16-byte loads from the first 16-byte aligned element of the chunk.
    const uint64_t lead_a = (uint64_t)(((16 - ((uintptr_t)(in + k0) & 15)) & 15) / 4);
    const uint64_t lead = lead_a < k1 - k0 ? lead_a : k1 - k0;
    const uint64_t nv = (k1 - k0 - lead) / 4;
    const int4 *vin = reinterpret_cast<const int4 *>(in + k0 + lead);
    auto count4 = [&](const int4 k) {
        count_key_pred(s_base, (uint32_t)k.x - base, w);
        count_key_pred(s_base, (uint32_t)k.y - base, w);
        count_key_pred(s_base, (uint32_t)k.z - base, w);
        count_key_pred(s_base, (uint32_t)k.w - base, w);
    };
    uint64_t v = tid;
    if (g.m == 1) {
        // One tile: every key is read once, so stream it (evict first).
        if (v + 5 * nt < nv) {
            int4 kn[6];
#pragma unroll
            for (int u = 0; u < 6; u++) kn[u] = __ldcs(vin + v + u * nt);
            v += 6 * nt;
            for (; v + 5 * nt < nv; v += 6 * nt) {
                int4 kc[6];
#pragma unroll
                for (int u = 0; u < 6; u++) kc[u] = kn[u];
#pragma unroll
                for (int u = 0; u < 6; u++) kn[u] = __ldcs(vin + v + u * nt);
#pragma unroll
                for (int u = 0; u < 6; u++) count4(kc[u]);
            }
#pragma unroll
            for (int u = 0; u < 6; u++) count4(kn[u]);
        }
        for (; v < nv; v += nt) count4(__ldcs(vin + v));
    } else {
        // Several tiles: the other tiles' items read the same chunk (L2 hits).
        if (v + 5 * nt < nv) {
            int4 kn[6];
#pragma unroll
            for (int u = 0; u < 6; u++) kn[u] = __ldg(vin + v + u * nt);
            v += 6 * nt;
            for (; v + 5 * nt < nv; v += 6 * nt) {
                int4 kc[6];
#pragma unroll
                for (int u = 0; u < 6; u++) kc[u] = kn[u];
#pragma unroll
                for (int u = 0; u < 6; u++) kn[u] = __ldg(vin + v + u * nt);
#pragma unroll
                for (int u = 0; u < 6; u++) count4(kc[u]);
            }
#pragma unroll
            for (int u = 0; u < 6; u++) count4(kn[u]);
        }
        for (; v < nv; v += nt) count4(__ldg(vin + v));
    }
    if (tid < lead) count_key_pred(s_base, (uint32_t)in[k0 + tid] - base, w);
    for (uint64_t i = k0 + lead + 4 * nv + tid; i < k1; i += nt)
        count_key_pred(s_base, (uint32_t)in[i] - base, w);
    __syncthreads();
    uint32_t *H = a.ws_u32 + g.hist_off + b;
    if (g.single_hist) {
        // The only chunk of this tile: store every count (H need not be zero).
        for (uint32_t i = tid; i < w; i += nt) H[i] = S[i];
    } else {
        for (uint32_t i = tid; i < w; i += nt) {
            const uint32_t c = S[i];
            if (c) atomicAdd(&H[i], c);
        }
    }
}

__device__ __forceinline__ void prof_item(const BatchArgs &a, uint32_t kind, unsigned long long t0,
                                          unsigned long long wait) {
    const unsigned long long t1 = global_ns();
    atomicAdd(a.prof + kind, t1 - t0);
    atomicAdd(a.prof + 4 + kind, 1ull);
    atomicMin(a.prof + 8 + kind, t0);
    atomicMax(a.prof + 12 + kind, t1);
    if (wait) atomicAdd(a.prof + 16 + kind, wait);
}

// Smallest j in [lo, hi] with e[j] > p, given e[hi] > p.
__device__ __forceinline__ uint32_t first_after(const uint32_t *e, uint32_t lo, uint32_t hi, uint32_t p) {
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (e[mid] > p) hi = mid; else lo = mid + 1;
    }
    return lo;
}

// The same when the answer is expected close to lo: probes lo, lo + 1,
// lo + 3, lo + 7, ... until e exceeds p, then a binary search inside the last
// step -- O(log(j - lo)) reads.
__device__ __forceinline__ uint32_t next_after(const uint32_t *e, uint32_t lo, uint32_t hi, uint32_t p) {
    uint32_t probe = lo, step = 1;
    while (e[probe] <= p) {  // e[hi] > p ends it
        lo = probe + 1;
        probe = min(hi, probe + step);
        step <<= 1;
    }
    return first_after(e, lo, probe, p);
}

}  // namespace

__device__ __forceinline__ DevListBounds dev_lb(const BatchArgs &a) {
    return DevListBounds{a.dev_bounds[0], a.dev_bounds[1], a.dev_bounds[2], a.dev_bounds[3], a.dev_bounds[4]};
}

__device__ __forceinline__ void first_item(const BatchArgs &a, uint32_t idx, uint32_t *sm) {
    const unsigned long long t0 = (a.prof && threadIdx.x == 0) ? global_ns() : 0ull;
    const BatchItem it = a.items[idx];
    const BatchSeg g = a.segs[it.seg];
    if (it.kind == kItemSmall) do_small(a, g, sm, kBatchSmallMaxR / 2, sm + kBatchSmallMaxR / 2);
    else do_hist(a, g, it, sm);
    if (a.prof) {
        __syncthreads();
        if (threadIdx.x == 0) prof_item(a, it.kind, t0, 0);
    }
}

// DEV: the lists were built on the device (their lengths are in
// a.dev_counts) and the grid is a fixed number of CTAs that take items by
// ticket; otherwise one CTA per item of the host-built plan.
// One 1024-thread CTA per SM (the registers of a whole SM: 64 per thread):
// with two per SM (32 registers per thread) the same items ran so much slower
// that the segmented sort took 1.038 against 0.969 ms (host plan; the device-
// planned form 1.12 against 1.035 ms), measured.  The shared memory stays at
// kSegSmemBytes (a larger tile, 57344 bins in 224 KB, made it slower again).
template <bool DEV>
__global__ void __launch_bounds__(kSegThreads, 1) seg_first_kernel(BatchArgs a) {
    extern __shared__ uint32_t sm[];
    // The scan launch may be scheduled as soon as every CTA here has started;
    // it waits for this grid to finish before reading anything.
    asm volatile("griddepcontrol.launch_dependents;");
    if (!DEV) {
        first_item(a, blockIdx.x, sm);
        return;
    }
    __shared__ uint32_t s_idx;
    const uint32_t n_hist = a.dev_counts[4], n_small1 = a.dev_counts[5];
    const uint32_t nc[kHistClasses] = {a.dev_counts[6], a.dev_counts[7], a.dev_counts[8]};
    for (;;) {
        if (threadIdx.x == 0) s_idx = atomicAdd(&a.ctl->first_ticket, 1u);
        __syncthreads();
        const uint32_t k = s_idx;
        __syncthreads();  // every thread has read s_idx (and the previous item's shared memory is free)
        if (k >= n_hist + n_small1) break;
        first_item(a, (uint32_t)devplan_first_pos(k, nc, n_small1, dev_lb(a)), sm);
    }
}

// One 4096-bin chunk per CTA of kScanCtaThreads threads (16 bins each): small
// CTAs, so that several are resident per SM -- a chunk is mostly latency (its
// loads, the lookback, the run-table stores).
constexpr int kScanCtaThreads = 256;
constexpr int kScanPerThread = kBatchScanChunk / kScanCtaThreads;  // 16

// The chunk's runs are staged in shared memory before they are written out.
// Shared index of the chunk's r-th run: one padding word per 32, so that the
// consecutive runs of the 32 lanes of a warp (16 apart in a dense chunk) fall
// in 32 distinct banks.
__device__ __forceinline__ uint32_t run_slot(uint32_t r) { return r + (r >> 5); }

// One 4096-bin chunk of a large segment's histogram: local CDF and offsets
// (Algorithm 6) by the segment's decoupled lookback, the chunk's runs and the
// first run of every output item that starts inside it.
// The shared arrays are the kernel's own __shared__ variables (declared
// separately: gathered into one struct, the staging buffer lost its
// alignment and the scan phase took 8 % longer, measured).
__device__ __forceinline__ void scan_chunk(const BatchArgs &a, const BatchItem &it, const BatchSeg &g, uint64_t *s_warp,
                                           uint64_t &s_prefix, uint64_t &s_total, unsigned long long &s_wait,
                                           uint32_t *s_buf, unsigned long long t0) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int kWarps = kScanCtaThreads / 32;
    uint32_t *s_end = s_buf;
    int32_t *s_val = reinterpret_cast<int32_t *>(s_buf + kScanStageWords);
    const uint32_t chunk = (uint32_t)it.a;
    uint32_t *H = a.ws_u32 + g.hist_off;
    uint64_t *state = reinterpret_cast<uint64_t *>(a.ws_u32 + g.state_off);
    uint32_t *run_end = a.ws_u32 + g.run_end_off;
    int32_t *run_val = reinterpret_cast<int32_t *>(a.ws_u32 + g.run_val_off);
    uint32_t *start_run = a.ws_u32 + g.start_run_off;
    const uint32_t cbase = chunk * kBatchScanChunk;
    const uint32_t first = tid * kScanPerThread;  // this thread's bins in the chunk

    // Sixteen counts per thread (H is padded to whole chunks), zeroed behind
    // us.  They wait for the second pass in shared memory (in the staging
    // area, which is not written before they are read back).
    uint4 *h4p = reinterpret_cast<uint4 *>(H + cbase + first);
    uint64_t run = 0;
#pragma unroll
    for (int k = 0; k < kScanPerThread / 4; k++) {
        const uint4 q = h4p[k];
        const uint32_t c4[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
        for (int e = 0; e < 4; e++) {
            run += ((uint64_t)(c4[e] > 0) << 32) | c4[e];
            s_buf[run_slot(first + 4 * k + e)] = c4[e];
        }
    }
#pragma unroll
    for (int k = 0; k < kScanPerThread / 4; k++) h4p[k] = make_uint4(0, 0, 0, 0);
    const uint64_t winc = warp_incl_scan_u64(run, lane);
    if (lane == 31) s_warp[warp] = winc;
    __syncthreads();
    if (warp == 0) {
        const uint64_t wt = lane < kWarps ? s_warp[lane] : 0ull;
        const uint64_t wi = warp_incl_scan_u64(wt, lane);
        if (lane < kWarps) s_warp[lane] = wi - wt;
        const uint64_t total = __shfl_sync(0xffffffffu, wi, 31);
        // Decoupled lookback within the segment.
        uint64_t prefix = 0;
        unsigned long long waited = 0;
        if (g.scan_chunks > 1) {
            if (chunk == 0) {
                if (lane == 0) st_release_u64(&state[0], kStIncl | total);
            } else {
                if (lane == 0) st_release_u64(&state[chunk], kStAgg | total);
                const unsigned long long w0 = a.prof ? global_ns() : 0ull;
                int64_t look = (int64_t)chunk - 1;
                uint32_t spins = 0;
                bool timed_out = false;
                while (true) {
                    const int64_t idx = look - lane;
                    uint64_t st = (idx >= 0) ? ld_acquire_u64(&state[idx]) : kStIncl;
                    while (!__all_sync(0xffffffffu, (st >> 62) != 0)) {
                        if (++spins > kMaxSpin) { timed_out = true; break; }
                        __nanosleep(64);
                        if ((st >> 62) == 0) st = ld_acquire_u64(&state[idx]);
                    }
                    if (timed_out) break;
                    const unsigned incl_mask = __ballot_sync(0xffffffffu, (st >> 62) == 2);
                    if (incl_mask) {
                        const int fi = __ffs(incl_mask) - 1;
                        prefix += warp_sum_u64((lane <= fi) ? (st & kStValue) : 0);
                        break;
                    }
                    prefix += warp_sum_u64(st & kStValue);
                    look -= 32;
                }
                if (timed_out && lane == 0) atomicOr(&a.ctl->status, kDevTimeout);
                if (lane == 0) st_release_u64(&state[chunk], kStIncl | (prefix + total));
                if (a.prof) waited = global_ns() - w0;
            }
        }
        if (lane == 0) {
            s_prefix = prefix;
            s_total = total;
            s_wait = waited;
        }
    }
    __syncthreads();
    // Positions before the chunk and runs before the chunk (in the segment).
    const uint32_t pos_lo = (uint32_t)s_prefix, run_base = (uint32_t)(s_prefix >> 32);
    uint64_t p = s_warp[warp] + (winc - run);  // exclusive prefix of this thread in the chunk
    uint32_t c[kScanPerThread];
#pragma unroll
    for (int i = 0; i < kScanPerThread; i++) c[i] = s_buf[run_slot(first + i)];
    __syncthreads();  // every count read before the staging area is written
#pragma unroll
    for (int i = 0; i < kScanPerThread; i++) {
        const uint32_t v = cbase + first + i;
        p += ((uint64_t)(c[i] > 0) << 32) | c[i];
        const uint32_t cnt_end = pos_lo + (uint32_t)p;  // sum_{u<=v} c_u
        const uint32_t runs = (uint32_t)(p >> 32);      // non-empty values of the chunk up to v
        if (c[i] > 0) {
            s_end[run_slot(runs - 1)] = cnt_end;
            s_val[run_slot(runs - 1)] = (int32_t)((uint32_t)g.minVal + v);
        }
        if (v == g.R - 1) {
            a.seg_ctl[it.seg].num_runs = run_base + runs;
            if (cnt_end != g.n) atomicOr(&a.ctl->status, kDevKeyOutOfRange);
        }
    }
    __syncthreads();
    // The chunk's runs, written out coalesced.
    const uint32_t chunk_runs = (uint32_t)(s_total >> 32);
    for (uint32_t r = tid; r < chunk_runs; r += kScanCtaThreads) {
        run_end[run_base + r] = s_end[run_slot(r)];
        run_val[run_base + r] = s_val[run_slot(r)];
    }
    // Output items whose first position j * fill_chunk lies in the chunk's
    // positions [pos_lo, pos_hi): the run holding it, i.e. the first run
    // whose end exceeds it (Algorithm 7's rule).
    const uint32_t pos_hi = pos_lo + (uint32_t)s_total;
    if (pos_hi > pos_lo) {
        const uint32_t fc = g.fill_chunk;
        const uint32_t j_lo = (uint32_t)(((uint64_t)pos_lo + fc - 1) / fc);
        const uint32_t j_hi = min((uint32_t)(((uint64_t)pos_hi + fc - 1) / fc), g.fill_items);
        for (uint32_t j = j_lo + tid; j < j_hi; j += kScanCtaThreads) {
            const uint32_t p0 = j * fc;
            uint32_t lo = 0, hi = chunk_runs - 1;
            while (lo < hi) {
                const uint32_t mid = (lo + hi) >> 1;
                if (s_end[run_slot(mid)] > p0) hi = mid; else lo = mid + 1;
            }
            start_run[j] = run_base + lo;
        }
    }
    if (a.prof) {
        __syncthreads();
        if (tid == 0) prof_item(a, kItemScan, t0, s_wait);
    }
}


template <bool DEV>
__global__ void __launch_bounds__(kScanCtaThreads, 6) seg_scan_kernel(BatchArgs a) {
    __shared__ uint32_t s_ticket;
    __shared__ uint64_t s_warp[kScanCtaThreads / 32];
    __shared__ uint64_t s_prefix, s_total;
    __shared__ unsigned long long s_wait;
    __shared__ uint32_t s_buf[kScanSmemWords];
    const int tid = threadIdx.x;
    // List lengths (device-built lists: from the device) and positions (the
    // scan chunks at a.n_first, the in-CTA segments at a.n_first + a.n_scan:
    // the host plan's lengths, or the device lists' bounds).
    const uint32_t n_scan = DEV ? a.dev_counts[1] : a.n_scan;
    const uint32_t n_small2 = DEV ? a.dev_counts[2] : a.n_small2;
    auto small_item = [&](uint32_t i) {
        const unsigned long long ts = (a.prof && tid == 0) ? global_ns() : 0ull;
        const BatchItem it = a.items[DEV ? devplan_pos(dev_lb(a), kListSmall2, i) : a.n_first + a.n_scan + i];
        const BatchSeg g = a.segs[it.seg];
        do_small(a, g, s_buf, kScanSmemWords - 64, s_buf + kScanSmemWords - 64);
        if (a.prof) {
            __syncthreads();
            if (tid == 0) prof_item(a, kItemSmall, ts, 0);
        }
    };
    if (DEV) {
        // Device-built lists, as for a host plan: the in-CTA segments by CTA
        // index at the front of the grid, then one chunk per CTA by ticket;
        // CTAs past the lists exit at once.  The grid is sized by the lists'
        // bounds but capped (CTAs past the lists cost about half a
        // microsecond per thousand); when the lists outgrow it, CTA b also
        // takes in-CTA segments b + grid, b + 2 grid, ... and every CTA then
        // loops over chunk tickets.  The two forms are separate code: with
        // the chunk inside the loop (or the in-CTA segments taken by ticket
        // too) every chunk ran about twice as slow, measured.
        const uint32_t grid = gridDim.x;
        if (grid >= n_small2 + n_scan) {
            if (blockIdx.x >= n_small2 + n_scan) return;
            if (blockIdx.x < n_small2) {
                asm volatile("griddepcontrol.launch_dependents;");
                small_item(blockIdx.x);
                return;
            }
            if (tid == 0) s_ticket = atomicAdd(&a.ctl->scan_ticket, 1u);
            __syncthreads();
            const BatchItem it = a.items[devplan_chain_pos(dev_lb(a), kListScan0, a.dev_counts + 9, 2, s_ticket)];
            const BatchSeg g = a.segs[it.seg];
            asm volatile("griddepcontrol.wait;" ::: "memory");
            asm volatile("griddepcontrol.launch_dependents;");
            const unsigned long long t0 = (a.prof && tid == 0) ? global_ns() : 0ull;
            scan_chunk(a, it, g, s_warp, s_prefix, s_total, s_wait, s_buf, t0);
            return;
        }
        for (uint32_t j = blockIdx.x; j < n_small2; j += grid) {
            small_item(j);
            __syncthreads();  // the segment's shared memory is free
        }
        asm volatile("griddepcontrol.wait;" ::: "memory");
        for (;;) {
            if (tid == 0) s_ticket = atomicAdd(&a.ctl->scan_ticket, 1u);
            __syncthreads();
            const uint32_t t = s_ticket;
            __syncthreads();  // every thread has read the ticket (and the previous chunk's shared memory is free)
            if (t >= n_scan) break;
            const BatchItem it = a.items[devplan_chain_pos(dev_lb(a), kListScan0, a.dev_counts + 9, 2, t)];
            const BatchSeg g = a.segs[it.seg];
            const unsigned long long t0 = (a.prof && tid == 0) ? global_ns() : 0ull;
            scan_chunk(a, it, g, s_warp, s_prefix, s_total, s_wait, s_buf, t0);
        }
        return;
    }
    // The in-CTA segments come first in the grid (dispatched first; spreading
    // them among the scan chunks was measured slower).
    if (blockIdx.x < n_small2) {
        // An in-CTA segment: independent of the first launch, so no wait.
        asm volatile("griddepcontrol.launch_dependents;");
        small_item(blockIdx.x);
        return;
    }
    // The ticket and the chunk's descriptors come from plan data, not from
    // the first launch: fetched before waiting for it.  (The ticket counter
    // was reset by the previous run's output launch, which finished before
    // this plan's first launch began.)
    if (tid == 0) s_ticket = atomicAdd(&a.ctl->scan_ticket, 1u);
    __syncthreads();
    if (s_ticket >= n_scan) {
        // Only with a workspace whose ticket was not zero: the chunk this
        // ticket stood for is never published, so the output launch must not
        // trust the run tables.
        if (tid == 0) atomicOr(&a.ctl->status, kDevTimeout);
        return;
    }
    const BatchItem it = a.items[a.n_first + s_ticket];
    const BatchSeg g = a.segs[it.seg];
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;");
    const unsigned long long t0 = (a.prof && tid == 0) ? global_ns() : 0ull;
    scan_chunk(a, it, g, s_warp, s_prefix, s_total, s_wait, s_buf, t0);
}

// Output CTAs of 512 threads: four resident per SM, so that one CTA's
// descriptor loads and window round trip overlap the others' stores.
constexpr int kFillCtaThreads = 512;

// One output item: positions [it.a, it.b) of its segment from the run table
// (Algorithm 7's rule).
__device__ __forceinline__ void fill_item(const BatchArgs &a, const BatchItem &it, const BatchSeg &g, uint32_t *s_end,
                                          int32_t *s_val, unsigned long long t0) {
    const uint32_t tid = threadIdx.x, nt = blockDim.x;
    if (it.aux == 0 && g.scan_chunks > 1) {
        // The segment's first output item leaves its lookback state zeroed.
        uint64_t *state = reinterpret_cast<uint64_t *>(a.ws_u32 + g.state_off);
        for (uint32_t i = tid; i < g.scan_chunks; i += nt) state[i] = 0;
    }
    // A wait that ran out (or a stray scan ticket) leaves run tables
    // incomplete: write nothing (the status word reports it).
    if (a.ctl->status & kDevTimeout) return;
    // Indices into the segment's run table stay below its R entries whatever
    // the scan left behind.
    const uint32_t D = min(a.seg_ctl[it.seg].num_runs, g.R);
    if (D == 0) return;
    const uint32_t *run_end = a.ws_u32 + g.run_end_off;
    const int32_t *run_val = reinterpret_cast<const int32_t *>(a.ws_u32 + g.run_val_off);
    const uint32_t *start_run = a.ws_u32 + g.start_run_off;
    uint32_t k_cur = min(start_run[it.aux], D - 1);
    // Last run this item can need: the one holding the next item's first position.
    const uint32_t k_last = (it.aux + 1 < g.fill_items) ? min(start_run[it.aux + 1], D - 1) : D - 1;
    int32_t *out = a.out + g.out_off;
    // Positions relative to the segment; vectors aligned to the global `out`.
    const uint32_t head = (uint32_t)(((16 - ((uintptr_t)out & 15)) & 15) / 4);
    int4 *vout = reinterpret_cast<int4 *>(out + head);
    uint32_t pos = (uint32_t)it.a;
    const uint32_t P1 = (uint32_t)it.b;
    while (pos < P1 && k_cur < D) {
        const uint32_t nw = min((uint32_t)kSegFillRuns, (k_last >= k_cur ? k_last - k_cur : 0u) + 1u);
        __syncthreads();
        for (uint32_t i = tid; i < nw; i += nt) {
            s_end[i] = run_end[k_cur + i];
            s_val[i] = run_val[k_cur + i];
        }
        __syncthreads();
        const uint32_t hi = min(P1, s_end[nw - 1]);
        const uint32_t w_lo = pos >= head ? (pos - head + 3) >> 2 : 0u;
        const uint32_t w_hi = hi >= head ? (hi - head) >> 2 : 0u;
        if (s_end[0] >= hi) {
            // One run covers the whole round: constant stores.
            const int32_t v = s_val[0];
            const int4 vv = make_int4(v, v, v, v);
            for (uint32_t w = w_lo + tid; w < w_hi; w += nt) __stcs(vout + w, vv);
        } else {
            const uint32_t lane = tid & 31, warp = tid >> 5, nwarps = nt >> 5;
            const uint32_t nvec = w_hi > w_lo ? w_hi - w_lo : 0u;
            const uint32_t per_warp = ((nvec + nwarps - 1) / nwarps + 31) & ~31u;
            const uint32_t wb = w_lo + warp * per_warp;
            const uint32_t we = min(w_hi, wb + per_warp);
            // The run of this lane's last vector, its end and value in
            // registers (no shared-memory read inside the same run).
            uint32_t j = 0;
            uint32_t ej = s_end[0];
            int32_t vj = s_val[0];
            for (uint32_t w = wb + lane; w < we; w += 32) {
                const uint32_t q = head + 4 * w;
                if (ej <= q) {
                    j = next_after(s_end, j + 1, nw - 1, q);
                    ej = s_end[j];
                    vj = s_val[j];
                }
                if (ej >= q + 4) {
                    __stcs(vout + w, make_int4(vj, vj, vj, vj));
                } else {
                    // Positions q..q+3 lie in runs j..j+3: q+e lies in run j
                    // plus the number of runs among j, j+1, j+2 that end at or
                    // before it (ends read independently, clamped to the
                    // window's last run, whose end exceeds every position).
                    const uint32_t e1 = s_end[min(j + 1, nw - 1)], e2 = s_end[min(j + 2, nw - 1)];
                    int32_t r[4];
                    r[0] = vj;  // q < ej
#pragma unroll
                    for (int e = 1; e < 4; e++) {
                        const uint32_t p = q + e;
                        r[e] = s_val[j + (p >= ej) + (p >= e1) + (p >= e2)];
                    }
                    __stcs(vout + w, make_int4(r[0], r[1], r[2], r[3]));
                }
            }
        }
        if (tid < 8) {
            const uint32_t q_lo = head + 4 * w_lo, q_hi = head + 4 * w_hi;
            uint32_t p;
            if (w_lo >= w_hi) {
                p = pos + tid;
            } else {
                const uint32_t n_front = q_lo - pos;
                p = tid < n_front ? pos + tid : q_hi + (tid - n_front);
            }
            if (p >= pos && p < hi && (w_lo >= w_hi || p < q_lo || p >= q_hi))
                out[p] = s_val[first_after(s_end, 0, nw - 1, p)];
        }
        pos = hi;
        k_cur += nw;
    }
    if (a.prof) {
        __syncthreads();
        if (tid == 0) prof_item(a, kItemFill, t0, 0);
    }
}


template <bool DEV>
__global__ void __launch_bounds__(kFillCtaThreads) seg_fill_kernel(BatchArgs a) {
    __shared__ uint32_t s_end[kSegFillRuns];
    __shared__ int32_t s_val[kSegFillRuns];
    const uint32_t tid = threadIdx.x;
    if (DEV && blockIdx.x == 0) {
        // The first CTA leaves the device planner's ticket and lookback
        // records zeroed for the next run (the planner finished before this
        // run's first launch began).
        for (uint32_t i = tid; i < a.plan_look_words; i += blockDim.x) a.plan_look[i] = 0;
        if (tid == 0) a.ctl->plan_ticket = 0;
    }
    if (DEV && blockIdx.x >= a.dev_counts[3]) {
        // Past the device-built list (the grid is sized by its bound); the
        // first CTA still resets the scan ticket, even for an empty list.
        if (blockIdx.x == 0) {
            asm volatile("griddepcontrol.wait;" ::: "memory");
            if (tid == 0) a.ctl->scan_ticket = 0;
        }
        return;
    }
    // The item and its segment are plan data: fetched before waiting for the
    // scan launch.  A host plan's output items sit after its other lists;
    // device-built ones in two lists by cost, the expensive one first.
    const BatchItem it = a.items[DEV ? devplan_chain_pos(dev_lb(a), kListFill0, a.dev_counts + 11, 2, blockIdx.x)
                                     : a.n_first + a.n_scan + a.n_small2 + blockIdx.x];
    const BatchSeg g = a.segs[it.seg];
    asm volatile("griddepcontrol.wait;" ::: "memory");
    const unsigned long long t0 = (a.prof && tid == 0) ? global_ns() : 0ull;
    if (blockIdx.x == 0 && tid == 0) a.ctl->scan_ticket = 0;
    fill_item(a, it, g, s_end, s_val, t0);
}

namespace {

cudaError_t launch_dep(const void *fn, uint32_t grid, int threads, const BatchArgs &a, bool programmatic,
                       cudaStream_t s) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = programmatic ? 1 : 0;
    void *args[] = {const_cast<BatchArgs *>(&a)};
    return cudaLaunchKernelExC(&cfg, fn, args);
}

}  // namespace

cudaError_t launch_batched(const BatchArgs &a, cudaStream_t s) {
    cudaError_t e = cudaFuncSetAttribute(seg_first_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kSegSmemBytes);
    if (e != cudaSuccess) return e;
    // A launch is a programmatic dependent only of the plan's own launch
    // before it (whose work it waits for, or which its CTAs do not read):
    // the first launch issued waits for all earlier work in the stream.
    bool chained = false;
    if (a.n_first) {
        seg_first_kernel<false><<<a.n_first, kSegThreads, kSegSmemBytes, s>>>(a);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        chained = true;
    }
    if (a.n_scan + a.n_small2) {
        e = launch_dep((const void *)seg_scan_kernel<false>, a.n_scan + a.n_small2, kScanCtaThreads, a, chained, s);
        if (e != cudaSuccess) return e;
        chained = true;
    }
    if (a.n_fill &&
        (e = launch_dep((const void *)seg_fill_kernel<false>, a.n_fill, kFillCtaThreads, a, chained, s)) != cudaSuccess)
        return e;
    return cudaSuccess;
}

cudaError_t launch_batched_dev(const BatchArgs &a, uint32_t first_ctas, uint32_t scan_ctas, uint32_t fill_ctas,
                               cudaStream_t s) {
    cudaError_t e = cudaFuncSetAttribute(seg_first_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kSegSmemBytes);
    if (e != cudaSuccess) return e;
    // The first launch waits for the planner; every launch runs (the lists
    // may be empty), so that the tickets are consumed and reset in order.
    seg_first_kernel<true><<<first_ctas, kSegThreads, kSegSmemBytes, s>>>(a);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    e = launch_dep((const void *)seg_scan_kernel<true>, scan_ctas, kScanCtaThreads, a, true, s);
    if (e != cudaSuccess) return e;
    return launch_dep((const void *)seg_fill_kernel<true>, fill_ctas, kFillCtaThreads, a, true, s);
}

}  // namespace rtcdf
