// Segmented RT-CDF: many independent arrays (segments) of uneven length n_s
// and range size R_s, each with its own [minVal_s, maxVal_s), sorted by ONE
// persistent launch.  The method per segment is unchanged (Algorithms 4-7:
// tile histogram, local CDF + offsets, output from the CDF); what is new is
// the schedule.
//
// Worker CTAs (two per SM) take work items from a global queue in order:
//   1. HIST  (large segments)  histogram of a chunk of keys for one range
//                              tile, merged into the segment's global H;
//   2. SMALL (n_s < 65536)     the whole sort of one segment inside one CTA:
//                              16-bit shared-memory counters (a count never
//                              exceeds n_s < 2^16), in-place CDF, output by
//                              Algorithm 7's search;
//   3. SCAN  (large segments)  local CDFs + offsets of the segment's H, its
//                              run table and the start run of each FILL item;
//   4. FILL  (large segments)  output of a range of positions from the run
//                              table.
// A SCAN item waits until every HIST item of its segment has finished, a FILL
// item until its segment's SCAN has.  Items are dequeued in order, so every
// item waited on has already been taken by a running CTA: no deadlock.  Every
// wait is bounded; one that gives up records RTCDF_DEV_TIMEOUT and moves on.
// The last worker to finish resets the queue and the per-segment counters, so
// the launch can be replayed (e.g. from a CUDA graph) with no host work.
#include "batched.h"

namespace rtcdf {

namespace {

__device__ __forceinline__ uint32_t ld_acquire_u32(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait (bounded) until *p >= target; thread 0 waits, the CTA follows.  With a
// profile buffer, the time spent waiting is added to wait_ns.
__device__ void wait_at_least(const uint32_t *p, uint32_t target, uint32_t *status,
                              unsigned long long *wait_ns) {
    if (threadIdx.x == 0) {
        const unsigned long long t0 = wait_ns ? global_ns() : 0ull;
        uint32_t spins = 0;
        int ok = 1;
        while (ld_acquire_u32(p) < target) {
            if (++spins > kMaxSpin) { ok = 0; break; }
            __nanosleep(128);
        }
        if (!ok) atomicOr(status, kDevTimeout);
        if (wait_ns) atomicAdd(wait_ns, global_ns() - t0);
    }
    __syncthreads();
}

__device__ __forceinline__ uint32_t block_excl_scan_u32(uint32_t x, uint32_t *s_tmp, uint32_t *total) {
    // s_tmp holds blockDim/32 + 1 entries.
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    uint32_t inc = x;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, inc, d);
        if (lane >= d) inc += y;
    }
    if (lane == 31) s_tmp[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        uint32_t t = lane < nw ? s_tmp[lane] : 0u;
        uint32_t ti = t;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, ti, d);
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

// ---------------------------------------------------------------- SMALL
// One segment, n < 65536 keys, R <= kBatchSmallMaxR values, in one CTA.
__device__ void do_small(const BatchArgs &a, const BatchSeg &g, uint32_t *sm) {
    const uint32_t R = g.R, n = g.n, nt = blockDim.x, tid = threadIdx.x;
    uint32_t *cnt = sm;                       // R 16-bit counters packed in words
    uint32_t *s_tmp = sm + kBatchSmallMaxR / 2;  // scan scratch
    const uint32_t words = (R + 1) / 2;
    for (uint32_t i = tid; i < words; i += nt) cnt[i] = 0;
    __syncthreads();
    const int32_t *in = a.in + g.off;
    const uint32_t min_u = (uint32_t)g.minVal;
    auto count1 = [&](int32_t key) {
        const uint32_t x = (uint32_t)key - min_u;
        if (x < R) atomicAdd(&cnt[x >> 1], 1u << ((x & 1) * 16));
    };
    // 16-byte loads, eight in flight per thread, after the unaligned head.
    const uint32_t lead_a = (uint32_t)(((16 - ((uintptr_t)in & 15)) & 15) / 4);
    const uint32_t lead = lead_a < n ? lead_a : n;
    const uint32_t nv = (n - lead) / 4;
    const int4 *vin = reinterpret_cast<const int4 *>(in + lead);
    uint32_t iv = tid;
    for (; iv + 7 * nt < nv; iv += 8 * nt) {
        int4 k[8];
#pragma unroll
        for (int u = 0; u < 8; u++) k[u] = __ldcs(vin + iv + u * nt);
#pragma unroll
        for (int u = 0; u < 8; u++) { count1(k[u].x); count1(k[u].y); count1(k[u].z); count1(k[u].w); }
    }
    for (; iv < nv; iv += nt) {
        const int4 k = __ldcs(vin + iv);
        count1(k.x); count1(k.y); count1(k.z); count1(k.w);
    }
    if (tid < lead) count1(in[tid]);
    for (uint32_t i = lead + 4 * nv + tid; i < n; i += nt) count1(in[i]);
    __syncthreads();
    // In-place inclusive CDF over the 16-bit counters (values <= n < 2^16).
    uint16_t *c16 = reinterpret_cast<uint16_t *>(cnt);
    const uint32_t per = (R + nt - 1) / nt;
    const uint32_t b0 = min(R, tid * per), b1 = min(R, b0 + per);
    uint32_t local = 0;
    for (uint32_t v = b0; v < b1; v++) local += c16[v];
    uint32_t total = 0;
    const uint32_t ex = block_excl_scan_u32(local, s_tmp, &total);
    uint32_t run = ex;
    for (uint32_t v = b0; v < b1; v++) {
        run += c16[v];
        c16[v] = (uint16_t)run;
    }
    if (tid == 0 && total != n) atomicOr(&a.ctl->status, kDevKeyOutOfRange);
    __syncthreads();
    // Output: position p holds minVal + min{v : CDF[v] >= p + 1} (Algorithm 7).
    // Each warp takes a contiguous block of positions, lanes interleaved (one
    // coalesced store per step); a lane's positions grow by 32, so after one
    // binary search its value index only moves forward (next value first,
    // binary search for longer jumps).
    int32_t *out = a.out + g.out_off;
    const uint32_t lim = min(n, total);
    const uint32_t lane = tid & 31, warp = tid >> 5, nwarps = nt >> 5;
    const uint32_t per_warp = ((lim + nwarps - 1) / nwarps + 31) & ~31u;
    const uint32_t pb = warp * per_warp, pe = min(lim, pb + per_warp);
    uint32_t v = 0;
    bool first = true;
    for (uint32_t p = pb + lane; p < pe; p += 32) {
        if (first || c16[v] <= p) {
            uint32_t lo = first ? 0u : v + 1, hi = R - 1;
            if (!first && c16[lo] > p) {
                hi = lo;
            }
            while (lo < hi) {
                const uint32_t mid = (lo + hi) >> 1;
                if (c16[mid] > p) hi = mid; else lo = mid + 1;
            }
            v = lo;
            first = false;
        }
        out[p] = (int32_t)(min_u + v);
    }
}

// ---------------------------------------------------------------- HIST
// S[y] += 1 when y < w: a predicated shared-memory reduction (as in the
// single-array histogram kernel).
__device__ __forceinline__ void count_key_pred(uint32_t s_base, uint32_t y, uint32_t w) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.lt.u32 p, %0, %1;\n\t"
        "@p red.shared.add.u32 [%2], 1;\n\t}"
        ::"r"(y), "r"(w), "r"(s_base + 4u * y));
}

__device__ void do_hist(const BatchArgs &a, const BatchSeg &g, const BatchItem &it, uint32_t *S) {
    const uint32_t tid = threadIdx.x, nt = blockDim.x;
    const uint32_t b = it.tile * g.T;
    const uint32_t w = min(g.T, g.R - b);
    for (uint32_t i = tid; i < w; i += nt) S[i] = 0;
    __syncthreads();
    const uint32_t base = (uint32_t)g.minVal + b;
    const int32_t *in = a.in + g.off;
    const uint64_t k0 = it.a, k1 = it.b;
    // 16-byte loads from the first 16-byte aligned element of the chunk.
    const uint64_t lead_a = (uint64_t)(((16 - ((uintptr_t)(in + k0) & 15)) & 15) / 4);
    const uint64_t lead = lead_a < k1 - k0 ? lead_a : k1 - k0;
    const uint64_t nv = (k1 - k0 - lead) / 4;
    const int4 *vin = reinterpret_cast<const int4 *>(in + k0 + lead);
    const uint32_t s_base = (uint32_t)__cvta_generic_to_shared(S);
    auto count4 = [&](const int4 k) {
        count_key_pred(s_base, (uint32_t)k.x - base, w);
        count_key_pred(s_base, (uint32_t)k.y - base, w);
        count_key_pred(s_base, (uint32_t)k.z - base, w);
        count_key_pred(s_base, (uint32_t)k.w - base, w);
    };
    uint64_t v = tid;
    for (; v + 7 * nt < nv; v += 8 * nt) {
        int4 k[8];
#pragma unroll
        for (int u = 0; u < 8; u++) k[u] = __ldcs(vin + v + u * nt);
#pragma unroll
        for (int u = 0; u < 8; u++) count4(k[u]);
    }
    for (; v < nv; v += nt) count4(__ldcs(vin + v));
    if (tid < lead) {
        const uint32_t y = (uint32_t)in[k0 + tid] - base;
        if (y < w) atomicAdd(&S[y], 1u);
    }
    for (uint64_t i = k0 + lead + 4 * nv + tid; i < k1; i += nt) {
        const uint32_t y = (uint32_t)in[i] - base;
        if (y < w) atomicAdd(&S[y], 1u);
    }
    __syncthreads();
    uint32_t *H = a.ws_u32 + g.hist_off + b;
    for (uint32_t i = tid; i < w; i += nt) {
        const uint32_t c = S[i];
        if (c) atomicAdd(&H[i], c);
    }
    __threadfence();
    __syncthreads();
    if (tid == 0) atomicAdd(&a.seg_ctl[it.seg].hist_done, 1u);
}

// ---------------------------------------------------------------- SCAN
__device__ void do_scan(const BatchArgs &a, const BatchSeg &g, const BatchItem &it, uint32_t *sm) {
    const uint32_t tid = threadIdx.x, nt = blockDim.x;
    BatchSegCtl &sc = a.seg_ctl[it.seg];
    wait_at_least(&sc.hist_done, g.hist_items, &a.ctl->status,
                  a.prof ? a.prof + 16 + kItemScan : nullptr);
    uint32_t *H = a.ws_u32 + g.hist_off;
    uint32_t *run_end = a.ws_u32 + g.run_end_off;
    int32_t *run_val = reinterpret_cast<int32_t *>(a.ws_u32 + g.run_val_off);
    uint32_t *start_run = a.ws_u32 + g.start_run_off;
    uint32_t *s_cdf = sm;                      // kBatchScanChunk entries
    uint32_t *s_runs = sm + kBatchScanChunk;   // kBatchScanChunk entries
    uint32_t *s_tmp = sm + 2 * kBatchScanChunk;
    constexpr uint32_t items = kBatchScanChunk / kBatchThreads;  // bins per thread per chunk
    static_assert(items % 4 == 0, "whole 16-byte vectors per thread");
    uint32_t cnt_prefix = 0, run_prefix = 0;
    for (uint32_t cb = 0; cb < g.R; cb += kBatchScanChunk) {
        // This thread's bins: [cb + tid * items, + items) -- H is padded to
        // whole kBatchScanChunk blocks, so whole 16-byte vectors can be read
        // (all loads first, then the zeroing stores).
        uint32_t cloc = 0, rloc = 0;
        const uint32_t v0 = cb + tid * items;
        uint4 *hv = reinterpret_cast<uint4 *>(H + v0);
        uint4 q[kBatchScanChunk / kBatchThreads / 4];
#pragma unroll
        for (uint32_t k = 0; k < items / 4; k++) q[k] = hv[k];
#pragma unroll
        for (uint32_t k = 0; k < items / 4; k++) hv[k] = make_uint4(0, 0, 0, 0);  // left zeroed
#pragma unroll
        for (uint32_t k = 0; k < items / 4; k++) {
            const uint32_t c4[4] = {q[k].x, q[k].y, q[k].z, q[k].w};
#pragma unroll
            for (int e = 0; e < 4; e++) {
                s_cdf[tid * items + 4 * k + e] = c4[e];
                cloc += c4[e];
                rloc += (c4[e] > 0);
            }
        }
        uint32_t ctot = 0, rtot = 0;
        const uint32_t cex = block_excl_scan_u32(cloc, s_tmp, &ctot);
        const uint32_t rex = block_excl_scan_u32(rloc, s_tmp, &rtot);
        uint32_t cr = cnt_prefix + cex, rr = run_prefix + rex;
        for (uint32_t i = 0; i < items; i++) {
            const uint32_t v = v0 + i;
            const uint32_t c = s_cdf[tid * items + i];
            cr += c;
            rr += (c > 0);
            s_cdf[tid * items + i] = cr;
            s_runs[tid * items + i] = rr;
            if (v < g.R && c > 0) {
                run_end[rr - 1] = cr;
                run_val[rr - 1] = (int32_t)((uint32_t)g.minVal + v);
            }
        }
        __syncthreads();
        // FILL items whose first position falls in [cnt_prefix, cnt_prefix + ctot).
        const uint32_t lo_pos = cnt_prefix, hi_pos = cnt_prefix + ctot;
        if (hi_pos > lo_pos) {
            const uint32_t fc = g.fill_chunk;
            const uint32_t j_lo = (lo_pos + fc - 1) / fc;
            const uint32_t j_hi = min((hi_pos + fc - 1) / fc, g.fill_items);
            for (uint32_t j = j_lo + tid; j < j_hi; j += nt) {
                const uint32_t p0 = j * fc;
                uint32_t lo = 0, hi = kBatchScanChunk - 1;
                while (lo < hi) {
                    const uint32_t mid = (lo + hi) >> 1;
                    if (s_cdf[mid] > p0) hi = mid; else lo = mid + 1;
                }
                start_run[j] = s_runs[lo] - 1;
            }
        }
        cnt_prefix += ctot;
        run_prefix += rtot;
        __syncthreads();
    }
    __threadfence();  // every thread's run-table writes, before the flag
    __syncthreads();
    if (tid == 0) {
        if (cnt_prefix != g.n) atomicOr(&a.ctl->status, kDevKeyOutOfRange);
        sc.num_runs = run_prefix;
        __threadfence();
        atomicExch(&sc.scan_done, 1u);
    }
}

// ---------------------------------------------------------------- FILL
__device__ __forceinline__ uint32_t first_after(const uint32_t *e, uint32_t lo, uint32_t hi, uint32_t p) {
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (e[mid] > p) hi = mid; else lo = mid + 1;
    }
    return lo;
}

__device__ void do_fill(const BatchArgs &a, const BatchSeg &g, const BatchItem &it, uint32_t *sm) {
    const uint32_t tid = threadIdx.x, nt = blockDim.x;
    BatchSegCtl &sc = a.seg_ctl[it.seg];
    wait_at_least(&sc.scan_done, 1u, &a.ctl->status, a.prof ? a.prof + 16 + kItemFill : nullptr);
    const uint32_t D = *(volatile uint32_t *)&sc.num_runs;
    const uint32_t *run_end = a.ws_u32 + g.run_end_off;
    const int32_t *run_val = reinterpret_cast<const int32_t *>(a.ws_u32 + g.run_val_off);
    uint32_t k_cur = a.ws_u32[g.start_run_off + it.aux];
    // Last run this item can need: the one holding the next item's first position.
    const uint32_t k_last = (it.aux + 1 < g.fill_items)
                                ? min(a.ws_u32[g.start_run_off + it.aux + 1], D - 1) : D - 1;
    // A window of up to four runs per thread (few rounds where runs are short).
    const uint32_t RW = 4 * nt;
    uint32_t *s_end = sm;
    int32_t *s_val = reinterpret_cast<int32_t *>(sm + RW);
    int32_t *out = a.out + g.out_off;
    // Positions relative to the segment; vectors aligned to the global `out`.
    const uint32_t head = (uint32_t)(((16 - ((uintptr_t)out & 15)) & 15) / 4);
    int4 *vout = reinterpret_cast<int4 *>(out + head);
    uint32_t pos = (uint32_t)it.a;
    const uint32_t P1 = (uint32_t)it.b;
    while (pos < P1 && k_cur < D) {
        const uint32_t nw = min(RW, (k_last >= k_cur ? k_last - k_cur : 0u) + 1u);
        __syncthreads();
        for (uint32_t i = tid; i < nw; i += nt) {
            s_end[i] = run_end[k_cur + i];
            s_val[i] = run_val[k_cur + i];
        }
        __syncthreads();
        const uint32_t hi = min(P1, s_end[nw - 1]);
        const uint32_t w_lo = pos >= head ? (pos - head + 3) >> 2 : 0u;
        const uint32_t w_hi = hi >= head ? (hi - head) >> 2 : 0u;
        const uint32_t lane = tid & 31, warp = tid >> 5, nwarps = nt >> 5;
        const uint32_t nvec = w_hi > w_lo ? w_hi - w_lo : 0u;
        const uint32_t per_warp = ((nvec + nwarps - 1) / nwarps + 31) & ~31u;
        const uint32_t wb = w_lo + warp * per_warp;
        const uint32_t we = min(w_hi, wb + per_warp);
        uint32_t j = 0;
        for (uint32_t w = wb + lane; w < we; w += 32) {
            const uint32_t q = head + 4 * w;
            if (s_end[j] <= q) j = (s_end[j + 1] > q) ? j + 1 : first_after(s_end, j + 2, nw - 1, q);
            if (s_end[j] >= q + 4) {
                const int32_t v = s_val[j];
                __stcs(vout + w, make_int4(v, v, v, v));
            } else {
                int32_t r[4];
                uint32_t jj = j;
#pragma unroll
                for (int e = 0; e < 4; e++) {
                    while (s_end[jj] <= q + e) jj++;
                    r[e] = s_val[jj];
                }
                __stcs(vout + w, make_int4(r[0], r[1], r[2], r[3]));
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
}

}  // namespace

// Each worker holds its current item and, taken while the current one runs,
// the index of its next (so the queue's atomic round trip is off the critical
// path).  Holding one item ahead cannot deadlock: the unfinished item with the
// lowest queue index is always some worker's current item (a held-ahead item
// has a lower-index current item in front of it), and everything it waits on
// has a lower index, hence has finished.
__global__ void __launch_bounds__(kBatchThreads, kBatchWorkersPerSM) batched_kernel(BatchArgs a) {
    extern __shared__ uint32_t sm[];
    __shared__ uint32_t s_item;
    if (threadIdx.x == 0) s_item = atomicAdd(&a.ctl->queue_head, 1u);
    __syncthreads();
    uint32_t i = s_item;
    while (i < a.num_items) {
        uint32_t next = 0;
        if (threadIdx.x == 0) next = atomicAdd(&a.ctl->queue_head, 1u);
        const BatchItem it = a.items[i];
        const BatchSeg g = a.segs[it.seg];
        const unsigned long long t_start = (a.prof && threadIdx.x == 0) ? global_ns() : 0ull;
        switch (it.kind) {
            case kItemSmall: do_small(a, g, sm); break;
            case kItemHist: do_hist(a, g, it, sm); break;
            case kItemScan: do_scan(a, g, it, sm); break;
            default: do_fill(a, g, it, sm); break;
        }
        __syncthreads();  // every thread is done with this item and with s_item
        if (a.prof && threadIdx.x == 0) {
            const unsigned long long t_end = global_ns();
            const uint32_t k = it.kind & 3u;
            atomicAdd(a.prof + k, t_end - t_start);
            atomicAdd(a.prof + 4 + k, 1ull);
            atomicMin(a.prof + 8 + k, t_start);
            atomicMax(a.prof + 12 + k, t_end);
        }
        if (threadIdx.x == 0) s_item = next;
        __syncthreads();
        i = s_item;
    }
    // The last worker out resets the queue and the per-segment counters.
    __syncthreads();
    __shared__ uint32_t s_last;
    if (threadIdx.x == 0) {
        __threadfence();
        s_last = (atomicAdd(&a.ctl->workers_done, 1u) == gridDim.x - 1);
    }
    __syncthreads();
    if (s_last) {
        for (uint32_t s = threadIdx.x; s < a.num_segs; s += blockDim.x) {
            a.seg_ctl[s].hist_done = 0;
            a.seg_ctl[s].scan_done = 0;
        }
        if (threadIdx.x == 0) {
            a.ctl->queue_head = 0;
            a.ctl->workers_done = 0;
        }
    }
}

cudaError_t launch_batched(const BatchArgs &a, int workers, cudaStream_t s) {
    cudaError_t e = cudaFuncSetAttribute(batched_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kBatchSmemBytes);
    if (e != cudaSuccess) return e;
    batched_kernel<<<workers, kBatchThreads, kBatchSmemBytes, s>>>(a);
    return cudaGetLastError();
}

}  // namespace rtcdf
