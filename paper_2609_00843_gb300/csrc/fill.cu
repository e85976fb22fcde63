// Output generation from the local CDFs (Algorithm 7), all tiles in one launch.
//
// Algorithm 7 assigns output positions to threads and finds the value at
// position p as the smallest x with C[x] >= p + 1 by binary search.  Here each
// CTA owns a contiguous range of positions [P0, P1) and walks the run table
// built by the scan (run_end[k] = exclusive end of the k-th non-empty value,
// run_val[k] = that value's key): it copies a window of consecutive runs into
// shared memory, then every thread writes 16-byte vectors of its positions,
// finding the run of a position with the same rule (smallest k with
// run_end[k] >= p + 1), starting from the run of its previous vector (a
// galloping search: the next run, then steps of 2, 4, ... runs, then a binary
// search inside the last step).  When a whole vector lies inside one run --
// the common case -- that is one shared load and one compare before the
// store; a vector across runs reads the next runs' ends independently.  The
// few positions of a window that do not fill a whole aligned vector are
// written one by one.
//
// All positions are below n < 2^32, so the index arithmetic is 32-bit.  The
// CTA also clears the scan's lookback state so the workspace is ready for the
// next sort.
#include "rtcdf_internal.h"

namespace rtcdf {

// Smallest j in [lo, hi] with s_end[j] > p, given s_end[hi] > p.
__device__ __forceinline__ int first_run_after(const uint32_t *s_end, int lo, int hi, uint32_t p) {
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (s_end[mid] > p) hi = mid; else lo = mid + 1;
    }
    return lo;
}

// The same when the answer is expected close to lo: probes lo, lo + 1,
// lo + 3, lo + 7, ... until s_end exceeds p, then a binary search inside the
// last step -- O(log(j - lo)) reads, so a lane that crosses a few short runs
// between its vectors does not pay a search over the whole window.
__device__ __forceinline__ int next_run_after(const uint32_t *s_end, int lo, int hi, uint32_t p) {
    int probe = lo, step = 1;
    while (s_end[probe] <= p) {  // s_end[hi] > p ends it
        lo = probe + 1;
        probe = min(hi, probe + step);
        step <<= 1;
    }
    return first_run_after(s_end, lo, probe, p);
}

// Runs per shared-memory window: four per thread, so that a CTA whose
// positions cross thousands of short runs (the tails of a peaked distribution
// over a wide range) needs few window rounds -- each round costs a global
// round trip and two barriers.
template <int WIN>
constexpr int kRunWindow = 4 * WIN;

// CTAs issued first that take the LAST output chunks.  With a peaked shape
// the chunks at both ends of the output cross by far the most runs (the
// tails, thousands of values of a few keys each); the first ones are issued
// first anyway, and the last ones, issued last, would end the launch.
constexpr uint32_t kTailChunksFirst = 32;

template <int WIN>
__global__ void __launch_bounds__(WIN) fill_kernel(FillArgs a) {
    constexpr int RW = kRunWindow<WIN>;
    __shared__ uint32_t s_end[RW];
    __shared__ int32_t s_val[RW];
    const int tid = threadIdx.x;
    const uint32_t K = min(kTailChunksFirst, a.fill_ctas);
    const uint32_t c = blockIdx.x < K ? a.fill_ctas - K + blockIdx.x : blockIdx.x - K;  // output chunk

    // Programmatic dependent of the scan: wait for its results.
    asm volatile("griddepcontrol.wait;" ::: "memory");
    for (uint32_t i = c * WIN + tid; i < a.scan_chunks; i += a.fill_ctas * WIN) a.scan_state[i] = 0;
    if (c == 0 && tid == 0) a.ctl->scan_ticket = 0;

    // A wait that ran out (or a stray scan ticket) leaves the run table and the
    // start runs incomplete: write nothing (the output is unspecified then and
    // the status word says so).  The status is sticky until read, so once it
    // is set later sorts on the workspace write nothing either.
    if (a.ctl->status & kDevTimeout) return;

    // Positions are those of the whole sorted array; this launch writes
    // [pos_base, n) of them, position p to out[p - pos_base].  hb is the
    // position of the first 16-byte aligned element of `out`.
    const uint32_t n = (uint32_t)a.n, head = a.head, fc = (uint32_t)a.fill_chunk;
    const uint32_t pb = a.pos_base, hb = pb + head;
    const uint32_t P0 = (c == 0) ? pb : hb + c * fc;
    const uint32_t P1 = (c + 1 == a.fill_ctas) ? n : hb + (c + 1) * fc;
    // Every index into the run table stays below the R entries it holds, even
    // if the scan's results were not what this sort expects.
    const uint32_t D = min(a.ctl->num_runs, a.R);
    if (D == 0) return;
    uint32_t k_cur = min(a.start_run[c], D - 1);
    // Last run this CTA can need: the one holding the next CTA's first position.
    const uint32_t k_last = (c + 1 < a.fill_ctas) ? min(a.start_run[c + 1], D - 1) : D - 1;
    int4 *vout = reinterpret_cast<int4 *>(a.out + head);  // 16-byte aligned frame
    uint32_t pos = P0;

    while (pos < P1 && k_cur < D) {
        const int nw = (int)min((uint32_t)RW, (k_last >= k_cur ? k_last - k_cur : 0u) + 1u);
        __syncthreads();  // previous window no longer in use
        for (int i = tid; i < nw; i += WIN) {
            s_end[i] = a.run_end[k_cur + i];
            s_val[i] = a.run_val[k_cur + i];
        }
        __syncthreads();
        const uint32_t hi = min(P1, s_end[nw - 1]);
        // Whole vectors w cover [hb + 4w, hb + 4w + 4) inside [pos, hi).
        const uint32_t w_lo = pos >= hb ? (pos - hb + 3) >> 2 : 0u;
        const uint32_t w_hi = hi >= hb ? (hi - hb) >> 2 : 0u;

        if (s_end[0] >= hi) {
            // One run covers the whole round: constant stores.
            const int32_t v = s_val[0];
            const int4 vv = make_int4(v, v, v, v);
            uint32_t w = w_lo + tid;
            for (; w + 3 * WIN < w_hi; w += 4 * WIN) {
                __stcs(vout + w, vv);
                __stcs(vout + w + WIN, vv);
                __stcs(vout + w + 2 * WIN, vv);
                __stcs(vout + w + 3 * WIN, vv);
            }
            for (; w < w_hi; w += WIN) __stcs(vout + w, vv);
        } else {
            // Each warp takes a contiguous share of the vectors and its lanes
            // interleave inside it: every store instruction still covers 512
            // contiguous bytes, while a lane's successive vectors are only 128
            // positions apart, so its run index usually stays put or moves to
            // the next run.
            const int lane = tid & 31, warp = tid >> 5;
            const uint32_t nvec = w_hi > w_lo ? w_hi - w_lo : 0u;
            const uint32_t per_warp = ((nvec + (WIN / 32) - 1) / (WIN / 32) + 31) & ~31u;
            const uint32_t wb = w_lo + warp * per_warp;
            const uint32_t we = min(w_hi, wb + per_warp);
            // The run of this lane's last vector (nondecreasing), with its end
            // and value kept in registers: a vector inside the same run needs
            // no shared-memory read.
            int j = 0;
            uint32_t ej = s_end[0];
            int32_t vj = s_val[0];
            for (uint32_t w = wb + lane; w < we; w += 32) {
                const uint32_t q = hb + 4 * w;
                if (ej <= q) {
                    // s_end[nw - 1] > q, so j + 1 <= nw - 1.
                    j = next_run_after(s_end, j + 1, nw - 1, q);
                    ej = s_end[j];
                    vj = s_val[j];
                }
                if (ej >= q + 4) {
                    __stcs(vout + w, make_int4(vj, vj, vj, vj));
                } else {
                    // Positions q..q+3 lie in runs j..j+3 (every run holds at
                    // least one position); q+e lies in run j plus the number of
                    // runs among j, j+1, j+2 that end at or before it.  The
                    // ends are read independently, clamped to the window's last
                    // run (whose end exceeds every position of the round).
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
        // Positions of [pos, hi) outside whole vectors: at most three before
        // the first vector and three after the last.
        if (tid < 8) {
            const uint32_t q_lo = hb + 4 * w_lo, q_hi = hb + 4 * w_hi;
            uint32_t p;
            if (w_lo >= w_hi) {
                p = pos + tid;  // no whole vector: hi - pos < 8
            } else {
                const uint32_t n_front = q_lo - pos;
                p = (uint32_t)tid < n_front ? pos + tid : q_hi + (tid - n_front);
            }
            if (p >= pos && p < hi && (w_lo >= w_hi || p < q_lo || p >= q_hi))
                a.out[p - pb] = s_val[first_run_after(s_end, 0, nw - 1, p)];
        }
        pos = hi;
        k_cur += nw;
    }
}

template <int WIN>
cudaError_t launch_fill_t(const FillArgs &a, cudaStream_t s) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(a.fill_ctas);
    cfg.blockDim = dim3(WIN);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, fill_kernel<WIN>, a);
}

cudaError_t launch_fill(const FillArgs &a, int threads, cudaStream_t s) {
    switch (threads) {
        case 256: return launch_fill_t<256>(a, s);
        case 512: return launch_fill_t<512>(a, s);
        case 1024: return launch_fill_t<1024>(a, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace rtcdf
