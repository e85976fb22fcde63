// Output generation from the local CDFs (Algorithm 7), all tiles in one launch.
//
// Algorithm 7 assigns output positions to threads and finds the value at
// position p as the smallest x with C[x] >= p + 1 by binary search.  Here each
// CTA owns a contiguous range of positions [P0, P1) and walks the run table
// built by the scan (run_end[k] = exclusive end of the k-th non-empty value,
// run_val[k] = that value's key): it copies a window of consecutive runs into
// shared memory, then every thread writes 16-byte vectors of its positions,
// finding the run of a position with the same rule (smallest k with
// run_end[k] >= p + 1), starting from the run of its previous vector.  When a
// whole vector lies inside one run -- the common case -- that is one shared
// load and one compare before the store.  Vectors cut by the window edge or
// by the array's ends are written element by element.
//
// The CTA also clears the scan's lookback state so the workspace is ready for
// the next sort.
#include "rtcdf_internal.h"

namespace rtcdf {

template <int WIN>
__global__ void __launch_bounds__(WIN) fill_kernel(FillArgs a) {
    __shared__ uint32_t s_end[WIN];
    __shared__ int32_t s_val[WIN];
    const int tid = threadIdx.x;
    const uint32_t c = blockIdx.x;

    for (uint32_t i = c * WIN + tid; i < a.scan_chunks; i += a.fill_ctas * WIN) a.scan_state[i] = 0;
    if (c == 0 && tid == 0) a.ctl->scan_ticket = 0;

    const int64_t n = (int64_t)a.n, head = a.head;
    const int64_t P0 = (c == 0) ? 0 : head + (int64_t)c * (int64_t)a.fill_chunk;
    const int64_t P1 = (c + 1 == a.fill_ctas) ? n : head + (int64_t)(c + 1) * (int64_t)a.fill_chunk;
    const uint32_t D = a.ctl->num_runs;
    uint32_t k_cur = a.start_run[c];
    int4 *vout = reinterpret_cast<int4 *>(a.out + head);  // 16-byte aligned frame
    int64_t pos = P0;

    while (pos < P1 && k_cur < D) {
        const int nw = (int)min((uint32_t)WIN, D - k_cur);
        __syncthreads();  // previous window no longer in use
        if (tid < nw) {
            s_end[tid] = a.run_end[k_cur + tid];
            s_val[tid] = a.run_val[k_cur + tid];
        }
        __syncthreads();
        const int64_t hi = min(P1, (int64_t)s_end[nw - 1]);
        // Vectors w cover positions [head + 4w, head + 4w + 4); w may be -1 for
        // the unaligned head.
        const int64_t w_first = (pos - head >= 0) ? (pos - head) / 4 : -1;
        const int64_t w_last = (hi - 1 - head >= 0) ? (hi - 1 - head) / 4 : -1;

        if (s_end[0] >= hi) {
            // One run covers the whole round: constant stores.
            const int32_t v = s_val[0];
            const int4 vv = make_int4(v, v, v, v);
            int64_t w = w_first + tid;
            for (; w <= w_last; w += WIN) {
                const int64_t q = head + 4 * w;
                if (q >= pos && q + 4 <= hi) {
                    __stcs(vout + w, vv);
                } else {
#pragma unroll
                    for (int e = 0; e < 4; e++) {
                        const int64_t p = q + e;
                        if (p >= pos && p < hi) a.out[p] = v;
                    }
                }
            }
        } else {
            int j = 0;  // run index within the window, nondecreasing per thread
            for (int64_t w = w_first + tid; w <= w_last; w += WIN) {
                const int64_t q = head + 4 * w;
                const int64_t q0 = q > pos ? q : pos;
                // Smallest j with s_end[j] > q0 (binary search above the last hit).
                if ((int64_t)s_end[j] <= q0) {
                    int lo = j + 1, hi_i = nw - 1;
                    while (lo < hi_i) {
                        int mid = (lo + hi_i) >> 1;
                        if ((int64_t)s_end[mid] > q0) hi_i = mid; else lo = mid + 1;
                    }
                    j = lo;
                }
                if (q >= pos && q + 4 <= hi) {
                    if ((int64_t)s_end[j] >= q + 4) {
                        const int32_t v = s_val[j];
                        __stcs(vout + w, make_int4(v, v, v, v));
                    } else {
                        int32_t r[4];
                        int jj = j;
#pragma unroll
                        for (int e = 0; e < 4; e++) {
                            while ((int64_t)s_end[jj] <= q + e) jj++;
                            r[e] = s_val[jj];
                        }
                        __stcs(vout + w, make_int4(r[0], r[1], r[2], r[3]));
                    }
                } else {
                    int jj = j;
                    for (int e = 0; e < 4; e++) {
                        const int64_t p = q + e;
                        if (p < pos || p >= hi) continue;
                        while ((int64_t)s_end[jj] <= p) jj++;
                        a.out[p] = s_val[jj];
                    }
                }
            }
        }
        pos = hi;
        k_cur += nw;
    }
}

cudaError_t launch_fill(const FillArgs &a, int threads, cudaStream_t s) {
    switch (threads) {
        case 256: fill_kernel<256><<<a.fill_ctas, 256, 0, s>>>(a); break;
        case 512: fill_kernel<512><<<a.fill_ctas, 512, 0, s>>>(a); break;
        case 1024: fill_kernel<1024><<<a.fill_ctas, 1024, 0, s>>>(a); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace rtcdf
