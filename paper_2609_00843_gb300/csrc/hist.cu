// Range-tile histogram (Algorithm 5, all m tiles in one launch as in Section 3.3).
//
// CTA b works on tile t = b mod m and is the q-th (q = b / m) of the g CTAs of
// that tile -- the paper's interleaving, which keeps the m CTAs that read the
// same part of the input co-resident so that every read after the first is an
// L2 hit.  Each CTA keeps a private histogram S[0..w_t-1] of 32-bit counters
// in shared memory, sweeps the input grid-stride with 16-byte loads, adds 1 to
// S[y] for every key whose position y = key - minVal - b_t inside the tile is
// below w_t (one unsigned compare tests both ends; keys outside [minVal,
// maxVal) fall outside every tile), and finally adds each non-zero S[y] to
// H[b_t + y] with one global atomic.
//
// Out-of-range keys need no per-key test: they are counted by no tile, so the
// histogram total falls short of n, which the scan detects.
//
// On GB300 a single shared-memory copy per CTA sustains the HBM read rate for
// uniform, normal and all-equal inputs alike, so there is no replication.
// Bytes in flight come from unrolled 16-byte loads.  For one tile, bulk L2
// prefetches issued ahead of the loads gave nothing; for 2 to 8 tiles they are
// part of the adaptive form below.
#include <map>
#include <mutex>
#include <tuple>

#include "rtcdf_internal.h"

namespace rtcdf {

template <bool STREAMING>
__device__ __forceinline__ int4 load_vec(const int4 *p) {
    if (STREAMING) return __ldcs(p);  // read once: evict first
    return __ldg(p);                  // re-read by the other tiles' CTAs: keep in L2
}

// S[y] += 1 when y < w, as a predicated shared-memory reduction (no branch).
// No "memory" clobber: S is only otherwise touched on the far side of a
// __syncthreads(), and the clobber would stop the next loads from being
// scheduled early.
__device__ __forceinline__ void count_key(uint32_t s_base, uint32_t y, uint32_t w) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.lt.u32 p, %0, %1;\n\t"
        "@p red.shared.add.u32 [%2], 1;\n\t}"
        ::"r"(y), "r"(w), "r"(s_base + 4u * y));
}

// S[min(y, w)] += 1: a key outside the tile adds to the trash word S[w]
// instead of being predicated off; all such lanes of a warp hit one address
// with an immediate increment and are combined.
__device__ __forceinline__ void count_key_trash(uint32_t s_base, uint32_t y, uint32_t w) {
    const uint32_t yy = y < w ? y : w;
    asm volatile("red.shared.add.u32 [%0], 1;" ::"r"(s_base + 4u * yy));
}

__device__ __forceinline__ void prefetch_l2(const void *p, uint32_t bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// ADAPT (2 to 8 tiles): out-of-tile keys go to a trash word, and the m CTAs
// that read the same vectors prefetch them into L2 two iterations ahead --
// unless the input is long (more than 2^28 keys) and a sample of it (one
// vector per warp) shows one tile holding more than 2/m of the keys without
// holding nearly all of them: the CTAs of such tiles then run at unequal
// speeds, over a long input the heavy tile's CTAs fall so far behind that
// the lines prefetched for them are gone, and the prefetches cost more than
// they save (n = 1e9, R = 2^18, normal keys: 3.04 ms with them against 2.93
// without; n = 1e8: 0.312 against 0.322 ms, measured).  The choice changes
// only the speed, never the counts.
template <bool STREAMING, int UNROLL, bool ADAPT>
__global__ void __launch_bounds__(1024) hist_kernel(HistArgs a) {
    extern __shared__ uint32_t S[];
    __shared__ uint32_t s_tc[8];
    const uint32_t t = blockIdx.x % a.m;
    const uint32_t q = blockIdx.x / a.m;
    const uint32_t b = t * a.T;
    const uint32_t w = min(a.T, a.R - b);
    const int tid = threadIdx.x, nt = blockDim.x;

    for (uint32_t i = tid; i < w + (ADAPT ? 1u : 0u); i += nt) S[i] = 0;  // + the trash word
    if (ADAPT && tid < 8) s_tc[tid] = 0;
    __syncthreads();

    const uint32_t base = a.min_u + b;  // key - base = position inside the tile
    const uint32_t s_base = (uint32_t)__cvta_generic_to_shared(S);

    // Grid-stride over 16-byte vectors: the g CTAs of a tile sweep the input
    // together, and the CTAs of the other tiles with the same q read the same
    // addresses at the same time (served from L2 after the first).
    const int4 *vin = reinterpret_cast<const int4 *>(a.in + a.head);
    const uint64_t stride = (uint64_t)a.g * nt;
    const uint64_t nvec = a.nvec;
    uint64_t v = (uint64_t)q * nt + tid;
    bool pf = false;
    if (ADAPT) {
        if ((tid & 31) == 0 && v < nvec) {
            const int4 k = __ldg(vin + v);
            const uint32_t y[4] = {(uint32_t)k.x - a.min_u, (uint32_t)k.y - a.min_u,
                                   (uint32_t)k.z - a.min_u, (uint32_t)k.w - a.min_u};
#pragma unroll
            for (int e = 0; e < 4; e++)
                if (y[e] < a.R) atomicAdd(&s_tc[min(y[e] / a.T, 7u)], 1u);
        }
        __syncthreads();
        uint32_t tot = 0, mx = 0;
#pragma unroll
        for (int i = 0; i < 8; i++) {
            tot += s_tc[i];
            mx = max(mx, s_tc[i]);
        }
        pf = tot > 0 && (a.nvec <= (1ull << 26) || mx * a.m <= 2 * tot || mx * 10 >= 9 * tot);
    }
    uint64_t vb = (uint64_t)q * nt;  // thread 0's vector of the iteration
    auto count_vec = [&](const int4 k) {
        if (ADAPT) {
            count_key_trash(s_base, (uint32_t)k.x - base, w);
            count_key_trash(s_base, (uint32_t)k.y - base, w);
            count_key_trash(s_base, (uint32_t)k.z - base, w);
            count_key_trash(s_base, (uint32_t)k.w - base, w);
        } else {
            count_key(s_base, (uint32_t)k.x - base, w);
            count_key(s_base, (uint32_t)k.y - base, w);
            count_key(s_base, (uint32_t)k.z - base, w);
            count_key(s_base, (uint32_t)k.w - base, w);
        }
    };
    if (!ADAPT) {
        // One tile: UNROLL vectors loaded, then counted (32 registers, so
        // that two CTAs fit an SM: with the pipeline below these CTAs took 64
        // registers and the 12-array step on three streams got slower).
        for (; v + (UNROLL - 1) * stride < nvec; v += UNROLL * stride) {
            int4 k[UNROLL];
#pragma unroll
            for (int u = 0; u < UNROLL; u++) k[u] = load_vec<STREAMING>(vin + v + u * stride);
#pragma unroll
            for (int u = 0; u < UNROLL; u++) count_vec(k[u]);
        }
    } else {
        // Several tiles (one CTA per SM, its shared memory being the tile):
        // software pipelined, the next P vectors in flight while the last P
        // are counted (R = 2^18 uniform, n = 1e8: 0.272 against 0.281 ms per
        // sort, measured).
        constexpr int P = UNROLL < 6 ? UNROLL : 6;
        if (v + (P - 1) * stride < nvec) {
            int4 kn[P];
#pragma unroll
            for (int u = 0; u < P; u++) kn[u] = load_vec<STREAMING>(vin + v + u * stride);
            v += P * stride;
            vb += P * stride;
            for (; v + (P - 1) * stride < nvec; v += P * stride, vb += P * stride) {
                if (pf && tid == 0) {
                    // This CTA's share (u = t, t + m, ...) of the vectors its
                    // group loads two stages from now.
                    const uint64_t ahead = vb + 2ull * P * stride;
                    for (uint32_t u = t; u < (uint32_t)P; u += a.m) {
                        const uint64_t s0 = ahead + (uint64_t)u * stride;
                        if (s0 + nt <= nvec) prefetch_l2(vin + s0, 16u * nt);
                    }
                }
                int4 kc[P];
#pragma unroll
                for (int u = 0; u < P; u++) kc[u] = kn[u];
#pragma unroll
                for (int u = 0; u < P; u++) kn[u] = load_vec<STREAMING>(vin + v + u * stride);
#pragma unroll
                for (int u = 0; u < P; u++) count_vec(kc[u]);
            }
#pragma unroll
            for (int u = 0; u < P; u++) count_vec(kn[u]);
        }
    }
    for (; v < nvec; v += stride) {
        int4 k0 = load_vec<STREAMING>(vin + v);
        count_key(s_base, (uint32_t)k0.x - base, w);
        count_key(s_base, (uint32_t)k0.y - base, w);
        count_key(s_base, (uint32_t)k0.z - base, w);
        count_key(s_base, (uint32_t)k0.w - base, w);
    }
    if (q == 0) {
        // Unaligned head and ragged tail, scalar.
        if ((uint32_t)tid < a.head) count_key(s_base, (uint32_t)a.in[tid] - base, w);
        for (uint64_t i = a.head + 4 * nvec + tid; i < a.n; i += nt)
            count_key(s_base, (uint32_t)a.in[i] - base, w);
    }
    // The scan may be scheduled now; it waits for this grid to finish before
    // reading H.
    asm volatile("griddepcontrol.launch_dependents;");

    __syncthreads();
    uint32_t *H = a.H + b;
    for (uint32_t i = tid; i < w; i += nt) {
        uint32_t c = S[i];
        if (c) atomicAdd(&H[i], c);
    }
}

// Kernel variant: streaming loads for one tile; the adaptive form for 2 to 8
// tiles; the plain predicated form beyond.
enum HistVariant { kHistStreaming = 0, kHistAdaptive = 1, kHistPlain = 2 };
int hist_variant(bool streaming, uint32_t m) {
    return streaming ? kHistStreaming : (m <= 8 ? kHistAdaptive : kHistPlain);
}

const void *hist_fn(int variant, int unroll) {
    const bool deep = unroll == 8;
    switch (variant) {
        case kHistStreaming:
            return deep ? (const void *)hist_kernel<true, 8, false> : (const void *)hist_kernel<true, 4, false>;
        case kHistAdaptive:
            return deep ? (const void *)hist_kernel<false, 8, true> : (const void *)hist_kernel<false, 4, true>;
        default:
            return deep ? (const void *)hist_kernel<false, 8, false> : (const void *)hist_kernel<false, 4, false>;
    }
}

// The deep form (UNROLL = 8) when only one CTA fits on an SM: eight loads in
// flight per thread in the one-tile and plain forms, a six-deep pipeline in
// the 2-to-8-tile form.
int hist_unroll(size_t smem) { return smem > 114 * 1024 ? 8 : 4; }

cudaError_t launch_hist(const HistArgs &a, int threads, size_t smem, bool streaming,
                        cudaStream_t s) {
    // hist_max_ctas_per_sm() has raised the shared-memory limit for this size.
    dim3 grid(a.m * a.g);
    void *args[] = {const_cast<HistArgs *>(&a)};
    return cudaLaunchKernel(hist_fn(hist_variant(streaming, a.m), hist_unroll(smem)), grid, dim3(threads),
                            args, smem, s);
}

// Occupancy of the histogram kernel for a launch shape, cached per device so
// that planning a sort inside CUDA graph capture makes no attribute calls.
cudaError_t hist_max_ctas_per_sm(int threads, size_t smem, bool streaming, int *ctas) {
    static std::mutex mu;
    static std::map<std::tuple<int, int, size_t, bool>, int> cache;
    static std::map<std::pair<int, bool>, size_t> smem_limit;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(mu);
    auto key = std::make_tuple(dev, threads, smem, streaming);
    auto it = cache.find(key);
    if (it != cache.end()) {
        *ctas = it->second;
        return cudaSuccess;
    }
    // The adaptive and plain multi-tile variants share the same sizes.
    const void *f = hist_fn(streaming ? kHistStreaming : kHistAdaptive, hist_unroll(smem));
    size_t &lim = smem_limit[std::make_pair(dev, streaming)];
    if (smem > lim) {
        for (int v : {kHistStreaming, kHistAdaptive, kHistPlain}) {
            if ((v == kHistStreaming) != streaming) continue;
            for (int u : {4, 8}) {
                e = cudaFuncSetAttribute(hist_fn(v, u), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
                if (e != cudaSuccess) return e;
            }
        }
        lim = smem;
    }
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas, f, threads, smem);
    if (e != cudaSuccess) return e;
    cache[key] = *ctas;
    return cudaSuccess;
}

}  // namespace rtcdf
