// Range-tile histogram for ranges wider than one CTA's shared memory
// (Algorithm 5 for m > 1 tiles), with every key read once.
//
// The paper's multi-tile histogram (Section 3.3) gives each tile its own CTAs,
// and every tile's CTAs scan the whole input: m reads of every key (from L2
// after the first) and m shared-memory updates per key, m - 1 of them for
// keys outside the tile.  Here the m tiles of one range live in the shared
// memory of the C CTAs of a thread-block cluster, and a key is routed to the
// CTA that holds its bin instead of being read by all of them:
//
//   * CTA o of a cluster (o = %cluster_ctarank) owns the values
//     y = key - minVal with y mod C == o, at local bin l = y / C.  Spreading
//     a tile over the range this way keeps the owners evenly loaded for any
//     smooth distribution, peaked or not.
//   * Rounds: every CTA loads 8 keys per thread (two 16-byte vectors) of the
//     cluster's current block of input, and each warp partitions its 256 keys
//     by owner -- ballots on the owner bits give each lane the lanes with the
//     same owner, so its rank among them -- into its own 256-entry region of
//     a staging buffer in shared memory, as 16-bit local bins, with the
//     region's per-owner boundaries beside it.  One cluster barrier later
//     every CTA reads, from each CTA of the cluster (distributed shared
//     memory), the keys that the same-numbered warp routed to it, and adds 1
//     to its bin.  Two staging buffers alternate, so one barrier per round
//     separates a buffer's writes from its reads and its next writes.
//   * A warp slot whose 32 keys are all equal (all-equal input, runs of a
//     sorted input) skips the staging: lane 0 keeps a running (value, count)
//     pair and adds the count to the owner's bin with one remote reduction
//     when the value changes and at the end.
//   * At the end each CTA adds a contiguous part of the global histogram H
//     from all C CTAs' bins (read across the cluster), so the global
//     reductions of a warp hit consecutive words.
//
// Out-of-range keys need no separate test: y >= R maps to a local bin no
// owner counts (bins are clamped to 16 bits, above every owner's width), so
// such a key is counted nowhere and the scan finds the total short of n.
//
// Every CTA of a cluster executes the same sequence of cluster barriers
// (the round count depends on the cluster index only), and no CTA leaves
// while another may still read its shared memory (a final barrier).
#include <map>
#include <mutex>
#include <tuple>

#include "rtcdf_internal.h"

namespace rtcdf {

namespace {

constexpr int kClWarps = kClThreads / 32;
constexpr int kClSlots = 8;                       // keys per thread per round
constexpr int kClWarpKeys = 32 * kClSlots;        // staging entries per warp
constexpr int kClSegStride = 16;                  // u16 boundary entries per warp (C + 1 used)
constexpr uint32_t kClVecPerRound = 2 * kClThreads;  // 16-byte vectors per CTA per round

__device__ __forceinline__ uint32_t cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

// Address of the same shared-memory location in CTA `rank` of the cluster.
__device__ __forceinline__ uint32_t map_rank(uint32_t saddr, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(saddr), "r"(rank));
    return r;
}

// Full cluster barrier: everything written to shared memory before it is
// visible to every CTA of the cluster after it.
__device__ __forceinline__ void cluster_sync_all() {
    asm volatile(
        "barrier.cluster.arrive.release.aligned;\n\t"
        "barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__device__ __forceinline__ uint32_t ld_cluster_u16(uint32_t addr) {
    uint16_t v;
    asm volatile("ld.shared::cluster.u16 %0, [%1];" : "=h"(v) : "r"(addr));
    return v;
}

__device__ __forceinline__ uint32_t ld_cluster_u32(uint32_t addr) {
    uint32_t v;
    asm volatile("ld.shared::cluster.u32 %0, [%1];" : "=r"(v) : "r"(addr));
    return v;
}

__device__ __forceinline__ void red_cluster(uint32_t addr, uint32_t v) {
    asm volatile("red.shared::cluster.add.u32 [%0], %1;" ::"r"(addr), "r"(v) : "memory");
}

// S[l] += 1 when l < w (predicated shared-memory reduction, no branch).
__device__ __forceinline__ void count_local(uint32_t s_base, uint32_t l, uint32_t w) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.lt.u32 p, %0, %1;\n\t"
        "@p red.shared.add.u32 [%2], 1;\n\t}"
        ::"r"(l), "r"(w), "r"(s_base + 4u * l));
}

// Lanes of the warp whose owner equals `o`, from the ballots of the owner bits.
template <int LC>
__device__ __forceinline__ uint32_t owner_mask(const uint32_t (&b)[LC], uint32_t o) {
    uint32_t m = 0xffffffffu;
#pragma unroll
    for (int j = 0; j < LC; j++) m &= ((o >> j) & 1u) ? b[j] : ~b[j];
    return m;
}

template <int C>
__global__ void __launch_bounds__(kClThreads, 1) hist_cluster_kernel(HistArgs a) {
    constexpr int LC = C == 2 ? 1 : (C == 4 ? 2 : 3);
    static_assert((1 << LC) == C, "cluster size is 2, 4 or 8");
    extern __shared__ __align__(16) uint32_t smem[];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t q = cluster_rank();
    const uint32_t cid = blockIdx.x / C, ncl = gridDim.x / C;
    const uint32_t R = a.R, min_u = a.min_u;
    const uint32_t Tc = (R + C - 1) >> LC;         // bins of owner 0 (the widest)
    const uint32_t Tpad = (Tc + 3) & ~3u;
    const uint32_t w_own = (R - q + C - 1) >> LC;  // bins of this owner: y = l * C + q < R
    uint32_t *S = smem;
    uint16_t *box = reinterpret_cast<uint16_t *>(smem + Tpad);  // [2][kClWarps][kClWarpKeys]
    uint16_t *seg = box + 2 * kClWarps * kClWarpKeys;           // [2][kClWarps][kClSegStride]
    const uint32_t s_base = (uint32_t)__cvta_generic_to_shared(S);
    const uint32_t box_base = (uint32_t)__cvta_generic_to_shared(box);
    const uint32_t seg_base = (uint32_t)__cvta_generic_to_shared(seg);

    for (uint32_t i = tid; i < Tpad; i += kClThreads) S[i] = 0;
    // Every CTA's bins are zero before any CTA adds to them.
    cluster_sync_all();

    const int4 *vin = reinterpret_cast<const int4 *>(a.in + a.head);
    const uint64_t nvec = a.nvec;
    const uint64_t per_round = (uint64_t)C * kClVecPerRound;
    const uint64_t total_rounds = (nvec + per_round - 1) / per_round;
    const uint64_t my_rounds = cid < total_rounds ? (total_rounds - cid + ncl - 1) / ncl : 0;
    const int4 none = make_int4((int)(min_u - 1u), (int)(min_u - 1u), (int)(min_u - 1u), (int)(min_u - 1u));
    auto load = [&](uint64_t r, int4 &k0, int4 &k1) {
        const uint64_t v0 = r * per_round + (uint64_t)q * kClVecPerRound + (uint64_t)tid;
        k0 = v0 < nvec ? __ldcs(vin + v0) : none;
        k1 = v0 + kClThreads < nvec ? __ldcs(vin + v0 + kClThreads) : none;
    };
    const uint32_t lt = (1u << lane) - 1u;
    // Lane 0's run of uniform warp slots.
    uint32_t run_y = 0xffffffffu, run_cnt = 0;
    auto flush_run = [&]() {
        if (run_cnt) red_cluster(map_rank(s_base + 4u * (run_y >> LC), run_y & (C - 1)), run_cnt);
    };

    int4 c0 = none, c1 = none, n0 = none, n1 = none;
    if (my_rounds) load(cid, c0, c1);
    for (uint64_t i = 0; i < my_rounds; i++) {
        const uint32_t buf = (uint32_t)(i & 1);
        if (i + 1 < my_rounds) load(cid + (i + 1) * ncl, n0, n1);
        const uint32_t key[kClSlots] = {(uint32_t)c0.x, (uint32_t)c0.y, (uint32_t)c0.z, (uint32_t)c0.w,
                                        (uint32_t)c1.x, (uint32_t)c1.y, (uint32_t)c1.z, (uint32_t)c1.w};
        // ---- produce: this warp's keys by owner into its staging region.
        // Pass 1: keys per owner (lane j < C counts owner j), uniform slots.
        uint32_t skip = 0, total = 0;
#pragma unroll
        for (int s = 0; s < kClSlots; s++) {
            const uint32_t y = key[s] - min_u;
            const uint32_t ly = __shfl_sync(0xffffffffu, y, 0);
            if (__all_sync(0xffffffffu, y == ly)) {
                skip |= 1u << s;
                if (lane == 0 && ly < R) {
                    if (ly == run_y) {
                        run_cnt += 32;
                    } else {
                        flush_run();
                        run_y = ly;
                        run_cnt = 32;
                    }
                }
                continue;
            }
            const uint32_t o = y & (C - 1);
            uint32_t b[LC];
#pragma unroll
            for (int j = 0; j < LC; j++) b[j] = __ballot_sync(0xffffffffu, (o >> j) & 1u);
            total += __popc(owner_mask<LC>(b, (uint32_t)lane));
        }
        // Region boundaries: owner j's keys start at the sum of the counts of
        // owners before it (lanes 0..C-1; lane C holds the region's total).
        uint32_t start = total;
#pragma unroll
        for (int d = 1; d < C; d <<= 1) {
            const uint32_t t = __shfl_up_sync(0xffffffffu, start, d);
            if (lane >= d) start += t;
        }
        start -= total;  // exclusive
        {
            const uint32_t tot = __shfl_sync(0xffffffffu, start + total, C - 1);
            uint16_t *sg = seg + (buf * kClWarps + warp) * kClSegStride;
            if (lane < C) sg[lane] = (uint16_t)start;
            if (lane == C) sg[C] = (uint16_t)tot;
        }
        // Pass 2: each key at its owner's start + keys of that owner before it.
        uint16_t *bx = box + (buf * kClWarps + warp) * kClWarpKeys;
        uint32_t running = start;
#pragma unroll
        for (int s = 0; s < kClSlots; s++) {
            if ((skip >> s) & 1u) continue;
            const uint32_t y = key[s] - min_u;
            const uint32_t o = y & (C - 1);
            const uint32_t l = min(y >> LC, 0xffffu);
            uint32_t b[LC];
#pragma unroll
            for (int j = 0; j < LC; j++) b[j] = __ballot_sync(0xffffffffu, (o >> j) & 1u);
            const uint32_t rank = __popc(owner_mask<LC>(b, o) & lt);
            const uint32_t base = __shfl_sync(0xffffffffu, running, o);
            bx[base + rank] = (uint16_t)l;
            running += __popc(owner_mask<LC>(b, (uint32_t)lane));
        }
        cluster_sync_all();
        // ---- consume: the keys warp `warp` of every CTA routed to this one.
        uint32_t lo = 0, hi = 0;
        if (lane < C) {
            const uint32_t sa = map_rank(seg_base + 2u * ((buf * kClWarps + warp) * kClSegStride + q), lane);
            lo = ld_cluster_u16(sa);
            hi = ld_cluster_u16(sa + 2);
        }
        uint32_t l0[C], l1[C], cnt[C], bxa[C];
#pragma unroll
        for (int p = 0; p < C; p++) {
            const uint32_t lp = __shfl_sync(0xffffffffu, lo, p);
            cnt[p] = __shfl_sync(0xffffffffu, hi, p) - lp;
            bxa[p] = map_rank(box_base + 2u * ((buf * kClWarps + warp) * kClWarpKeys + lp), p);
            l0[p] = (uint32_t)lane < cnt[p] ? ld_cluster_u16(bxa[p] + 2u * lane) : 0xffffu;
            l1[p] = (uint32_t)lane + 32 < cnt[p] ? ld_cluster_u16(bxa[p] + 2u * (lane + 32)) : 0xffffu;
        }
#pragma unroll
        for (int p = 0; p < C; p++) {
            count_local(s_base, l0[p], w_own);
            count_local(s_base, l1[p], w_own);
        }
#pragma unroll
        for (int p = 0; p < C; p++)
            for (uint32_t e = lane + 64; e < cnt[p]; e += 32) count_local(s_base, ld_cluster_u16(bxa[p] + 2u * e), w_own);
        c0 = n0;
        c1 = n1;
    }
    if (lane == 0) flush_run();
    // Unaligned head and ragged tail (at most three keys each): the first
    // cluster's first CTA adds them to their owners' bins directly.
    if (cid == 0 && q == 0 && tid < 8) {
        const uint64_t i = tid < 4 ? (uint64_t)tid : a.head + 4 * nvec + (uint64_t)(tid - 4);
        const bool in_head = tid < 4 && (uint32_t)tid < a.head;
        const bool in_tail = tid >= 4 && i < a.n;
        if (in_head || in_tail) {
            const uint32_t y = (uint32_t)a.in[i] - min_u;
            if (y < R) red_cluster(map_rank(s_base + 4u * (y >> LC), y & (C - 1)), 1u);
        }
    }
    // The scan may be scheduled now; it waits for this grid before reading H.
    asm volatile("griddepcontrol.launch_dependents;");
    cluster_sync_all();
    // Add the cluster's counts to H: this CTA takes local bins [l_lo, l_hi) of
    // every owner, i.e. the consecutive values l * C + o.
    const uint32_t l_lo = (uint32_t)((uint64_t)Tc * q / C), l_hi = (uint32_t)((uint64_t)Tc * (q + 1) / C);
    for (uint32_t idx = tid; idx < (l_hi - l_lo) * C; idx += kClThreads) {
        const uint32_t l = l_lo + (idx >> LC), o = idx & (C - 1);
        const uint32_t y = l * C + o;
        if (y < R) {
            const uint32_t v = ld_cluster_u32(map_rank(s_base + 4u * l, o));
            if (v) atomicAdd(&a.H[y], v);
        }
    }
    // No CTA leaves while another may still read its bins.
    cluster_sync_all();
}

const void *cluster_fn(int C) {
    switch (C) {
        case 2: return (const void *)hist_cluster_kernel<2>;
        case 4: return (const void *)hist_cluster_kernel<4>;
        case 8: return (const void *)hist_cluster_kernel<8>;
        default: return nullptr;
    }
}

}  // namespace

size_t hist_cluster_smem(uint32_t R, int C) {
    const uint32_t Tc = (R + (uint32_t)C - 1) / (uint32_t)C;
    const size_t Tpad = (Tc + 3) & ~3u;
    return Tpad * 4 + 2ull * kClWarps * kClWarpKeys * 2 + 2ull * kClWarps * kClSegStride * 2;
}

// Clusters of C CTAs (one per SM, `smem` bytes each) that fit on the device
// at once; cached per (device, C, smem) so that planning inside CUDA graph
// capture makes no attribute calls.
cudaError_t hist_cluster_max_clusters(int C, size_t smem, int *clusters) {
    static std::mutex mu;
    static std::map<std::tuple<int, int, size_t>, int> cache;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const void *f = cluster_fn(C);
    if (!f) return cudaErrorInvalidValue;
    std::lock_guard<std::mutex> lk(mu);
    auto key = std::make_tuple(dev, C, smem);
    auto it = cache.find(key);
    if (it != cache.end()) {
        *clusters = it->second;
        return cudaSuccess;
    }
    e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int sms = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(sms / C * C));
    cfg.blockDim = dim3(kClThreads);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    e = cudaOccupancyMaxActiveClusters(&n, f, &cfg);
    if (e != cudaSuccess) return e;
    cache[key] = n;
    *clusters = n;
    return cudaSuccess;
}

cudaError_t launch_hist_cluster(const HistArgs &a, int C, uint32_t clusters, size_t smem, cudaStream_t s) {
    const void *f = cluster_fn(C);
    if (!f || clusters == 0) return cudaErrorInvalidValue;
    // hist_cluster_max_clusters() has raised the shared-memory limit for this size.
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(clusters * (unsigned)C);
    cfg.blockDim = dim3(kClThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    void *args[] = {const_cast<HistArgs *>(&a)};
    return cudaLaunchKernelExC(&cfg, f, args);
}

}  // namespace rtcdf
