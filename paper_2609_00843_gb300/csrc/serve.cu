// Continuous-batching sort server (rtcdf_serve_* in include/rtcdf.h).
//
// A request is "sort these n keys from [minVal, maxVal)".  The server keeps
// one device slab of `budget_bytes`; a request is admitted when its slot (input
// + output, 8n bytes) fits, in arrival order.  Admitted requests whose input is
// in place are launched as soon as one of `num_streams` streams is free:
// requests with at least `single_min_keys` keys alone, through the single-array
// pipeline (Algorithms 4-7, three kernels); all other pending requests together,
// as one segmented sort (its three launches; a lone small request, under light
// load, also takes the single-array pipeline).  New arrivals keep being admitted while
// earlier launches run, launches on different streams overlap on the device,
// and a request's slot is released as soon as its launch completes.  Results
// stay on the device; an optional order-dependent digest of each sorted output
// lets a caller compare runs.
#include <chrono>
#include <cstring>
#include <deque>
#include <map>
#include <thread>
#include <vector>

#include "../../include/rtcdf.h"
#include "batched.h"

using namespace rtcdf;

namespace {

using Clock = std::chrono::steady_clock;

// First-fit allocator over [0, cap) in 256-byte units, with coalescing.
class Slab {
  public:
    explicit Slab(size_t cap) { free_[0] = cap / 256 * 256; }
    bool alloc(size_t bytes, size_t *off) {
        bytes = (bytes + 255) / 256 * 256;
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                *off = it->first;
                const size_t rest = it->second - bytes, at = it->first + bytes;
                free_.erase(it);
                if (rest) free_[at] = rest;
                used_ += bytes;
                if (used_ > peak_) peak_ = used_;
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t bytes) {
        bytes = (bytes + 255) / 256 * 256;
        used_ -= bytes;
        auto it = free_.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
    size_t peak() const { return peak_; }
    size_t used() const { return used_; }

  private:
    std::map<size_t, size_t> free_;
    size_t used_ = 0, peak_ = 0;
};

__device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// One digest per request: sum over positions i of mix64((i << 32) | out[i]),
// mod 2^64 -- order-dependent, so two equal digests mean equal arrays with
// overwhelming probability.  blockIdx.y selects the request.
struct DigestSeg {
    uint64_t out_off, n, slot;
};

__global__ void digest_kernel(const int32_t *base, const DigestSeg *segs, uint64_t *digests) {
    const DigestSeg d = segs[blockIdx.y];
    const int32_t *out = base + d.out_off;
    uint64_t h = 0;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < d.n;
         i += (uint64_t)gridDim.x * blockDim.x)
        h += mix64((i << 32) | (uint32_t)out[i]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) h += __shfl_xor_sync(0xffffffffu, h, o);
    if ((threadIdx.x & 31) == 0 && h) atomicAdd((unsigned long long *)&digests[d.slot], (unsigned long long)h);
}

struct Launch {
    cudaEvent_t done;
    int stream;
    std::vector<int64_t> reqs;
    size_t ws_off = 0, ws_bytes = 0;  // batch workspace + tables in the slab
    bool batched = false;
    bool large = false;   // a request of at least single_min_keys keys
};

double secs(Clock::time_point t0) {
    return std::chrono::duration<double>(Clock::now() - t0).count();
}

// Everything rtcdf_serve_trace creates, released by the destructor on every
// way out -- a normal return, an error, or an exception (a failed host
// allocation) -- after the device has finished with it.
struct ServeResources {
    char *slab = nullptr;
    uint64_t *d_digest = nullptr;
    std::vector<cudaStream_t> streams, fill_streams;
    std::vector<char *> stage;
    std::vector<cudaEvent_t> ev_pool, req_ev;
    std::vector<Launch> inflight;
    ~ServeResources() {
        cudaDeviceSynchronize();  // nothing in flight still uses the slab or the staging
        for (cudaStream_t s : streams)
            if (s) cudaStreamDestroy(s);
        for (cudaStream_t s : fill_streams)
            if (s) cudaStreamDestroy(s);
        for (char *p : stage)
            if (p) cudaFreeHost(p);
        for (cudaEvent_t e : ev_pool) cudaEventDestroy(e);
        for (cudaEvent_t e : req_ev)
            if (e) cudaEventDestroy(e);
        for (Launch &L : inflight) cudaEventDestroy(L.done);  // launches left by an error
        cudaFree(d_digest);
        cudaFree(slab);
    }
};

}  // namespace

extern "C" {

rtcdf_status rtcdf_serve_trace(const rtcdf_server_config *cfg, const rtcdf_request *reqs,
                               int64_t count, rtcdf_result *results, rtcdf_serve_stats *stats) try {
    if (!cfg || (count > 0 && (!reqs || !results)) || count < 0) return RTCDF_ERR_INVALID_ARG;
    if (!cfg->fill || cfg->num_streams < 1 || cfg->num_streams > 16 || cfg->max_batch < 1)
        return RTCDF_ERR_INVALID_ARG;
    int64_t maxR = 1;
    for (int64_t i = 0; i < count; i++) {
        const int64_t R = reqs[i].maxVal - reqs[i].minVal;
        if (R <= 0 || R > (int64_t)kBatchMaxR || reqs[i].minVal < INT32_MIN ||
            reqs[i].maxVal > ((int64_t)1 << 31) || reqs[i].n >= (1ull << 32))
            return RTCDF_ERR_RANGE;
        if (R > maxR) maxR = R;
    }
    const int K = cfg->num_streams;
    const bool want_digest = cfg->digests != 0;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return RTCDF_ERR_CUDA;
    // A failed setup call is remembered and skips the trace; everything
    // created before it is released at the end as usual.
    rtcdf_status err = RTCDF_OK;
    auto check = [&](cudaError_t e, rtcdf_status code) {
        if (e != cudaSuccess && !err) err = code;
    };

    ServeResources res;
    // Device slab = admission budget.  Per stream, a single-array workspace
    // for the widest range is carved out of it first.
    char *&slab = res.slab;
    if (cudaMalloc(&slab, cfg->budget_bytes) != cudaSuccess) return RTCDF_ERR_NO_MEMORY;
    Slab alloc(cfg->budget_bytes);
    size_t ws_bytes = 0;
    rtcdf_workspace_size(maxR, &ws_bytes);
    // With large_priority, large requests get K streams of their own at the
    // device's highest stream priority ([K, 2K)), batches the default ones
    // ([0, K)): the block scheduler then issues a large sort's CTAs before
    // the batches' whenever both wait, so it runs about as fast as alone
    // while batches fill the gaps.  Stream priority is a property of the
    // process's streams, not a device setting.
    const bool prio = cfg->large_priority != 0;
    const int NS = prio ? 2 * K : K;
    int prio_least = 0, prio_greatest = 0;
    if (prio) check(cudaDeviceGetStreamPriorityRange(&prio_least, &prio_greatest), RTCDF_ERR_CUDA);
    auto make_stream = [&](cudaStream_t *st, bool high) {
        if (high) check(cudaStreamCreateWithPriority(st, cudaStreamNonBlocking, prio_greatest), RTCDF_ERR_CUDA);
        else check(cudaStreamCreateWithFlags(st, cudaStreamNonBlocking), RTCDF_ERR_CUDA);
    };
    std::vector<size_t> ws_off(NS);
    std::vector<cudaStream_t> &streams = res.streams;
    streams.assign(NS, nullptr);
    for (int k = 0; k < NS; k++) {
        if (!alloc.alloc(ws_bytes, &ws_off[k])) return RTCDF_ERR_NO_MEMORY;
        check(cudaMemset(slab + ws_off[k], 0, ws_bytes), RTCDF_ERR_CUDA);
        make_stream(&streams[k], k >= K);
    }
    // Inputs are written on their own streams (round robin), so writing the
    // next arrivals overlaps the sorts already running.  Each request's write
    // is marked by an event (from a pool, returned when the request retires):
    // a launch waits for its own requests' inputs only.  With large_priority
    // a large request's keys are written on high-priority streams too.
    std::vector<cudaStream_t> &fill_streams = res.fill_streams;
    fill_streams.assign(NS, nullptr);
    for (int k = 0; k < NS; k++) make_stream(&fill_streams[k], k >= K);
    int fill_rr = 0, fill_rr_hi = 0;
    std::vector<cudaEvent_t> &ev_pool = res.ev_pool, &req_ev = res.req_ev;
    req_ev.assign((size_t)count, nullptr);
    auto take_event = [&]() {
        cudaEvent_t e = nullptr;
        if (!ev_pool.empty()) {
            e = ev_pool.back();
            ev_pool.pop_back();
        } else if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
            e = nullptr;
        }
        return e;
    };
    uint64_t *&d_digest = res.d_digest;
    if (want_digest) {
        const size_t db = sizeof(uint64_t) * (size_t)std::max<int64_t>(1, count);
        check(cudaMalloc(&d_digest, db), RTCDF_ERR_NO_MEMORY);
        if (d_digest) check(cudaMemset(d_digest, 0, db), RTCDF_ERR_CUDA);
    }
    // Pinned staging for plan uploads, one per stream (reused once that
    // stream's previous launch has completed).
    const size_t stage_bytes = 64u << 20;
    std::vector<char *> &stage = res.stage;
    // Every launch stream has one; a high-priority stream only ever uploads
    // the digest entry of its single request, so a small one does.
    stage.assign(NS, nullptr);
    std::vector<size_t> stage_cap(NS, 0);
    for (int k = 0; k < NS; k++) {
        stage_cap[k] = k < K ? stage_bytes : (size_t)4096;
        check(cudaMallocHost(&stage[k], stage_cap[k]), RTCDF_ERR_NO_MEMORY);
    }
    check(cudaDeviceSynchronize(), RTCDF_ERR_CUDA);

    std::vector<size_t> slot_off(count, 0), slot_bytes(count, 0);
    for (int64_t i = 0; i < count; i++) {
        memset(&results[i], 0, sizeof(rtcdf_result));
        results[i].status = -1;
    }
    std::deque<int64_t> pending;            // admitted, input enqueued
    std::vector<Launch> &inflight = res.inflight;
    std::vector<bool> stream_busy(NS, false);
    int64_t next = 0, done = 0;
    uint64_t launches_batched = 0, launches_single = 0, batched_requests = 0;
    int max_inflight = 0;
    const size_t reserve = std::min<size_t>(cfg->budget_bytes / 8, (size_t)1 << 30);
    int batch_cap = cfg->max_batch;
    const int max_large = cfg->max_large_inflight > 0 ? cfg->max_large_inflight : K;
    int large_inflight = 0;
    int64_t pending_large = 0;  // admitted large requests not launched yet
    const Clock::time_point t0 = Clock::now();

    while (done < count && !err) {
        bool progressed = false;
        const double now = secs(t0);
        // 1. Admit arrived requests, in order, while their slots fit.
        while (next < count && reqs[next].arrival_s <= now) {
            const rtcdf_request &r = reqs[next];
            size_t off = 0;
            const size_t bytes = (size_t)r.n * 8 + 512;
            if ((size_t)r.n * 8 + 512 + reserve > cfg->budget_bytes - (size_t)NS * ws_bytes) {
                results[next].status = RTCDF_ERR_NO_MEMORY;  // can never fit
                results[next].admit_s = results[next].done_s = secs(t0);
                next++, done++;
                continue;
            }
            // Keep `reserve` bytes free for launch tables and batch workspaces.
            if (alloc.used() + (bytes + 255) / 256 * 256 + reserve > cfg->budget_bytes ||
                !alloc.alloc(bytes, &off))
                break;  // wait for memory (in order)
            slot_off[next] = off;
            slot_bytes[next] = bytes;
            int32_t *in = reinterpret_cast<int32_t *>(slab + off);
            int fs;
            if (prio && r.n >= cfg->single_min_keys) {
                fs = K + fill_rr_hi;
                fill_rr_hi = (fill_rr_hi + 1) % K;
            } else {
                fs = fill_rr;
                fill_rr = (fill_rr + 1) % K;
            }
            if (r.n && !cfg->fill_at_launch) {
                if (cfg->fill(in, r.n, 0, r.minVal, r.maxVal - r.minVal, r.dist, r.seed,
                              (rtcdf_stream_t)fill_streams[fs]) != 0) {
                    err = RTCDF_ERR_CUDA;
                    break;
                }
                req_ev[next] = take_event();
                if (!req_ev[next] || cudaEventRecord(req_ev[next], fill_streams[fs]) != cudaSuccess) {
                    err = RTCDF_ERR_CUDA;
                    break;
                }
            }
            results[next].admit_s = secs(t0);
            pending.push_back(next);
            if (r.n >= cfg->single_min_keys) pending_large++;
            next++;
            progressed = true;
        }
        // 2. Launch pending requests on free streams.
        while (!pending.empty() && !err) {
            // A large request alone (while fewer than max_large of them run),
            // or every small pending request together.
            const int64_t head = pending.front();
            // The limit on large launches in flight holds while the waiting
            // large requests are fewer than large_queue_burst; a backlog
            // lets them use every stream.
            const int large_cap =
                (cfg->large_queue_burst > 0 && pending_large >= cfg->large_queue_burst) ? K : max_large;
            const bool take_large = reqs[head].n >= cfg->single_min_keys && large_inflight < large_cap;
            const int k_lo = (prio && take_large) ? K : 0, k_hi = prio ? k_lo + K : K;
            int k = -1;
            for (int j = k_lo; j < k_hi; j++)
                if (!stream_busy[j]) { k = j; break; }
            if (k < 0) break;
            cudaStream_t s = streams[k];
            Launch L;
            L.stream = k;
            if (take_large) {
                pending.pop_front();
                pending_large--;
                L.reqs.push_back(head);
                L.large = true;
            } else {
                for (auto it = pending.begin(); it != pending.end() && (int)L.reqs.size() < batch_cap;) {
                    if (reqs[*it].n < cfg->single_min_keys) {
                        L.reqs.push_back(*it);
                        it = pending.erase(it);
                    } else {
                        ++it;
                    }
                }
                if (L.reqs.empty()) break;  // only large requests wait: a large launch must finish
            }
            for (int64_t i : L.reqs)  // inputs written before the sort reads them
                if (req_ev[i]) cudaStreamWaitEvent(s, req_ev[i], 0);
            if (cfg->fill_at_launch) {
                // The keys are written on the launch's own stream right before
                // its sort, as a one-at-a-time server writes them.
                for (int64_t i : L.reqs) {
                    if (!reqs[i].n) continue;
                    int32_t *in = reinterpret_cast<int32_t *>(slab + slot_off[i]);
                    if (cfg->fill(in, reqs[i].n, 0, reqs[i].minVal, reqs[i].maxVal - reqs[i].minVal, reqs[i].dist,
                                  reqs[i].seed, (rtcdf_stream_t)s) != 0) {
                        err = RTCDF_ERR_CUDA;
                        break;
                    }
                }
                if (err) break;
            }
            const double launch_t = secs(t0);
            // A lone request (large, or small with nothing to batch it with --
            // light load) goes through the single-array pipeline, which needs
            // no table upload.
            const bool single = L.reqs.size() == 1;
            // One slab region per launch, released when it completes:
            // [segment table | work items | digest table | batch workspace].
            HostPlan hp;
            std::vector<SegSpec> spec;
            if (!single) {
                spec.resize(L.reqs.size());
                for (size_t j = 0; j < L.reqs.size(); j++) {
                    const int64_t i = L.reqs[j];
                    const uint64_t in_off = slot_off[i] / 4;  // input at the slot start, output after it
                    spec[j] = SegSpec{in_off, in_off + reqs[i].n, reqs[i].n, reqs[i].minVal, reqs[i].maxVal};
                }
                if (build_host_plan(spec.data(), (uint32_t)spec.size(), &hp)) { err = RTCDF_ERR_RANGE; break; }
            }
            std::vector<DigestSeg> dg;
            if (want_digest) {
                dg.resize(L.reqs.size());
                for (size_t j = 0; j < L.reqs.size(); j++) {
                    const int64_t i = L.reqs[j];
                    dg[j] = DigestSeg{slot_off[i] / 4 + reqs[i].n, reqs[i].n, (uint64_t)i};
                }
            }
            const size_t seg_b = hp.segs.size() * sizeof(BatchSeg);
            const size_t item_b = hp.items.size() * sizeof(BatchItem);
            const size_t dig_at = (seg_b + item_b + 15) / 16 * 16;
            const size_t dig_b = dg.size() * sizeof(DigestSeg);
            const size_t tab_b = (dig_at + dig_b + 255) / 256 * 256;
            const size_t wsb = hp.ws_words * 4;
            if (tab_b > stage_cap[k]) { err = RTCDF_ERR_NO_MEMORY; break; }
            if (tab_b + wsb > 0 && !alloc.alloc(tab_b + wsb, &L.ws_off)) {
                if (inflight.empty() && L.reqs.size() > 1) {
                    // Nothing will free memory: retry with the first request alone.
                    for (auto it = L.reqs.rbegin(); it != L.reqs.rend(); ++it) pending.push_front(*it);
                    batch_cap = 1;
                    continue;
                }
                if (inflight.empty()) { err = RTCDF_ERR_NO_MEMORY; break; }
                for (auto it = L.reqs.rbegin(); it != L.reqs.rend(); ++it) pending.push_front(*it);
                break;  // wait for a launch to complete
            }
            L.ws_bytes = tab_b + wsb;
            char *tab = slab + L.ws_off;
            if (seg_b + item_b + dig_b) {
                memcpy(stage[k], hp.segs.data(), seg_b);
                memcpy(stage[k] + seg_b, hp.items.data(), item_b);
                memcpy(stage[k] + dig_at, dg.data(), dig_b);
                if (cudaMemcpyAsync(tab, stage[k], dig_at + dig_b, cudaMemcpyHostToDevice, s) != cudaSuccess) {
                    err = RTCDF_ERR_CUDA;
                    break;
                }
            }
            if (single) {
                const int64_t i = L.reqs[0];
                int32_t *in = reinterpret_cast<int32_t *>(slab + slot_off[i]);
                int32_t *out = in + reqs[i].n;
                const rtcdf_status st = rtcdf_sort_ws(in, out, reqs[i].n, reqs[i].minVal, reqs[i].maxVal,
                                                      slab + ws_off[k], ws_bytes, (rtcdf_stream_t)s);
                if (st) { err = st; break; }
                launches_single++;
            } else {
                uint32_t *ws = reinterpret_cast<uint32_t *>(tab + tab_b);
                if (cudaMemsetAsync(ws, 0, wsb, s) != cudaSuccess) {
                    err = RTCDF_ERR_CUDA;
                    break;
                }
                BatchArgs a;
                a.in = reinterpret_cast<const int32_t *>(slab);
                a.out = reinterpret_cast<int32_t *>(slab);
                a.segs = reinterpret_cast<const BatchSeg *>(tab);
                a.items = reinterpret_cast<const BatchItem *>(tab + seg_b);
                a.n_first = hp.n_first;
                a.n_scan = hp.n_scan;
                a.n_small2 = hp.n_small2;
                a.n_fill = hp.n_fill;
                a.num_segs = (uint32_t)hp.segs.size();
                a.ws_u32 = ws;
                a.ctl = reinterpret_cast<BatchCtl *>(ws + hp.ctl_off);
                a.seg_ctl = reinterpret_cast<BatchSegCtl *>(ws + hp.segctl_off);
                if (launch_batched(a, s) != cudaSuccess) {
                    err = RTCDF_ERR_CUDA;
                    break;
                }
                L.batched = true;
                launches_batched++;
                batched_requests += L.reqs.size();
            }
            if (want_digest) {
                uint32_t chunks = 1;
                for (const DigestSeg &d : dg)
                    chunks = std::max<uint32_t>(chunks, (uint32_t)std::min<uint64_t>(256, (d.n + 8191) / 8192));
                for (size_t j0 = 0; j0 < dg.size(); j0 += 65535) {
                    const uint32_t ny = (uint32_t)std::min<size_t>(65535, dg.size() - j0);
                    digest_kernel<<<dim3(chunks, ny), 256, 0, s>>>(
                        reinterpret_cast<const int32_t *>(slab),
                        reinterpret_cast<const DigestSeg *>(tab + dig_at) + j0, d_digest);
                }
            }
            batch_cap = cfg->max_batch;
            if (cudaEventCreateWithFlags(&L.done, cudaEventDisableTiming) != cudaSuccess) {
                err = RTCDF_ERR_CUDA;
                break;
            }
            if (cudaEventRecord(L.done, s) != cudaSuccess) {
                cudaEventDestroy(L.done);
                err = RTCDF_ERR_CUDA;
                break;
            }
            for (int64_t i : L.reqs) results[i].launch_s = launch_t, results[i].batch_id = (int32_t)(launches_batched + launches_single);
            stream_busy[k] = true;
            if (L.large) large_inflight++;
            inflight.push_back(std::move(L));
            if ((int)inflight.size() > max_inflight) max_inflight = (int)inflight.size();
            progressed = true;
        }
        // 3. Retire completed launches, release their memory.
        for (size_t j = 0; j < inflight.size();) {
            if (cudaEventQuery(inflight[j].done) == cudaSuccess) {
                const double t = secs(t0);
                Launch &L = inflight[j];
                for (int64_t i : L.reqs) {
                    results[i].done_s = t;
                    results[i].status = 0;
                    // The result is complete: copy it out if the caller asked.
                    if (cfg->outputs && cfg->outputs[i] && reqs[i].n &&
                        cudaMemcpy(cfg->outputs[i], slab + slot_off[i] + 4 * reqs[i].n, 4 * reqs[i].n,
                                   cudaMemcpyDeviceToHost) != cudaSuccess) {
                        results[i].status = RTCDF_ERR_CUDA;
                        if (!err) err = RTCDF_ERR_CUDA;
                    }
                    alloc.release(slot_off[i], slot_bytes[i]);
                    if (req_ev[i]) ev_pool.push_back(req_ev[i]);  // complete: the launch waited for it
                    req_ev[i] = nullptr;
                    done++;
                }
                if (L.ws_bytes) alloc.release(L.ws_off, L.ws_bytes);
                if (L.large) large_inflight--;
                stream_busy[L.stream] = false;
                cudaEventDestroy(L.done);
                inflight.erase(inflight.begin() + j);
                progressed = true;
            } else {
                j++;
            }
        }
        if (!progressed) std::this_thread::yield();
    }
    check(cudaDeviceSynchronize(), RTCDF_ERR_CUDA);
    const double makespan = secs(t0);
    if (want_digest && !err && count > 0) {
        std::vector<uint64_t> h((size_t)count);
        check(cudaMemcpy(h.data(), d_digest, sizeof(uint64_t) * (size_t)count, cudaMemcpyDeviceToHost),
              RTCDF_ERR_CUDA);
        if (!err)
            for (int64_t i = 0; i < count; i++) results[i].digest = h[i];
    }
    uint64_t keys = 0;
    for (int64_t i = 0; i < count; i++) keys += reqs[i].n;
    if (stats) {
        memset(stats, 0, sizeof(*stats));
        stats->makespan_s = makespan;
        stats->total_keys = keys;
        stats->launches_batched = launches_batched;
        stats->launches_single = launches_single;
        stats->batched_requests = batched_requests;
        stats->max_inflight = max_inflight;
        stats->peak_bytes = alloc.peak();
    }
    if (err) return err;  // `res` releases everything the call created
    return cudaGetLastError() == cudaSuccess ? RTCDF_OK : RTCDF_ERR_CUDA;
} catch (...) {  // an allocation failed (std::bad_alloc and the like)
    return RTCDF_ERR_NO_MEMORY;
}

rtcdf_status rtcdf_serve_sequential(const rtcdf_server_config *cfg, const rtcdf_request *reqs,
                                    int64_t count, rtcdf_result *results, rtcdf_serve_stats *stats) try {
    if (!cfg || (count > 0 && (!reqs || !results)) || count < 0 || !cfg->fill)
        return RTCDF_ERR_INVALID_ARG;
    uint64_t max_n = 1;
    int64_t maxR = 1;
    for (int64_t i = 0; i < count; i++) {
        const int64_t R = reqs[i].maxVal - reqs[i].minVal;
        if (R <= 0 || R > RTCDF_MAX_R || reqs[i].minVal < INT32_MIN ||
            reqs[i].maxVal > ((int64_t)1 << 31) || reqs[i].n >= (1ull << 32))
            return RTCDF_ERR_RANGE;
        max_n = std::max<uint64_t>(max_n, reqs[i].n);
        maxR = std::max(maxR, R);
    }
    size_t ws_bytes = 0;
    rtcdf_workspace_size(maxR, &ws_bytes);
    // Released on every way out, after the device has finished with them.
    struct SeqResources {
        char *buf = nullptr;
        uint64_t *d_digest = nullptr;
        DigestSeg *d_seg = nullptr;
        cudaStream_t s = nullptr;
        ~SeqResources() {
            cudaDeviceSynchronize();
            if (s) cudaStreamDestroy(s);
            cudaFree(d_seg);
            cudaFree(d_digest);
            cudaFree(buf);
        }
    } res;
    char *&buf = res.buf;
    if (cudaMalloc(&buf, max_n * 8 + ws_bytes + 512) != cudaSuccess) return RTCDF_ERR_NO_MEMORY;
    char *ws = buf + (max_n * 8 + 255) / 256 * 256;
    rtcdf_status err = RTCDF_OK;
    auto check = [&](cudaError_t e, rtcdf_status code) {
        if (e != cudaSuccess && !err) err = code;
    };
    check(cudaMemset(ws, 0, ws_bytes), RTCDF_ERR_CUDA);
    uint64_t *&d_digest = res.d_digest;
    DigestSeg *&d_seg = res.d_seg;
    if (cfg->digests) {
        const size_t db = sizeof(uint64_t) * (size_t)std::max<int64_t>(1, count);
        check(cudaMalloc(&d_digest, db), RTCDF_ERR_NO_MEMORY);
        if (d_digest) check(cudaMemset(d_digest, 0, db), RTCDF_ERR_CUDA);
        check(cudaMalloc(&d_seg, sizeof(DigestSeg)), RTCDF_ERR_NO_MEMORY);
    }
    cudaStream_t &s = res.s;
    check(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking), RTCDF_ERR_CUDA);
    check(cudaDeviceSynchronize(), RTCDF_ERR_CUDA);
    for (int64_t i = 0; i < count; i++) {
        results[i] = rtcdf_result{};
        results[i].status = -1;
    }
    const Clock::time_point t0 = Clock::now();
    for (int64_t i = 0; i < count && !err; i++) {
        while (secs(t0) < reqs[i].arrival_s) std::this_thread::yield();
        results[i] = rtcdf_result{};
        results[i].admit_s = secs(t0);
        int32_t *in = reinterpret_cast<int32_t *>(buf);
        int32_t *out = in + reqs[i].n;
        if (reqs[i].n) {
            if (cfg->fill(in, reqs[i].n, 0, reqs[i].minVal, reqs[i].maxVal - reqs[i].minVal, reqs[i].dist,
                          reqs[i].seed, (rtcdf_stream_t)s) != 0) { err = RTCDF_ERR_CUDA; break; }
            results[i].launch_s = secs(t0);
            err = rtcdf_sort_ws(in, out, reqs[i].n, reqs[i].minVal, reqs[i].maxVal, ws, ws_bytes,
                                (rtcdf_stream_t)s);
            if (cfg->digests && !err) {
                DigestSeg d{(uint64_t)reqs[i].n, reqs[i].n, (uint64_t)i};
                check(cudaMemcpyAsync(d_seg, &d, sizeof(d), cudaMemcpyHostToDevice, s), RTCDF_ERR_CUDA);
                const uint32_t chunks = (uint32_t)std::min<uint64_t>(256, (reqs[i].n + 8191) / 8192);
                digest_kernel<<<dim3(chunks, 1), 256, 0, s>>>(reinterpret_cast<const int32_t *>(buf), d_seg, d_digest);
            }
        }
        check(cudaStreamSynchronize(s), RTCDF_ERR_CUDA);
        results[i].done_s = secs(t0);
        if (!err && cfg->outputs && cfg->outputs[i] && reqs[i].n)
            check(cudaMemcpy(cfg->outputs[i], buf + 4 * reqs[i].n, 4 * reqs[i].n, cudaMemcpyDeviceToHost),
                  RTCDF_ERR_CUDA);
        results[i].status = err ? (int32_t)err : 0;
        results[i].batch_id = (int32_t)i;
    }
    const double makespan = secs(t0);
    if (cfg->digests && !err && count > 0) {
        std::vector<uint64_t> h((size_t)count);
        check(cudaMemcpy(h.data(), d_digest, sizeof(uint64_t) * (size_t)count, cudaMemcpyDeviceToHost),
              RTCDF_ERR_CUDA);
        if (!err)
            for (int64_t i = 0; i < count; i++) results[i].digest = h[i];
    }
    uint64_t keys = 0;
    for (int64_t i = 0; i < count; i++) keys += reqs[i].n;
    if (stats) {
        memset(stats, 0, sizeof(*stats));
        stats->makespan_s = makespan;
        stats->total_keys = keys;
        stats->launches_single = (uint64_t)count;
        stats->max_inflight = 1;
        stats->peak_bytes = max_n * 8 + ws_bytes;
    }
    return err;  // `res` releases the buffers and the stream
} catch (...) {  // an allocation failed (std::bad_alloc and the like)
    return RTCDF_ERR_NO_MEMORY;
}

}  // extern "C"
