// Host-side check of the segmented-sort planner (rtcdf::build_host_plan):
// for random segment shapes and several work-item sizes, the work list splits
// into the three launches with the right kinds, every segment's scan chunks
// come in ascending order (a chunk's lookback only reaches earlier chunks of
// its segment, handed out before it), the items of every segment cover its
// keys and positions exactly once, and the per-segment workspace regions are
// disjoint; the output launch issues its items by non-increasing estimated
// cost (length x (1/4 + min(R, n) / n): vectors plus the runs crossed when
// every value is present).  The same shapes go through the host emulation of
// the device planner (devplan_host: the rules the planner kernel applies): its
// lists sit at their fixed bases and hold the right kinds in the right order,
// each of the three histogram lists only items of its size class, the
// positions past a list's length stay unused, every segment's scan chunks
// ascend, the items cover every segment's keys and positions exactly once, the
// list lengths stay within the bounds the workspace was sized for, the first
// launch's tickets map one-to-one onto the histogram lists (one after another)
// and the in-CTA segments (evenly spread), and every segment's regions lie
// inside its own slot.
// Usage: planner_check <seed> <segments>; prints "OK" or the first violation.
// planner_check --emit <file> reads bounds and metadata ("S N maxR", then S+1
// offsets, S minVal, S maxVal) and prints the layout, the lists' bounds and
// lengths, the descriptors and the items array (every position, unused ones
// zero) of the emulated device plan (compared with the GPU planner's
// workspace by a GPU test).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <random>
#include <string>
#include <vector>

#include "batched.h"

using namespace rtcdf;

static int fail(const char *what, long a, long b) {
    std::printf("FAIL %s (%ld, %ld)\n", what, a, b);
    return 1;
}

static int check(const std::vector<SegSpec> &spec, const BatchTuning &tun) {
    HostPlan P;
    if (build_host_plan(spec.data(), (uint32_t)spec.size(), &P, tun)) return fail("plan rejected", 0, 0);
    const uint32_t S = (uint32_t)spec.size();
    if ((size_t)P.n_first + P.n_scan + P.n_small2 + P.n_fill != P.items.size()) return fail("launch sizes", 0, 0);
    std::vector<uint32_t> small_seen(S, 0), next_chunk(S, 0);
    double prev_cost = HUGE_VAL;
    std::vector<std::vector<std::pair<uint64_t, uint64_t>>> hist_rng(S), fill_rng(S);
    for (size_t q = 0; q < P.items.size(); q++) {
        const BatchItem &it = P.items[q];
        if (it.seg >= S) return fail("segment index", (long)q, it.seg);
        const BatchSeg &g = P.segs[it.seg];
        // 0: first launch, 1: scan chunks, 3: in-CTA segments of the scan launch, 2: output launch
        const size_t e1 = (size_t)P.n_first + P.n_scan, e3 = e1 + P.n_small2;
        const int launch = q < P.n_first ? 0 : (q < e1 ? 1 : (q < e3 ? 3 : 2));
        switch (it.kind) {
            case kItemHist:
                if (launch != 0) return fail("hist outside the first launch", (long)q, launch);
                if (it.tile >= g.m) return fail("tile index", (long)q, it.tile);
                hist_rng[it.seg].push_back({it.a * 1024 + it.tile, it.b});
                break;
            case kItemSmall:
                if (launch != 0 && launch != 3) return fail("small in a wrong launch", (long)q, launch);
                if ((launch == 3) != (g.R <= tun.small_scan_max_R)) return fail("small launch by range", (long)q, g.R);
                small_seen[it.seg]++;
                break;
            case kItemScan:
                if (launch != 1) return fail("scan outside the scan launch", (long)q, launch);
                if (it.a != next_chunk[it.seg]) return fail("scan chunk order", (long)q, (long)it.a);
                next_chunk[it.seg]++;
                break;
            case kItemFill:
                if (launch != 2) return fail("fill outside the output launch", (long)q, launch);
                fill_rng[it.seg].push_back({it.a, it.b});
                if (it.aux >= g.fill_items || it.a != (uint64_t)it.aux * g.fill_chunk)
                    return fail("fill index", (long)q, it.aux);
                {
                    const double cost = (double)(it.b - it.a) * (0.25 + (double)std::min(g.R, g.n) / (double)g.n);
                    if (cost > prev_cost) return fail("output item order", (long)q, (long)cost);
                    prev_cost = cost;
                }
                break;
            default: return fail("item kind", (long)q, it.kind);
        }
    }
    size_t ws_prev_end = P.segctl_off + S * sizeof(BatchSegCtl) / 4;
    if (P.segctl_off < P.ctl_off + sizeof(BatchCtl) / 4) return fail("control blocks overlap", 0, 0);
    for (uint32_t s = 0; s < S; s++) {
        const BatchSeg &g = P.segs[s];
        if (spec[s].n == 0) {
            if (small_seen[s] || next_chunk[s] || !hist_rng[s].empty()) return fail("empty segment has items", s, 0);
            continue;
        }
        const bool large = g.m > 0;
        if (!large) {
            if (small_seen[s] != 1) return fail("small segment not exactly once", s, small_seen[s]);
            if (g.n > tun.small_max_n || g.R > kBatchSmallMaxR) return fail("small limits", s, g.R);
            continue;
        }
        if (small_seen[s]) return fail("large segment sorted in one CTA", s, 0);
        if (next_chunk[s] != g.scan_chunks || (uint64_t)g.scan_chunks * kBatchScanChunk < g.R)
            return fail("scan chunks", s, next_chunk[s]);
        // histogram items: for each tile, key ranges tile [0, n) without overlap
        std::vector<std::vector<std::pair<uint64_t, uint64_t>>> per_tile(g.m);
        for (auto &r : hist_rng[s]) per_tile[r.first % 1024].push_back({r.first / 1024, r.second});
        uint32_t nh = 0;
        for (uint32_t t = 0; t < g.m; t++) {
            auto &v = per_tile[t];
            std::sort(v.begin(), v.end());
            uint64_t at = 0;
            for (auto &r : v) {
                if (r.first != at || r.second <= r.first) return fail("hist key ranges", s, t);
                at = r.second;
            }
            if (at != g.n) return fail("hist keys not covered", s, t);
            if (g.single_hist != (v.size() == 1 ? 1u : 0u)) return fail("single_hist flag", s, t);
            nh += (uint32_t)v.size();
        }
        if (nh != g.hist_items) return fail("hist item count", s, nh);
        auto &f = fill_rng[s];
        std::sort(f.begin(), f.end());
        uint64_t at = 0;
        for (auto &r : f) {
            if (r.first != at || r.second <= r.first) return fail("fill positions", s, (long)r.first);
            at = r.second;
        }
        if (at != g.n || f.size() != g.fill_items) return fail("fill coverage", s, (long)at);
        if ((uint64_t)g.T * g.m < g.R || g.T > kBatchTileMax) return fail("tiles", s, g.T);
        // workspace regions in order, disjoint, inside ws_words; the lookback
        // state is 8-byte aligned
        const size_t regs[5][2] = {{g.hist_off, (size_t)g.scan_chunks * kBatchScanChunk},
                                   {g.run_end_off, g.R}, {g.run_val_off, g.R},
                                   {g.start_run_off, g.fill_items}, {g.state_off, 2 * (size_t)g.scan_chunks}};
        for (auto &r : regs) {
            if (r[0] < ws_prev_end) return fail("workspace overlap", s, (long)r[0]);
            ws_prev_end = r[0] + r[1];
        }
        if (g.state_off % 2) return fail("state alignment", s, (long)g.state_off);
        if (g.hist_off % 4) return fail("histogram alignment", s, (long)g.hist_off);
        if (ws_prev_end > P.ws_words) return fail("workspace size", s, (long)ws_prev_end);
    }
    return 0;
}

// Invariants of the device plan (host emulation) for the shapes of `spec`.
static int check_dev(const std::vector<SegSpec> &spec, const BatchTuning &tun, uint32_t max_R) {
    const uint32_t S = (uint32_t)spec.size();
    std::vector<int64_t> offs(S + 1), mn(S), mx(S);
    uint64_t N = 0;
    for (uint32_t s = 0; s < S; s++) {
        offs[s] = (int64_t)spec[s].in_off;
        mn[s] = spec[s].minVal;
        mx[s] = spec[s].maxVal;
        N = spec[s].in_off + spec[s].n;
    }
    offs[S] = (int64_t)N;
    const DevBounds b{S, max_R, N + 12345};
    DevLayout L;
    if (devplan_layout(b, tun, &L)) return fail("dev layout", 0, 0);
    std::vector<BatchSeg> segs;
    std::vector<DevPfx> pfx;
    DevPlanHdr hdr;
    std::vector<BatchItem> items;
    const int rc = devplan_host(offs.data(), mn.data(), mx.data(), b, tun, L, &segs, &pfx, &hdr, &items);
    bool any_bad = false;
    for (uint32_t s = 0; s < S; s++) any_bad |= mx[s] - mn[s] > (int64_t)max_R;
    if (any_bad) return rc ? 0 : fail("dev plan accepted a range above max_R", 0, 0);
    if (rc) return fail("dev plan rejected", rc, 0);
    if (hdr.n_first != hdr.n_hist + hdr.n_small1) return fail("dev first list", hdr.n_first, hdr.n_hist);
    if (hdr.n_hist != (uint64_t)hdr.n_hist_class[0] + hdr.n_hist_class[1] + hdr.n_hist_class[2])
        return fail("dev histogram lists", hdr.n_hist, hdr.n_hist_class[0]);
    if (items.size() != L.item_bound) return fail("dev items array", (long)items.size(), (long)L.item_bound);
    const DevListBounds &lb = L.lb;
    if (lb.first != kHistClasses * lb.hist + lb.small2) return fail("dev first bound", 0, 0);
    if (hdr.n_hist > lb.hist || hdr.n_small1 > S || hdr.n_scan > lb.scan || hdr.n_small2 > lb.small2 ||
        hdr.n_fill > lb.fill)
        return fail("dev bounds", hdr.n_first, hdr.n_scan);
    if (hdr.n_scan != hdr.n_scan_class[0] + hdr.n_scan_class[1] || hdr.n_fill != hdr.n_fill_class[0] + hdr.n_fill_class[1])
        return fail("dev class lengths", hdr.n_scan, hdr.n_fill);
    // Each list sits at its fixed base (the bounds of the lists before it);
    // the positions past a list's length stay unused.
    const uint64_t fb = lb.first + 2 * lb.scan + lb.small2;
    const uint64_t list_base[kNumLists] = {0, lb.hist, 2 * lb.hist, 3 * lb.hist, lb.first, lb.first + lb.scan,
                                           lb.first + 2 * lb.scan, fb, fb + lb.fill};
    const uint64_t list_bound[kNumLists] = {lb.hist, lb.hist, lb.hist, S, lb.scan, lb.scan, lb.small2, lb.fill, lb.fill};
    const uint32_t list_len[kNumLists] = {hdr.n_hist_class[0], hdr.n_hist_class[1], hdr.n_hist_class[2],
                                          hdr.n_small1, hdr.n_scan_class[0], hdr.n_scan_class[1], hdr.n_small2,
                                          hdr.n_fill_class[0], hdr.n_fill_class[1]};
    const uint32_t list_kind[kNumLists] = {kItemHist, kItemHist, kItemHist, kItemSmall, kItemScan, kItemScan,
                                           kItemSmall, kItemFill, kItemFill};
    if (fb + 2 * lb.fill != L.item_bound) return fail("dev item bound", 0, 0);
    for (uint32_t f = 0; f < kNumLists; f++)
        if (devplan_pos(lb, f, 0) != list_base[f]) return fail("dev list base", f, (long)devplan_pos(lb, f, 0));
    std::vector<uint32_t> small_seen(S, 0), next_chunk(S, 0);
    std::vector<std::vector<uint32_t>> fill_aux(S);
    std::vector<std::vector<std::pair<uint64_t, uint64_t>>> hist_rng(S);
    for (uint32_t f = 0; f < kNumLists; f++) {
        for (uint64_t k = list_len[f]; k < list_bound[f]; k++) {
            const BatchItem &u = items[list_base[f] + k];
            if (u.kind || u.seg || u.a || u.b || u.tile || u.aux) return fail("dev unused position", f, (long)k);
        }
        std::vector<int64_t> last_aux(S, -1);
        for (uint64_t k = 0; k < list_len[f]; k++) {
            const size_t q = list_base[f] + k;
            const BatchItem &it = items[q];
            if (it.seg >= S) return fail("dev segment index", (long)q, it.seg);
            const BatchSeg &g = segs[it.seg];
            if (it.kind != list_kind[f]) return fail("dev item kind", (long)q, it.kind);
            switch (it.kind) {
                case kItemHist:
                    if (it.tile >= g.m) return fail("dev tile index", (long)q, it.tile);
                    // each histogram list holds the items of its size class
                    if (devplan_hist_class(it.b - it.a, tun.hist_chunk) != f) return fail("dev histogram class", (long)q, f);
                    hist_rng[it.seg].push_back({it.a * 1024 + it.tile, it.b});
                    break;
                case kItemSmall:
                    if ((f == kListSmall2) != (g.R <= tun.small_scan_max_R))
                        return fail("dev small list by range", (long)q, g.R);
                    small_seen[it.seg]++;
                    break;
                case kItemScan:
                    // long chains in the first list; a segment's chunks ascend
                    if ((f == kListScan0) != (g.scan_chunks >= kLongChain)) return fail("dev scan class", (long)q, f);
                    if (it.a != next_chunk[it.seg]) return fail("dev scan chunk order", (long)q, (long)it.a);
                    next_chunk[it.seg]++;
                    break;
                case kItemFill:
                    if (it.aux >= g.fill_items || it.a != (uint64_t)it.aux * g.fill_chunk ||
                        it.b != std::min<uint64_t>(g.n, (uint64_t)(it.aux + 1) * g.fill_chunk))
                        return fail("dev fill item", (long)q, it.aux);
                    // each output list holds the items of its cost class; a
                    // segment's items ascend within a list
                    if (kListFill0 + devplan_fill_class(it.b - it.a, g) != f) return fail("dev fill class", (long)q, f);
                    if ((int64_t)it.aux <= last_aux[it.seg]) return fail("dev fill order", (long)q, it.aux);
                    last_aux[it.seg] = it.aux;
                    fill_aux[it.seg].push_back(it.aux);
                    break;
            }
        }
    }
    // The first launch's tickets: a bijection onto the three histogram lists
    // (taken one after another, each in list order) and the in-CTA segments
    // (in list order, evenly spread: between consecutive ones at most
    // ceil(T / ns) tickets).
    {
        const uint64_t nh = hdr.n_hist, ns = hdr.n_small1, T = nh + ns;
        uint64_t next_h = 0, next_s = 0, last_s = 0;
        const uint64_t hb = lb.hist;
        auto hist_pos = [&](uint64_t h) {  // the h-th histogram item over the three lists
            uint32_t c = 0;
            while (c + 1 < kHistClasses && h >= hdr.n_hist_class[c]) h -= hdr.n_hist_class[c++];
            return c * hb + h;
        };
        for (uint64_t k = 0; k < T; k++) {
            const uint64_t q = devplan_first_pos(k, hdr.n_hist_class, ns, lb);
            if (q < kHistClasses * hb) {
                if (q != hist_pos(next_h++)) return fail("dev first ticket (histogram)", (long)k, (long)q);
            } else {
                if (q != kHistClasses * hb + next_s) return fail("dev first ticket (in-CTA)", (long)k, (long)q);
                if (next_s > 0 && (k - last_s) * ns > T + ns) return fail("dev first ticket spread", (long)k, 0);
                last_s = k;
                next_s++;
            }
        }
        if (next_h != nh || next_s != ns) return fail("dev first tickets", (long)next_h, (long)next_s);
    }
    for (uint32_t s = 0; s < S; s++) {
        const BatchSeg &g = segs[s];
        if (g.n != spec[s].n || g.off != spec[s].in_off || (int64_t)g.minVal != spec[s].minVal)
            return fail("dev descriptor", s, g.n);
        if (spec[s].n == 0) {
            if (small_seen[s] || next_chunk[s] || !fill_aux[s].empty() || !hist_rng[s].empty())
                return fail("dev empty segment has items", s, 0);
            continue;
        }
        if (g.m == 0) {
            if (small_seen[s] != 1) return fail("dev small segment not exactly once", s, small_seen[s]);
            continue;
        }
        if (small_seen[s]) return fail("dev large segment in one CTA", s, 0);
        if (next_chunk[s] != g.scan_chunks) return fail("dev scan chunks", s, next_chunk[s]);
        {
            // every output item of the segment exactly once, over both lists
            std::vector<uint32_t> &v = fill_aux[s];
            std::sort(v.begin(), v.end());
            for (uint32_t i = 0; i < v.size(); i++)
                if (v[i] != i) return fail("dev fill items", s, v[i]);
            if (v.size() != g.fill_items || (uint64_t)g.fill_items * g.fill_chunk < g.n)
                return fail("dev fill coverage", s, (long)v.size());
        }
        std::vector<std::vector<std::pair<uint64_t, uint64_t>>> per_tile(g.m);
        for (auto &r : hist_rng[s]) per_tile[r.first % 1024].push_back({r.first / 1024, r.second});
        for (uint32_t t = 0; t < g.m; t++) {
            auto &v = per_tile[t];
            std::sort(v.begin(), v.end());
            uint64_t at = 0;
            for (auto &r : v) {
                if (r.first != at || r.second <= r.first) return fail("dev hist key ranges", s, t);
                at = r.second;
            }
            if (at != g.n) return fail("dev hist keys not covered", s, t);
        }
        // regions inside the segment's own slot, the start runs inside the pool
        const size_t slot = L.slots + (size_t)s * L.slot_words;
        if (g.hist_off != slot || g.state_off != slot + L.slot_state) return fail("dev slot", s, (long)g.hist_off);
        if (g.hist_off + (size_t)g.scan_chunks * kBatchScanChunk > g.state_off) return fail("dev hist region", s, 0);
        if (g.state_off + 2 * (size_t)g.scan_chunks > g.run_end_off) return fail("dev state region", s, 0);
        if (g.run_end_off + g.R > g.run_val_off || g.run_val_off + g.R > slot + L.slot_words)
            return fail("dev run tables", s, 0);
        if (g.state_off % 2 || g.hist_off % 4) return fail("dev alignment", s, 0);
        if (g.start_run_off < L.start || g.start_run_off + g.fill_items > L.start + lb.fill)
            return fail("dev start runs", s, (long)g.start_run_off);
        if (slot + L.slot_words > L.total_words) return fail("dev workspace size", s, 0);
    }
    {
        // the segments' start-run slots do not overlap
        std::vector<std::pair<size_t, size_t>> rs;
        for (uint32_t s = 0; s < S; s++)
            if (segs[s].m > 0) rs.push_back({segs[s].start_run_off, segs[s].start_run_off + segs[s].fill_items});
        std::sort(rs.begin(), rs.end());
        for (size_t i = 1; i < rs.size(); i++)
            if (rs[i].first < rs[i - 1].second) return fail("dev start runs overlap", (long)i, (long)rs[i].first);
    }
    return 0;
}

// --emit: the emulated device plan for the bounds and metadata in a file.
static int emit(const char *path) {
    FILE *f = std::fopen(path, "r");
    if (!f) return fail("cannot open", 0, 0);
    unsigned long long S = 0, N = 0, maxR = 0;
    if (std::fscanf(f, "%llu %llu %llu", &S, &N, &maxR) != 3) return fail("header", 0, 0);
    std::vector<int64_t> offs(S + 1), mn(S), mx(S);
    for (auto *v : {&offs, &mn, &mx})
        for (auto &x : *v)
            if (std::fscanf(f, "%lld", (long long *)&x) != 1) return fail("metadata", 0, 0);
    std::fclose(f);
    const DevBounds b{(uint32_t)S, (uint32_t)maxR, N};
    const BatchTuning tun;
    DevLayout L;
    if (devplan_layout(b, tun, &L)) return fail("layout", 0, 0);
    std::vector<BatchSeg> segs;
    std::vector<DevPfx> pfx;
    DevPlanHdr hdr;
    std::vector<BatchItem> items;
    const int rc = devplan_host(offs.data(), mn.data(), mx.data(), b, tun, L, &segs, &pfx, &hdr, &items);
    std::printf("layout %zu %zu %zu %zu %zu %zu\n", L.ctl, L.hdr, L.segs, L.look, L.items, L.total_words);
    std::printf("bounds %llu %llu %llu %llu %llu\n", (unsigned long long)L.lb.hist,
                (unsigned long long)L.lb.first, (unsigned long long)L.lb.scan,
                (unsigned long long)L.lb.small2, (unsigned long long)L.lb.fill);
    std::printf("rc %d\n", rc);
    std::printf("hdr %u %u %u %u %u %u %u %u %u %u %u %u %u\n", hdr.n_first, hdr.n_scan, hdr.n_small2, hdr.n_fill,
                hdr.n_hist, hdr.n_small1, hdr.n_hist_class[0], hdr.n_hist_class[1], hdr.n_hist_class[2],
                hdr.n_scan_class[0], hdr.n_scan_class[1], hdr.n_fill_class[0], hdr.n_fill_class[1]);
    for (const BatchSeg &g : segs)
        std::printf("seg %llu %u %u %d %u %u %u %u %u %u %u %llu %llu %llu %llu %llu\n",
                    (unsigned long long)g.off, g.n, g.R, g.minVal, g.T, g.m, g.hist_items, g.fill_items,
                    g.fill_chunk, g.scan_chunks, g.single_hist, (unsigned long long)g.hist_off,
                    (unsigned long long)g.run_end_off, (unsigned long long)g.run_val_off,
                    (unsigned long long)g.start_run_off, (unsigned long long)g.state_off);
    for (const BatchItem &it : items)
        std::printf("item %u %u %llu %llu %u %u\n", it.kind, it.seg, (unsigned long long)it.a,
                    (unsigned long long)it.b, it.tile, it.aux);
    return 0;
}

int main(int argc, char **argv) {
    if (argc > 2 && std::string(argv[1]) == "--emit") return emit(argv[2]);
    const unsigned seed = argc > 1 ? (unsigned)atoi(argv[1]) : 1;
    const int S = argc > 2 ? atoi(argv[2]) : 500;
    std::mt19937_64 rng(seed);
    std::vector<SegSpec> spec(S);
    uint64_t off = 0;
    for (int s = 0; s < S; s++) {
        const double u = std::uniform_real_distribution<double>(0, 1)(rng);
        const uint64_t n = (rng() % 7 == 0) ? 0 : (uint64_t)std::exp(u * std::log(3e6));
        const int64_t R = 1 + (int64_t)(rng() % ((rng() % 3 == 0) ? (1u << 20) : 60000u));
        const int64_t mn = (int64_t)(rng() % 2000000) - 1000000;
        spec[s] = SegSpec{off, off, n, mn, mn + R};
        off += n;
    }
    BatchTuning tunings[7];
    tunings[1].hist_chunk = 4096; tunings[1].fill_chunk = 4096; tunings[1].small_max_n = 100;
    tunings[2].hist_chunk = 1ull << 22; tunings[2].fill_chunk = 1u << 20; tunings[2].small_max_n = 1;
    tunings[3].hist_chunk = 5000; tunings[3].fill_chunk = 6000;
    tunings[4].small_scan_max_R = 1;
    tunings[5].small_scan_max_R = kSmallInScanCapR;
    tunings[6].small_by_time = 0;
    for (auto &t : tunings)
        if (check(spec, t)) return 1;
    // The device planner's rules, with bounds that hold and with one that
    // some segment breaks.
    for (auto &t : tunings)
        for (uint32_t max_R : {1u << 20, 60000u})
            if (check_dev(spec, t, max_R)) return 1;
    std::printf("OK\n");
    return 0;
}
