// Launch-parameter tuning: the per-process table that rtcdf_sort consults, and
// rtcdf_autotune, which measures candidates and ranks them by the geometric
// mean of their normalised times (Section 4.1's selection of the tile width,
// applied to every launch parameter).
#include <algorithm>
#include <cmath>
#include <mutex>
#include <vector>

#include "../../include/rtcdf.h"
#include "rtcdf_internal.h"

namespace {

// The table compiled into the library (written by the package's tune module
// from measurements on GB300).
const rtcdf_tune_entry kBuiltin[] = {
#include "tune_table.inc"
    {-1, -1, {0, 0, 0, 0, 0, 0, {0, 0}}}  // terminator, never matched
};

std::mutex g_tune_mu;
std::vector<rtcdf_tune_entry> g_table;
bool g_loaded = false;

void load_builtin_locked() {
    g_table.clear();
    for (const rtcdf_tune_entry &e : kBuiltin)
        if (e.log2_R >= 0) g_table.push_back(e);
    g_loaded = true;
}

int32_t log2_ceil(uint32_t R) {
    int32_t l = 0;
    while (l < 31 && (1u << l) < R) l++;
    return l;
}

}  // namespace

namespace rtcdf {

bool tune_lookup(uint64_t n, uint32_t R, rtcdf_params *out) {
    const int32_t lr = log2_ceil(R), nc = rtcdf_tune_n_class(n);
    std::lock_guard<std::mutex> lk(g_tune_mu);
    if (!g_loaded) {
        try {
            load_builtin_locked();
        } catch (...) {  // no memory for the table: the built-in rules apply
            g_table.clear();
            return false;
        }
    }
    // The last entry with the key wins.
    for (auto it = g_table.rbegin(); it != g_table.rend(); ++it) {
        if (it->log2_R == lr && it->n_class == nc) {
            *out = it->params;
            return true;
        }
    }
    return false;
}

}  // namespace rtcdf

extern "C" {

int32_t rtcdf_tune_n_class(uint64_t n) {
    if (n < (1ull << 20)) return RTCDF_TUNE_N_SMALL;
    if (n < (1ull << 26)) return RTCDF_TUNE_N_MEDIUM;
    return RTCDF_TUNE_N_LARGE;
}

rtcdf_status rtcdf_tune_set(const rtcdf_tune_entry *entries, int32_t count) try {
    if (count < 0 || (count > 0 && !entries)) return RTCDF_ERR_INVALID_ARG;
    for (int32_t i = 0; i < count; i++) {
        const rtcdf_tune_entry &e = entries[i];
        if (e.log2_R < 0 || e.log2_R > 24 || e.n_class < 0 || e.n_class > 2) return RTCDF_ERR_INVALID_ARG;
        const rtcdf_params &p = e.params;
        if (p.tile_width < 0 || p.hist_ctas_per_tile < 0 || p.fill_ctas < 0) return RTCDF_ERR_INVALID_ARG;
        for (int32_t th : {p.hist_threads, p.fill_threads})
            if (th != 0 && th != 256 && th != 512 && th != 1024) return RTCDF_ERR_INVALID_ARG;
    }
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_table.assign(entries, entries + count);
    g_loaded = true;
    return RTCDF_OK;
} catch (...) {  // an allocation failed (std::bad_alloc and the like)
    return RTCDF_ERR_NO_MEMORY;
}

rtcdf_status rtcdf_tune_reset(void) try {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    load_builtin_locked();
    return RTCDF_OK;
} catch (...) {  // an allocation failed (std::bad_alloc and the like)
    return RTCDF_ERR_NO_MEMORY;
}

rtcdf_status rtcdf_tune_get(rtcdf_tune_entry *entries, int32_t capacity, int32_t *count) {
    if (!count || capacity < 0 || (capacity > 0 && !entries)) return RTCDF_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    if (!g_loaded) load_builtin_locked();
    *count = (int32_t)g_table.size();
    for (int32_t i = 0; i < capacity && i < (int32_t)g_table.size(); i++) entries[i] = g_table[i];
    return RTCDF_OK;
}

rtcdf_status rtcdf_autotune(const rtcdf_tune_case *cases, int32_t num_cases,
                            const rtcdf_params *candidates, int32_t num_candidates, int32_t reps,
                            void *workspace, size_t ws_bytes, float *times_ms, double *geomean,
                            int32_t *best, rtcdf_stream_t stream) try {
    if (!cases || num_cases <= 0 || !candidates || num_candidates <= 0 || reps <= 0 || !workspace ||
        !times_ms || !geomean || !best)
        return RTCDF_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<cudaEvent_t> ev((size_t)reps + 1, nullptr);
    rtcdf_status result = RTCDF_OK;
    for (cudaEvent_t &e : ev)
        if (cudaEventCreate(&e) != cudaSuccess) {
            e = nullptr;
            result = RTCDF_ERR_CUDA;
            break;
        }
    std::vector<float> t((size_t)reps);
    for (int32_t c = 0; c < num_cases && result == RTCDF_OK; c++) {
        const rtcdf_tune_case &tc = cases[c];
        for (int32_t k = 0; k < num_candidates; k++) {
            float &cell = times_ms[(size_t)c * num_candidates + k];
            cell = -1.0f;
            // One untimed sort; a candidate that cannot run here is skipped.
            rtcdf_status st = rtcdf_sort_ex(tc.in, tc.out, tc.n, tc.minVal, tc.maxVal, &candidates[k],
                                            workspace, ws_bytes, nullptr, stream);
            if (st == RTCDF_ERR_INVALID_ARG) continue;
            if (st) { result = st; break; }
            if (cudaEventRecord(ev[0], s) != cudaSuccess) { result = RTCDF_ERR_CUDA; break; }
            for (int32_t r = 0; r < reps && result == RTCDF_OK; r++) {
                st = rtcdf_sort_ex(tc.in, tc.out, tc.n, tc.minVal, tc.maxVal, &candidates[k], workspace,
                                   ws_bytes, nullptr, stream);
                if (st) result = st;
                else if (cudaEventRecord(ev[(size_t)r + 1], s) != cudaSuccess) result = RTCDF_ERR_CUDA;
            }
            if (result) break;
            if (cudaEventSynchronize(ev[(size_t)reps]) != cudaSuccess) { result = RTCDF_ERR_CUDA; break; }
            for (int32_t r = 0; r < reps && !result; r++)
                if (cudaEventElapsedTime(&t[(size_t)r], ev[(size_t)r], ev[(size_t)r + 1]) != cudaSuccess)
                    result = RTCDF_ERR_CUDA;
            if (result) break;
            std::sort(t.begin(), t.end());
            cell = t[(size_t)reps / 2];
        }
    }
    for (cudaEvent_t &e : ev)
        if (e) cudaEventDestroy(e);
    if (result) return result;
    int32_t dev_status = 0;
    rtcdf_status st = rtcdf_ws_status_get(workspace, stream, &dev_status);
    if (st) return st;
    // Normalise per condition, geometric mean per candidate.
    std::vector<double> logsum((size_t)num_candidates, 0.0);
    std::vector<bool> ok((size_t)num_candidates, true);
    for (int32_t c = 0; c < num_cases; c++) {
        double tmin = HUGE_VAL;
        for (int32_t k = 0; k < num_candidates; k++) {
            const float v = times_ms[(size_t)c * num_candidates + k];
            if (v > 0.0f) tmin = std::min(tmin, (double)v);
        }
        for (int32_t k = 0; k < num_candidates; k++) {
            const float v = times_ms[(size_t)c * num_candidates + k];
            if (!(v > 0.0f)) { ok[(size_t)k] = false; continue; }
            logsum[(size_t)k] += std::log((double)v / tmin);
        }
    }
    int32_t b = -1;
    for (int32_t k = 0; k < num_candidates; k++) {
        geomean[k] = ok[(size_t)k] ? std::exp(logsum[(size_t)k] / num_cases) : HUGE_VAL;
        if (ok[(size_t)k] && (b < 0 || geomean[k] < geomean[b])) b = k;
    }
    *best = b;
    return b < 0 ? RTCDF_ERR_INVALID_ARG : RTCDF_OK;
} catch (...) {  // an allocation failed (std::bad_alloc and the like)
    return RTCDF_ERR_NO_MEMORY;
}

}  // extern "C"
