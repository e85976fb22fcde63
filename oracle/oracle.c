/*
 * oracle.c -- plain, sequential CPU oracle for Range-Tiled CDF sort (RT-CDF).
 *
 * TEST INFRASTRUCTURE, NOT PART OF THE PRODUCT.  Only the test suite, the
 * smoke check and the benchmark's CPU-baseline / reference arm may load this
 * library.  It shares no code, header or table with the CUDA path and never
 * includes anything from it.
 *
 * Everything here is integer arithmetic, single-threaded, written for
 * readability rather than speed.  Notation follows the paper
 * ("Shared-Memory Range-Tiled CDF Sort for Small-Range Integer Keys on GPUs"):
 *   A[0..n-1]  input keys, all in [minVal, maxVal), R = maxVal - minVal
 *   B[0..n-1]  output, A in nondecreasing order
 *   c_v        number of occurrences of the normalised value v = key - minVal
 *   T, m       tile width and number of tiles m = ceil(R / T)
 *   b_t, w_t   first value and width of tile t: b_t = tT, w_t = min(T, R - b_t)
 *   H, O       per-tile histograms / local CDFs, and tile output offsets
 *
 * Parity pins for every function live in tests/test_oracle.py; nothing here is
 * "parity unpinned".
 *
 * Return codes (shared meaning with the library's status codes, defined here
 * independently): 0 ok, 1 invalid argument, 2 range size R <= 0 or too large,
 * 3 a key outside [minVal, maxVal), 5 out of host memory.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_OK 0
#define OR_ERR_INVALID_ARG 1
#define OR_ERR_RANGE 2
#define OR_ERR_KEY_OUT_OF_RANGE 3
#define OR_ERR_NO_MEMORY 5

/* Largest range the oracle accepts: 2^32 values (the whole int32 key space). */
#define OR_MAX_R (((int64_t)1) << 32)

static int range_size(int64_t minVal, int64_t maxVal, int64_t *R) {
    /* R = maxVal - minVal (Section 2.1); maxVal is exclusive. */
    if (maxVal <= minVal) return OR_ERR_RANGE;
    *R = maxVal - minVal;
    if (*R > OR_MAX_R) return OR_ERR_RANGE;
    return OR_OK;
}

/*
 * Histogram of the normalised keys: cnt[v] = c_v for v in [0, R)
 * (Section 2.1, "H[v] = c_v").  A key outside [minVal, maxVal) is an error:
 * the paper treats the range as a precondition, the oracle reports it.
 */
int oracle_histogram(const int32_t *A, uint64_t n, int64_t minVal, int64_t maxVal,
                     uint64_t *cnt) {
    int64_t R;
    int rc = range_size(minVal, maxVal, &R);
    if (rc) return rc;
    if (n > 0 && (A == NULL || cnt == NULL)) return OR_ERR_INVALID_ARG;
    memset(cnt, 0, (size_t)R * sizeof(uint64_t));
    for (uint64_t i = 0; i < n; i++) {
        int64_t x = (int64_t)A[i] - minVal;
        if (x < 0 || x >= R) return OR_ERR_KEY_OUT_OF_RANGE;
        cnt[x] += 1;
    }
    return OR_OK;
}

/*
 * Counting sort, the plain definition of the result (Section 2.1): value v,
 * occurring c_v times, occupies output positions
 *     [ sum_{u<v} c_u , sum_{u<=v} c_u ).
 * Histogram, then walk the values in increasing order writing each c_v times.
 */
int oracle_counting_sort(const int32_t *A, int32_t *B, uint64_t n, int64_t minVal,
                         int64_t maxVal) {
    int64_t R;
    int rc = range_size(minVal, maxVal, &R);
    if (rc) return rc;
    if (n == 0) return OR_OK;
    if (A == NULL || B == NULL) return OR_ERR_INVALID_ARG;
    uint64_t *cnt = (uint64_t *)malloc((size_t)R * sizeof(uint64_t));
    if (!cnt) return OR_ERR_NO_MEMORY;
    rc = oracle_histogram(A, n, minVal, maxVal, cnt);
    if (rc) { free(cnt); return rc; }
    uint64_t p = 0;
    for (int64_t v = 0; v < R; v++) {
        for (uint64_t c = 0; c < cnt[v]; c++) B[p++] = (int32_t)(minVal + v);
    }
    free(cnt);
    return OR_OK;
}

/*
 * Counting sort of Kolonias et al. as simplified in Algorithm 1: H = histogram,
 * P[0] = 0, P[1..R] = prefix sums of H, then every value v fills [P[v], P[v+1]).
 * A second formulation of the same output, used as a cross-check.
 */
int oracle_kolonias_sort(const int32_t *A, int32_t *B, uint64_t n, int64_t minVal,
                         int64_t maxVal) {
    int64_t R;
    int rc = range_size(minVal, maxVal, &R);
    if (rc) return rc;
    if (n == 0) return OR_OK;
    if (A == NULL || B == NULL) return OR_ERR_INVALID_ARG;
    uint64_t *H = (uint64_t *)malloc((size_t)R * sizeof(uint64_t));
    uint64_t *P = (uint64_t *)malloc((size_t)(R + 1) * sizeof(uint64_t));
    if (!H || !P) { free(H); free(P); return OR_ERR_NO_MEMORY; }
    rc = oracle_histogram(A, n, minVal, maxVal, H);
    if (rc) { free(H); free(P); return rc; }
    P[0] = 0;
    for (int64_t v = 0; v < R; v++) P[v + 1] = P[v] + H[v];
    for (int64_t v = 0; v < R; v++)
        for (uint64_t p = P[v]; p < P[v + 1]; p++) B[p] = (int32_t)(minVal + v);
    free(H);
    free(P);
    return OR_OK;
}

/*
 * H-P sort, Algorithm 2: H1 = histogram of A, P1 = inclusive prefix sums of H1,
 * H2[0..n] = histogram of the values of P1, B = inclusive prefix sums of
 * H2[0..n-1].  B[i] counts the values whose interval ends at or before i, which
 * is the normalised value at position i.  minVal is added back at the end.
 */
int oracle_hp_sort(const int32_t *A, int32_t *B, uint64_t n, int64_t minVal,
                   int64_t maxVal) {
    int64_t R;
    int rc = range_size(minVal, maxVal, &R);
    if (rc) return rc;
    if (n == 0) return OR_OK;
    if (A == NULL || B == NULL) return OR_ERR_INVALID_ARG;
    uint64_t *H1 = (uint64_t *)malloc((size_t)R * sizeof(uint64_t));
    uint64_t *H2 = (uint64_t *)calloc((size_t)(n + 1), sizeof(uint64_t));
    if (!H1 || !H2) { free(H1); free(H2); return OR_ERR_NO_MEMORY; }
    rc = oracle_histogram(A, n, minVal, maxVal, H1);
    if (rc) { free(H1); free(H2); return rc; }
    uint64_t P1 = 0;
    for (int64_t v = 0; v < R; v++) {
        P1 += H1[v];          /* P1[v] */
        H2[P1] += 1;          /* histogram of P1 over [0..n] */
    }
    uint64_t acc = 0;
    for (uint64_t i = 0; i < n; i++) {
        acc += H2[i];
        B[i] = (int32_t)(minVal + (int64_t)acc);
    }
    free(H1);
    free(H2);
    return OR_OK;
}

/*
 * RefHP output generation, Algorithm 3: B = 0; for every d in [1, R) where the
 * CDF steps (P1[d] > P1[d-1]) write B[P1[d-1]] = d; then the inclusive prefix
 * maximum of B.  minVal is added back at the end.
 */
int oracle_refhp_sort(const int32_t *A, int32_t *B, uint64_t n, int64_t minVal,
                      int64_t maxVal) {
    int64_t R;
    int rc = range_size(minVal, maxVal, &R);
    if (rc) return rc;
    if (n == 0) return OR_OK;
    if (A == NULL || B == NULL) return OR_ERR_INVALID_ARG;
    uint64_t *P1 = (uint64_t *)malloc((size_t)R * sizeof(uint64_t));
    int64_t *Bn = (int64_t *)calloc((size_t)n, sizeof(int64_t));
    if (!P1 || !Bn) { free(P1); free(Bn); return OR_ERR_NO_MEMORY; }
    rc = oracle_histogram(A, n, minVal, maxVal, P1);
    if (rc) { free(P1); free(Bn); return rc; }
    for (int64_t v = 1; v < R; v++) P1[v] += P1[v - 1];   /* CDF in place */
    for (int64_t d = 1; d < R; d++)
        if (P1[d] > P1[d - 1]) Bn[P1[d - 1]] = d;
    int64_t run = 0;
    for (uint64_t i = 0; i < n; i++) {
        if (Bn[i] > run) run = Bn[i];
        B[i] = (int32_t)(minVal + run);
    }
    free(P1);
    free(Bn);
    return OR_OK;
}

/*
 * RT-CDF itself, sequentially and step by step (Algorithms 4-7), exposing the
 * intermediates so that a device implementation's debug export can be compared:
 *   tile_hist[0..R-1]  the per-tile histograms (H after Algorithm 5)
 *   local_cdf[0..R-1]  H after the in-place inclusive scan of every tile
 *   O[0..m-1]          tile offsets (Algorithm 6)
 *   B[0..n-1]          output (Algorithm 7)
 * Any of the output pointers except B may be NULL.
 */
int oracle_rtcdf_sort(const int32_t *A, int32_t *B, uint64_t n, int64_t minVal,
                      int64_t maxVal, int64_t T, uint64_t *tile_hist,
                      uint64_t *local_cdf, uint64_t *O) {
    int64_t R;
    int rc = range_size(minVal, maxVal, &R);
    if (rc) return rc;
    if (T <= 0) return OR_ERR_INVALID_ARG;
    if (n > 0 && (A == NULL || B == NULL)) return OR_ERR_INVALID_ARG;
    int64_t m = (R + T - 1) / T;                       /* m = ceil(R / T) */
    uint64_t *H = (uint64_t *)calloc((size_t)R, sizeof(uint64_t));   /* H = 0 */
    uint64_t *Ot = (uint64_t *)malloc((size_t)m * sizeof(uint64_t));
    uint64_t *S = (uint64_t *)malloc((size_t)T * sizeof(uint64_t));
    if (!H || !Ot || !S) { free(H); free(Ot); free(S); return OR_ERR_NO_MEMORY; }

    for (uint64_t i = 0; i < n; i++) {                 /* range precondition */
        int64_t x = (int64_t)A[i] - minVal;
        if (x < 0 || x >= R) { free(H); free(Ot); free(S); return OR_ERR_KEY_OUT_OF_RANGE; }
    }

    /* Algorithm 5 for every tile: private histogram S of the keys falling in
     * [b, b + w), then H[b + x] += S[x]. */
    for (int64_t t = 0; t < m; t++) {
        int64_t b = t * T;
        int64_t w = (T < R - b) ? T : (R - b);
        memset(S, 0, (size_t)w * sizeof(uint64_t));
        for (uint64_t i = 0; i < n; i++) {
            int64_t x = ((int64_t)A[i] - minVal) - b;
            if (0 <= x && x < w) S[x] += 1;
        }
        for (int64_t x = 0; x < w; x++) H[b + x] += S[x];
    }
    if (tile_hist) memcpy(tile_hist, H, (size_t)R * sizeof(uint64_t));

    /* Local CDF: inclusive scan of H[b_t .. b_t + w_t - 1], in place. */
    for (int64_t t = 0; t < m; t++) {
        int64_t b = t * T;
        int64_t w = (T < R - b) ? T : (R - b);
        for (int64_t x = 1; x < w; x++) H[b + x] += H[b + x - 1];
    }
    if (local_cdf) memcpy(local_cdf, H, (size_t)R * sizeof(uint64_t));

    /* Algorithm 6: O[t] = number of keys in the tiles before t. */
    uint64_t offset = 0;
    for (int64_t t = 0; t < m; t++) {
        int64_t b = t * T;
        int64_t w = (T < R - b) ? T : (R - b);
        Ot[t] = offset;
        offset += H[b + w - 1];
    }
    if (O) memcpy(O, Ot, (size_t)m * sizeof(uint64_t));

    /* Algorithm 7 for every tile: B[O[t] + p] = b + min{ j : C[j] >= p + 1 }.
     * p runs upward, so the smallest j never decreases: it is found by
     * advancing j from its previous value while C[j] < p + 1. */
    for (int64_t t = 0; t < m; t++) {
        int64_t b = t * T;
        int64_t w = (T < R - b) ? T : (R - b);
        const uint64_t *C = H + b;
        uint64_t tileStart = Ot[t];
        uint64_t tileCount = C[w - 1];
        int64_t j = 0;
        for (uint64_t p = 0; p < tileCount; p++) {
            while (C[j] < p + 1) j++;
            B[tileStart + p] = (int32_t)(minVal + b + j);
        }
    }
    free(H);
    free(Ot);
    free(S);
    return OR_OK;
}

/*
 * Invariant checker for any claimed output B of input A (Lemmas 1-3 and
 * Theorem 1):
 *   (a) B is nondecreasing and every B[i] lies in [minVal, maxVal);
 *   (b) value v occupies exactly [CDF(v-1), CDF(v)), where CDF is computed from
 *       A, which together with (a) makes hist(B) = hist(A).
 * Returns 0 when all hold, 3 when A has a key out of range, otherwise -1 and
 * the first offending position in *bad (n when the failure is not positional).
 */
int oracle_check_sorted(const int32_t *A, const int32_t *B, uint64_t n, int64_t minVal,
                        int64_t maxVal, uint64_t *bad) {
    int64_t R;
    int rc = range_size(minVal, maxVal, &R);
    if (rc) return rc;
    *bad = n;
    if (n == 0) return OR_OK;
    uint64_t *cnt = (uint64_t *)malloc((size_t)R * sizeof(uint64_t));
    if (!cnt) return OR_ERR_NO_MEMORY;
    rc = oracle_histogram(A, n, minVal, maxVal, cnt);
    if (rc) { free(cnt); return rc; }
    /* Walk B against the CDF of A: position p must hold the value v whose
     * interval [start, start + c_v) contains p. */
    uint64_t start = 0;
    int64_t v = 0;
    for (uint64_t p = 0; p < n; p++) {
        while (v < R && start + cnt[v] <= p) { start += cnt[v]; v++; }
        int64_t got = (int64_t)B[p] - minVal;
        if (v >= R || got != v) { *bad = p; free(cnt); return -1; }
    }
    free(cnt);
    return OR_OK;
}

/*
 * Inclusive CDF of A (CDF[v] = sum_{u<=v} c_u), the quantity every output
 * position is defined by; used to compute single output values at sizes where
 * a full oracle output is not kept.
 */
int oracle_cdf(const int32_t *A, uint64_t n, int64_t minVal, int64_t maxVal,
               uint64_t *cdf) {
    int rc = oracle_histogram(A, n, minVal, maxVal, cdf);
    if (rc) return rc;
    int64_t R = maxVal - minVal;
    for (int64_t v = 1; v < R; v++) cdf[v] += cdf[v - 1];
    return OR_OK;
}
