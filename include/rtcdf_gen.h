/*
 * rtcdf_gen.h -- seeded synthetic key generator (librtcdf_gen), used by the
 * tests and benchmarks to feed the sort and the CPU oracle the same inputs.
 * Not part of the sort: it holds none of the method's arithmetic.
 *
 * The three input shapes are those of the paper's evaluation (Section 4.1):
 * integers uniform on [minVal, minVal + R - 1]; a normal shape with mean
 * minVal + R/2 and standard deviation R/8, rounded and clipped to the range;
 * and all keys equal.  The stream is SplitMix64 indexed by element, so any
 * slice [first, first + n) can be generated on its own, on the host (numpy,
 * paper_2609_00843_gb300/gen) or on the device (this library), bit-identically.
 */
#ifndef RTCDF_GEN_H
#define RTCDF_GEN_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define RTCDF_GEN_UNIFORM 0
#define RTCDF_GEN_NORMAL 1
#define RTCDF_GEN_ALL_EQUAL 2

/*
 * Write keys first .. first + n - 1 of stream `seed` to the device buffer
 * `out` (n int32, caller-owned), asynchronously on `stream`.
 * Returns 0 on success, 1 bad argument, 2 range outside int32, 4 CUDA error
 * (no current device, or the launch failed).
 */
int rtcdf_gen_keys(int32_t *out, uint64_t n, uint64_t first, int64_t minVal, int64_t R,
                   int dist, uint64_t seed, struct CUstream_st *stream);

#ifdef __cplusplus
}
#endif

#endif /* RTCDF_GEN_H */
