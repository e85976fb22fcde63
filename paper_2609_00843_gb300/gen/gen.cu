// Device version of the seeded input generator (see gen/__init__.py for the
// definition).  Holds none of the sort's arithmetic; produces, for the same
// (seed, index range, minVal, R, distribution), exactly the keys the numpy
// version produces.  Every floating-point step of the normal shape is a single
// correctly rounded IEEE-754 double operation (no contraction into FMA).
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/rtcdf_gen.h"

namespace {

__device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ uint64_t word(uint64_t seed, uint64_t ctr) {
    return mix64(seed + (ctr + 1) * 0x9E3779B97F4A7C15ull);
}

__global__ void gen_kernel(int32_t *out, uint64_t n, uint64_t first, int64_t minVal, int64_t R,
                           int dist, uint64_t seed) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const double mu = __dadd_rn((double)minVal, (double)R / 2.0);
    const double sigma = (double)R / 8.0;
    const double lo = (double)minVal, hi = (double)(minVal + R - 1);
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += stride) {
        const uint64_t idx = first + i;
        int64_t key;
        if (dist == RTCDF_GEN_UNIFORM) {
            uint64_t u = word(seed, idx * 16) >> 32;
            key = minVal + (int64_t)((u * (uint64_t)R) >> 32);
        } else if (dist == RTCDF_GEN_NORMAL) {
            uint64_t S = 0;
#pragma unroll
            for (int j = 0; j < 12; j++) S += word(seed, idx * 16 + j) >> 32;
            double z = __dadd_rn(__dmul_rn((double)S, 0x1p-32), -6.0);
            double xr = __dadd_rn(mu, __dmul_rn(sigma, z));
            double r = (xr >= 0.0) ? floor(__dadd_rn(xr, 0.5)) : -floor(__dadd_rn(-xr, 0.5));
            r = fmin(fmax(r, lo), hi);
            key = (int64_t)r;
        } else {
            key = minVal + R / 3;
        }
        out[i] = (int32_t)key;
    }
}

}  // namespace

extern "C" int rtcdf_gen_keys(int32_t *out, uint64_t n, uint64_t first, int64_t minVal,
                              int64_t R, int dist, uint64_t seed, cudaStream_t stream) {
    if (n == 0) return 0;
    if (!out || R <= 0 || R > (1ll << 32)) return 1;
    if (minVal < -(1ll << 31) || minVal + R > (1ll << 31)) return 2;
    if (dist < 0 || dist > 2) return 1;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    uint64_t blocks = (n + 255) / 256;
    uint64_t cap = (uint64_t)(sms > 0 ? sms : 132) * 16;
    if (blocks > cap) blocks = cap;
    gen_kernel<<<(unsigned)blocks, 256, 0, stream>>>(out, n, first, minVal, R, dist, seed);
    return cudaGetLastError() == cudaSuccess ? 0 : 4;
}
