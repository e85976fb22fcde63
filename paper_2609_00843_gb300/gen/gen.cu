// Device version of the seeded input generator (see gen/__init__.py for the
// definition).  Holds none of the sort's arithmetic; produces, for the same
// (seed, index range, minVal, R, distribution), exactly the keys the numpy
// version produces.  Every floating-point step of the normal shape is a single
// correctly rounded IEEE-754 single-precision operation (no contraction into
// FMA), matching numpy's float32 arithmetic.
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
    const float Rf = __ull2float_rn((unsigned long long)R);
    const float half = __fdiv_rn(Rf, 2.0f), sigma = __fdiv_rn(Rf, 8.0f);
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += stride) {
        const uint64_t idx = first + i;
        int64_t key;
        if (dist == RTCDF_GEN_UNIFORM) {
            uint64_t u = word(seed, idx * 16) >> 32;
            key = minVal + (int64_t)((u * (uint64_t)R) >> 32);
        } else if (dist == RTCDF_GEN_NORMAL) {
            uint64_t S = 0;
#pragma unroll
            for (int j = 0; j < 6; j++) {
                const uint64_t w = word(seed, idx * 16 + j);
                S += (w >> 32) + (w & 0xFFFFFFFFull);
            }
            const float z = __fadd_rn(__fmul_rn(__ull2float_rn(S), 0x1p-32f), -6.0f);
            const float o = __fadd_rn(half, __fmul_rn(sigma, z));
            const float r = (o >= 0.0f) ? floorf(__fadd_rn(o, 0.5f)) : -floorf(__fadd_rn(-o, 0.5f));
            int64_t ri = (int64_t)r;
            ri = ri < 0 ? 0 : (ri > R - 1 ? R - 1 : ri);
            key = minVal + ri;
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
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
        return 4;
    uint64_t blocks = (n + 255) / 256;
    uint64_t cap = (uint64_t)sms * 16;
    if (blocks > cap) blocks = cap;
    gen_kernel<<<(unsigned)blocks, 256, 0, stream>>>(out, n, first, minVal, R, dist, seed);
    return cudaGetLastError() == cudaSuccess ? 0 : 4;
}
