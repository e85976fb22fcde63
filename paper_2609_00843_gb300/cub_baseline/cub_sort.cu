// On-GPU comparison for the benchmark, not part of the sort: CUB's stable LSD
// radix sort (cub::DeviceRadixSort::SortKeys, a library call) restricted to
// the bits [0, ceil(log2 R)) that a known range of size R can occupy -- the
// configuration the paper compares against (Section 4.2).  Keys are first
// normalised to uint32 (key - minVal) and denormalised afterwards, in two
// small kernels that the benchmark times separately.
#include <cstdint>
#include <cub/device/device_radix_sort.cuh>
#include <cuda_runtime.h>

namespace {

__global__ void normalize_kernel(const int32_t *in, uint32_t *out, uint64_t n, uint32_t min_u) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x)
        out[i] = (uint32_t)in[i] - min_u;
}

__global__ void denormalize_kernel(const uint32_t *in, int32_t *out, uint64_t n, uint32_t min_u) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x)
        out[i] = (int32_t)(in[i] + min_u);
}

int end_bit_for(int64_t R) {
    int b = 0;
    while (b < 32 && ((int64_t)1 << b) < R) b++;
    return b == 0 ? 1 : b;
}

unsigned grid_for(uint64_t n) {
    uint64_t g = (n + 255) / 256;
    return (unsigned)(g > 152ull * 16 ? 152ull * 16 : (g ? g : 1));
}

}  // namespace

extern "C" {

// Temporary storage CUB needs for n keys over `bits` bits.
int rtcdf_cub_temp_bytes(uint64_t n, int64_t R, size_t *bytes) {
    size_t t = 0;
    cudaError_t e = cub::DeviceRadixSort::SortKeys(nullptr, t, (const uint32_t *)nullptr,
                                                   (uint32_t *)nullptr, (int64_t)n, 0, end_bit_for(R));
    *bytes = t;
    return e == cudaSuccess ? 0 : 4;
}

int rtcdf_cub_normalize(const int32_t *in, uint32_t *keys, uint64_t n, int64_t minVal,
                        cudaStream_t s) {
    normalize_kernel<<<grid_for(n), 256, 0, s>>>(in, keys, n, (uint32_t)(int32_t)minVal);
    return cudaGetLastError() == cudaSuccess ? 0 : 4;
}

int rtcdf_cub_sort_keys(const uint32_t *keys_in, uint32_t *keys_out, void *temp, size_t temp_bytes,
                        uint64_t n, int64_t R, cudaStream_t s) {
    cudaError_t e = cub::DeviceRadixSort::SortKeys(temp, temp_bytes, keys_in, keys_out, (int64_t)n,
                                                   0, end_bit_for(R), s);
    return e == cudaSuccess ? 0 : 4;
}

int rtcdf_cub_denormalize(const uint32_t *keys, int32_t *out, uint64_t n, int64_t minVal,
                          cudaStream_t s) {
    denormalize_kernel<<<grid_for(n), 256, 0, s>>>(keys, out, n, (uint32_t)(int32_t)minVal);
    return cudaGetLastError() == cudaSuccess ? 0 : 4;
}

}  // extern "C"
