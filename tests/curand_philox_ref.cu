// Test helper: cuRAND's own Philox4x32-10 block function (curand_kernel.h),
// one block per (counter, key) pair, to check the library's generator against.
#include <curand_kernel.h>

__global__ void curand_philox_kernel(const uint4 *ctr, const uint2 *key, long long n, uint4 *out)
{
    const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q < n) out[q] = curand_Philox4x32_10(ctr[q], key[q]);
}

extern "C" int curand_philox_blocks(const void *ctr, const void *key, long long n, void *out)
{
    if (n <= 0) return 0;
    curand_philox_kernel<<<(unsigned)((n + 255) / 256), 256>>>(static_cast<const uint4 *>(ctr),
                                                               static_cast<const uint2 *>(key), n,
                                                               static_cast<uint4 *>(out));
    if (cudaGetLastError() != cudaSuccess) return 1;
    return cudaDeviceSynchronize() == cudaSuccess ? 0 : 2;
}
