// Bandwidth probes behind the on-chip roofline peaks the benchmark reports
// against (HBM and the tensor pipes are measured by other means): streaming
// reads of an L2-resident buffer, and random 8-byte gathers from shared
// memory.  Built and run by paper_1211_3991_gb300/peaks.py; not part of
// libxyl.
#include <cuda_runtime.h>
#include <stdint.h>

namespace {

// Every thread reads float4s of the buffer, grid-strided, `reps` times over;
// the sum goes to sink so that no load is dropped.
__global__ void l2_read_kernel(const float4 *__restrict__ buf, size_t n4, int reps, float *sink)
{
    float acc = 0.f;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (int r = 0; r < reps; ++r)
        for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += stride) {
            const float4 v = __ldcg(buf + i);
            acc += v.x + v.y + v.z + v.w;
        }
    if (acc == 12345.678f) sink[0] = acc;  // never true for the zeroed buffer; keeps the loads
}

// Each CTA fills kWords 8-byte words of shared memory, then every thread
// makes `rounds` x kGathers independent gathers at pseudo-random word indices
// (the top bits of a per-thread linear congruential sequence, one multiply-add
// an index), kGathers loads in flight at a time.
constexpr int kWords = 16384;  // 128 KB
constexpr int kGathers = 8;

__global__ void smem_gather_kernel(int rounds, float *sink)
{
    extern __shared__ float2 words[];
    for (int k = threadIdx.x; k < kWords; k += blockDim.x) words[k] = make_float2((float)k, 1.f);
    __syncthreads();
    uint32_t x = (blockIdx.x * 1024u + threadIdx.x) * 2654435761u + 12345u;
    float acc = 0.f;
    for (int r = 0; r < rounds; ++r) {
        uint32_t idx[kGathers];
#pragma unroll
        for (int q = 0; q < kGathers; ++q) {
            x = x * 1664525u + 1013904223u;
            idx[q] = x >> 18;  // 14 bits: [0, kWords)
        }
        float2 v[kGathers];
#pragma unroll
        for (int q = 0; q < kGathers; ++q) v[q] = words[idx[q]];
#pragma unroll
        for (int q = 0; q < kGathers; ++q) acc += v[q].x * v[q].y;
    }
    if (acc == -1.f) sink[0] = acc;  // never true: the words are non-negative
}

}  // namespace

extern "C" int probe_l2_read(const void *buf, size_t bytes, int reps, float *sink, int blocks, int threads,
                             void *stream)
{
    l2_read_kernel<<<blocks, threads, 0, (cudaStream_t)stream>>>(static_cast<const float4 *>(buf), bytes / 16, reps,
                                                                 sink);
    return (int)cudaGetLastError();
}

extern "C" int probe_smem_gather(int rounds, float *sink, int blocks, int threads, void *stream)
{
    const size_t smem = kWords * sizeof(float2);
    cudaError_t e = cudaFuncSetAttribute(smem_gather_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return (int)e;
    smem_gather_kernel<<<blocks, threads, smem, (cudaStream_t)stream>>>(rounds, sink);
    return (int)cudaGetLastError();
}
