// Simple random walks on a CSR graph: the self-return counts whose decay
// P(tau) ~ tau^(-dbar/2) gives the spectral dimension of a Levy graph (Sec.
// "Spectral dimension", Eq. (eqbard); App. A).
//
// One thread per walker.  Step tau of walker w takes word tau mod 4 of Philox
// block floor(tau / 4) at counter (w, floor(tau / 4), WALK<<24, 0): on a node
// of degree k > 0 the walker moves to neighbour floor(word * k / 2^32) of its
// CSR row; on a node without neighbours it stays.  The walk is a chain of
// dependent loads (row bounds, then the neighbour id), so the kernel is bound
// by memory latency; every walker of a warp steps together, and a warp adds
// its returns of a step with one atomic (ballot + popcount).
//
// Also here: xyl_philox, the raw generator of every random stream.
#include <cuda_runtime.h>

#include "internal.h"
#include "philox.cuh"

namespace xyl {
namespace {

constexpr int kWalkThreads = 256;

__global__ void __launch_bounds__(kWalkThreads) walk_kernel(const int32_t *__restrict__ row_ptr,
                                                            const int32_t *__restrict__ col, int32_t n, int64_t nnz,
                                                            const int32_t *__restrict__ start, uint32_t n_walkers,
                                                            uint32_t first_walker, int32_t n_steps, uint64_t key,
                                                            unsigned long long *returns)
{
    const uint32_t w = blockIdx.x * blockDim.x + threadIdx.x;
    const int s = w < n_walkers ? __ldg(start + w) : -1;
    // a start outside the graph leaves the walker out (returns[0] counts the walkers that ran)
    bool active = s >= 0 && s < n;
    const unsigned started = __ballot_sync(0xffffffffu, active);
    if ((threadIdx.x & 31u) == 0 && started) atomicAdd(returns, (unsigned long long)__popc(started));
    int v = s;
    Words4 x{0u, 0u, 0u, 0u};
    for (int32_t t = 0; t < n_steps; ++t) {
        if (active) {
            if ((t & 3) == 0) x = philox_draw(first_walker + w, (uint32_t)(t >> 2), kPurposeWalk, 0u, 0u, key);
            const int rb = __ldg(row_ptr + v), re = __ldg(row_ptr + v + 1);
            const uint32_t word = (t & 3) == 0 ? x.w0 : (t & 3) == 1 ? x.w1 : (t & 3) == 2 ? x.w2 : x.w3;
            if (rb < 0 || re < rb || (int64_t)re > nnz) {
                active = false;  // a row outside the CSR stops this walker
            } else if (re > rb) {
                const int next = __ldg(col + rb + (int)__umulhi(word, (uint32_t)(re - rb)));
                if (next < 0 || next >= n) active = false;  // a neighbour outside the graph stops it
                else v = next;
            }
        }
        const unsigned back = __ballot_sync(0xffffffffu, active && v == s);
        if ((threadIdx.x & 31u) == 0 && back) atomicAdd(returns + t + 1, (unsigned long long)__popc(back));
    }
}

// One Philox4x32-10 block per thread: the generator every stream of the
// library draws from, exposed so that it can be checked against other
// implementations.
__global__ void philox_kernel(const uint32_t *__restrict__ ctr, const uint32_t *__restrict__ key, int64_t n,
                              uint32_t *__restrict__ out)
{
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    const uint4 c = __ldg(reinterpret_cast<const uint4 *>(ctr) + q);
    const uint2 k = __ldg(reinterpret_cast<const uint2 *>(key) + q);
    const Words4 w = philox4x32_10(Words4{c.x, c.y, c.z, c.w}, k.x, k.y);
    reinterpret_cast<uint4 *>(out)[q] = make_uint4(w.w0, w.w1, w.w2, w.w3);
}

}  // namespace
}  // namespace xyl

using namespace xyl;

extern "C" int xyl_philox(const uint32_t *ctr, const uint32_t *key, int64_t n, uint32_t *out, void *stream)
{
    clear_error();
    if (n < 0) return fail(XYL_EINVAL, "xyl_philox: n < 0");
    if (n == 0) return XYL_OK;
    if (!ctr || !key || !out) return fail(XYL_EINVAL, "xyl_philox: NULL pointer");
    if ((reinterpret_cast<uintptr_t>(ctr) | reinterpret_cast<uintptr_t>(out)) % 16 ||
        reinterpret_cast<uintptr_t>(key) % 8)
        return fail(XYL_EINVAL, "xyl_philox: counters and outputs need 16-byte, keys 8-byte alignment");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const int64_t blocks = (n + 255) / 256;
    if (blocks > 0x7fffffff) return fail(XYL_EINVAL, "xyl_philox: too many blocks");
    philox_kernel<<<(unsigned)blocks, 256, 0, st>>>(ctr, key, n, out);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? XYL_OK : fail(XYL_ECUDA, "xyl_philox: %s", cudaGetErrorString(e));
}

extern "C" int xyl_walk_returns(const int32_t *row_ptr, const int32_t *col, int32_t n, int64_t nnz,
                                const int32_t *start, int64_t n_walkers, uint32_t first_walker, int32_t n_steps,
                                uint64_t seed, uint64_t *returns, void *stream)
{
    clear_error();
    if (n < 1 || nnz < 0 || n_steps < 0 || n_walkers < 0)
        return fail(XYL_EINVAL, "xyl_walk_returns: bad sizes (n=%d, nnz=%lld, n_steps=%d, n_walkers=%lld)", n,
                    (long long)nnz, n_steps, (long long)n_walkers);
    if ((uint64_t)first_walker + (uint64_t)n_walkers > 0x100000000ull)
        return fail(XYL_EINVAL, "xyl_walk_returns: walker ids beyond 2^32");
    if (!row_ptr || !returns || (nnz > 0 && !col) || (n_walkers > 0 && !start))
        return fail(XYL_EINVAL, "xyl_walk_returns: NULL pointer");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemsetAsync(returns, 0, sizeof(uint64_t) * ((size_t)n_steps + 1), st);
    if (e == cudaSuccess && n_walkers > 0) {
        const unsigned blocks = (unsigned)((n_walkers + kWalkThreads - 1) / kWalkThreads);
        walk_kernel<<<blocks, kWalkThreads, 0, st>>>(row_ptr, col, n, nnz, start, (uint32_t)n_walkers, first_walker,
                                                     n_steps, seed, reinterpret_cast<unsigned long long *>(returns));
        e = cudaGetLastError();
    }
    return e == cudaSuccess ? XYL_OK : fail(XYL_ECUDA, "xyl_walk_returns: %s", cudaGetErrorString(e));
}
