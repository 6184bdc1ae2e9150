// Philox4x32-10 counter-based generator (Salmon, Moraes, Dror & Shaw, SC'11):
// ten rounds of the 4x32 Philox bijection keyed by a 64-bit key bumped by the
// Weyl constants between rounds.  Usable from host and device code.
#pragma once

#include <stdint.h>

#if defined(__CUDACC__)
#define XYL_HD __host__ __device__ __forceinline__
#else
#define XYL_HD inline
#endif

namespace xyl {

struct Words4 {
    uint32_t w0, w1, w2, w3;
};

// Stream purposes: top byte of counter word 2.
enum : uint32_t { kPurposeGraph = 0u, kPurposeInit = 1u, kPurposeMet = 2u, kPurposePt = 3u, kPurposeWalk = 4u };

XYL_HD uint32_t mul_hi32(uint32_t a, uint32_t b)
{
#if defined(__CUDA_ARCH__)
    return __umulhi(a, b);
#else
    return (uint32_t)(((uint64_t)a * (uint64_t)b) >> 32);
#endif
}

XYL_HD Words4 philox4x32_10(Words4 c, uint32_t k0, uint32_t k1)
{
    const uint32_t kMulA = 0xD2511F53u, kMulB = 0xCD9E8D57u;
    const uint32_t kWeylA = 0x9E3779B9u, kWeylB = 0xBB67AE85u;
#if defined(__CUDACC__)
#pragma unroll
#endif
    for (int round = 0; round < 10; ++round) {
        const uint32_t hiA = mul_hi32(kMulA, c.w0), loA = kMulA * c.w0;
        const uint32_t hiB = mul_hi32(kMulB, c.w2), loB = kMulB * c.w2;
        Words4 n;
        n.w0 = hiB ^ c.w1 ^ k0;
        n.w1 = loB;
        n.w2 = hiA ^ c.w3 ^ k1;
        n.w3 = loA;
        c = n;
        k0 += kWeylA;
        k1 += kWeylB;
    }
    return c;
}

// Counter layout shared by every stream: (w0, w1, purpose<<24 | sub, sample).
XYL_HD Words4 philox_draw(uint32_t w0, uint32_t w1, uint32_t purpose, uint32_t sub, uint32_t sample,
                          uint64_t key)
{
    Words4 c{w0, w1, (purpose << 24) | (sub & 0xFFFFFFu), sample};
    return philox4x32_10(c, (uint32_t)key, (uint32_t)(key >> 32));
}

// Uniforms in [0,1): 53 bits from (hi, lo) words, 24 bits from one word.
XYL_HD double uniform53(uint32_t hi, uint32_t lo)
{
    const uint64_t v = ((((uint64_t)hi) << 32) | (uint64_t)lo) >> 11;
    return (double)v * (1.0 / 9007199254740992.0);
}

XYL_HD float uniform24(uint32_t x)
{
    return (float)(x >> 8) * (1.0f / 16777216.0f);
}

}  // namespace xyl
