// Device-side descriptors and the per-spin update arithmetic shared by the
// engines of libxyl.  Spins are unit 2-vectors (XY; O(3) spins, unit
// 3-vectors stored as padded 4-vectors, run on the plain engines); the
// Hamiltonian is H = -sum_{i<j} J_ij S_i . S_j, Eq. (HXY).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/xyl.h"
#include "philox.cuh"

namespace xyl {

// Per-replica sums produced by the last pass of a sweep (FP64 slots):
// energy, magnetisation and the Fourier sums at k1 = (2pi/L, 0), k2 = (0, 2pi/L)
// for both spin components (Sec. III, definition of xi_2).
enum ObsField : int {
    kObsE = 0,
    kObsMx, kObsMy,
    kObsF1xRe, kObsF1xIm, kObsF1yRe, kObsF1yIm,   // k1: spin x / spin y components
    kObsF2xRe, kObsF2xIm, kObsF2yRe, kObsF2yIm,   // k2
    kObsCount,                                    // fields of two-component spins
    kObsMz = kObsCount,                           // O(3): third component
    kObsF1zRe, kObsF1zIm, kObsF2zRe, kObsF2zIm,
    kObsCount3                                    // fields of three-component spins
};
constexpr int kObsStride = 16;
constexpr int kMaxColorsBatched = 32;  // colour classes per graph the batched engine accepts
constexpr int kSinTerms = 15;
constexpr int kCosTerms = 16;
constexpr int kAccCount = XYL_ACC_COUNT;

struct DevSample {
    int32_t N, Q, R, L;
    uint32_t sample_id;
    int32_t max_deg;
    int32_t color_off;   // into color_ptr (Q + 1 entries per sample)
    int32_t rep_off;     // into per-replica and per-slot arrays (R per sample)
    int64_t site_off;    // into perm / phase arrays (N per sample)
    int64_t row_off;     // into row_ptr (N + 1 per sample)
    int64_t col_off;     // into col (nnz per sample)
    int64_t spin_off;    // into the spin array, in vectors
};

struct DevPlan {
    const DevSample *samples;
    int32_t n_samples;
    int32_t total_R;
    const int32_t *row_ptr;
    const int32_t *col;        // colour-sorted ids local to the sample
    const int32_t *perm;       // colour-sorted id -> original id
    const int32_t *color_ptr;
    const void *phase;         // per site (cos kx, sin kx, cos ky, sin ky): float4 or double4_32a
    void *spins;               // float2 / double2 (O(3): float4 / double4_32a)
    const double *beta;        // per slot
    const double *delta;       // per slot
    int32_t *slot_of;          // per replica: slot it sits at
    int32_t *rep_at;           // per slot: replica sitting there
    double *obs;               // [2][total_R][kObsStride] per-replica sums of the current sweep
    double *last_E;            // [total_R] energy after the last sweep
    double *acc;               // [total_R slots][kAccCount]
    unsigned long long *met_acc, *met_try, *pt_acc, *pt_try;  // per slot
    uint32_t *sweep;           // per sample sweep counter
    int32_t *status;           // 0 or an XYL_E* code
    unsigned int *barrier;     // per sample arrival counters (batched engine)
    double *drift;             // largest |E_fused - E_fp64| seen by a recompute
    const uint16_t *push;      // per site: CTAs of its group (bit = rank) that read it (site-split resident shape)
    const void *field;         // per site (colour-sorted, site_off): field vector float2 / double2, or NULL
    uint64_t key;              // Philox key of the spin streams
    // Maclaurin coefficients (-1)^k / (2k+1)! and (-1)^k / (2k)! of the FP64 sin/cos
    double sin_coef[kSinTerms];
    double cos_coef[kCosTerms];
};

// Debug builds (compiled with XYL_DEBUG): every neighbour id a kernel is about
// to follow is checked against its array before the access.  A bad id sets the
// status word to XYL_EBOUNDS (the first error code recorded stays) and is
// replaced by `safe`, so that the access stays inside the array; the run goes
// on and the caller reads the status.  Release builds compile the check out.
__device__ __forceinline__ int checked_id(const DevPlan &P, int j, int limit, int safe)
{
#ifdef XYL_DEBUG
    if ((unsigned)j >= (unsigned)limit) {
        atomicCAS(P.status, 0, XYL_EBOUNDS);
        return safe;
    }
#endif
    return j;
}

// Whether sweep t (its index before the increment at its end) ends with a
// measurement: every measure_every-th sweep (0: never).
__device__ __forceinline__ bool measurement_sweep(uint32_t t, int measure_every)
{
    return measure_every > 0 && ((t + 1u) % (uint32_t)measure_every) == 0u;
}

// The colour class [cb, ce) of a sample, checked in debug builds to lie in [0, n].
__device__ __forceinline__ void checked_class(const DevPlan &P, int &cb, int &ce, int n)
{
#ifdef XYL_DEBUG
    if (cb < 0 || cb > ce || ce > n) {
        atomicCAS(P.status, 0, XYL_EBOUNDS);
        cb = ce = 0;
    }
#endif
}

// sin and cos of |x| <= pi by their Maclaurin series (Horner in x^2 with IEEE
// fused multiply-add; truncation below 3e-17).  Every rounding step is fixed,
// so the FP64 engine's trajectory does not depend on a math library.
__device__ __forceinline__ void sincos_series(const DevPlan &P, double x, double *sn, double *cs)
{
    const double y = x * x;
    double p = P.sin_coef[kSinTerms - 1];
#pragma unroll
    for (int k = kSinTerms - 2; k >= 0; --k) p = fma(p, y, P.sin_coef[k]);
    double q = P.cos_coef[kCosTerms - 1];
#pragma unroll
    for (int k = kCosTerms - 2; k >= 0; --k) q = fma(q, y, P.cos_coef[k]);
    *sn = x * p;
    *cs = q;
}

template <typename Real> struct Vec2T;
template <> struct Vec2T<float> { using type = float2; };
template <> struct Vec2T<double> { using type = double2; };
template <typename Real> using Vec2 = typename Vec2T<Real>::type;

template <typename Real> struct Vec4T;
template <> struct Vec4T<float> { using type = float4; };
template <> struct Vec4T<double> { using type = double4_32a; };
template <typename Real> using Vec4 = typename Vec4T<Real>::type;

// ---------------------------------------------------------------------------
// Metropolis step of one spin (App. B): proposal = rotation of s by
// delta = Delta (2u - 1); dE = -(s' - s) . h; accept iff dE <= 0 or
// u' < exp(-beta dE).  FP64 uses 53-bit uniforms from (w0,w1) and (w2,w3);
// FP32 uses 24-bit uniforms from w0 and w1, hardware sincos/exp and
// renormalises the rotated proposal.
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool metropolis_step(const DevPlan &P, double sx, double sy, double hx, double hy,
                                                double beta, double half_width, Words4 x, double &nx, double &ny)
{
    const double ud = uniform53(x.w0, x.w1), ua = uniform53(x.w2, x.w3);
    double sn, cs;
    sincos_series(P, half_width * (2.0 * ud - 1.0), &sn, &cs);
    nx = cs * sx - sn * sy;
    ny = sn * sx + cs * sy;
    const double dE = -((nx - sx) * hx + (ny - sy) * hy);
    return dE <= 0.0 || ua < exp(-beta * dE);
}

// FP32 draws: one Philox block at counter (site, t, MET<<24 | r/2, sample)
// serves replicas 2p and 2p+1; the even replica takes (w0, w1), the odd one
// (w2, w3).
__device__ __forceinline__ Words4 met_block_f32(uint32_t site, uint32_t t, int r, uint32_t sample, uint64_t key)
{
    return philox_draw(site, t, kPurposeMet, (uint32_t)(r >> 1), sample, key);
}

__device__ __forceinline__ bool metropolis_step_f32(float sx, float sy, float hx, float hy, float beta,
                                                    float half_width, uint32_t wd, uint32_t wa, float &nx, float &ny)
{
    // explicit roundings: the result does not depend on how a kernel is compiled
    const float ud = uniform24(wd), ua = uniform24(wa);
    float sn, cs;
    __sincosf(__fmul_rn(half_width, __fmaf_rn(2.0f, ud, -1.0f)), &sn, &cs);
    const float px = __fmaf_rn(cs, sx, __fmul_rn(-sn, sy));
    const float py = __fmaf_rn(sn, sx, __fmul_rn(cs, sy));
    const float inv = rsqrtf(__fmaf_rn(px, px, __fmul_rn(py, py)));
    nx = __fmul_rn(px, inv);
    ny = __fmul_rn(py, inv);
    const float dE = -__fmaf_rn(__fsub_rn(nx, sx), hx, __fmul_rn(__fsub_rn(ny, sy), hy));
    return dE <= 0.0f || ua < __expf(__fmul_rn(-beta, dE));
}

// Overrelaxation (App. B; Creutz): reflection of s about the local field h,
// s' = 2 (s.h) h / |h|^2 - s; s unchanged when h = 0.
__device__ __forceinline__ void overrelax_step(double sx, double sy, double hx, double hy, double &nx, double &ny)
{
    const double h2 = hx * hx + hy * hy;
    if (h2 > 0.0) {
        const double k = 2.0 * (sx * hx + sy * hy) / h2;
        nx = k * hx - sx;
        ny = k * hy - sy;
    } else {
        nx = sx;
        ny = sy;
    }
}

__device__ __forceinline__ void overrelax_step(float sx, float sy, float hx, float hy, float &nx, float &ny)
{
    const float h2 = __fmaf_rn(hx, hx, __fmul_rn(hy, hy));
    if (h2 > 0.0f) {
        const float k = __fdividef(__fmul_rn(2.0f, __fmaf_rn(sx, hx, __fmul_rn(sy, hy))), h2);
        nx = __fmaf_rn(k, hx, -sx);
        ny = __fmaf_rn(k, hy, -sy);
    } else {
        nx = sx;
        ny = sy;
    }
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Bounded spin on a monotone counter; returns false after `limit` polls.
__device__ __forceinline__ bool wait_counter_at_least(const unsigned int *ctr, unsigned int target, unsigned int limit)
{
    for (unsigned int it = 0; it < limit; ++it) {
        unsigned int v;
        asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(ctr) : "memory");
        if (v >= target) return true;
        __nanosleep(64);
    }
    return false;
}

}  // namespace xyl
