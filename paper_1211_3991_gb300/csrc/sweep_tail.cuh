// End of a sweep in the FP32 batched kernels: parallel tempering over the
// slots of one sample and the leader's bookkeeping.  Every CTA of the sample
// calls it with the same energies, so every CTA takes the same decisions.
#pragma once

#include "device.cuh"

namespace xyl {

constexpr int kMaxReplicas = 256;

// Cluster barrier in two halves (release on arrival, acquire on wait), so a
// CTA can do work that does not depend on the other CTAs in between.
__device__ __forceinline__ void cluster_arrive() { asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory"); }
__device__ __forceinline__ void cluster_wait() { asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory"); }

// The FP64 test u < exp(x), mostly decided without a double-precision exp:
// exp(x) >= 1 > u for x >= 0; for x < -80, exp(x) < 2^-53, so only u = 0
// passes; otherwise a single-precision estimate (relative error below 1e-5
// for |x| <= 80: the rounding of x to float and of x log2(e), and the 2^-22
// error of the hardware exponential) decides whenever u lies outside its
// error band, and the double-precision exp decides the rest.
__device__ __forceinline__ bool pt_accept(double u, double x)
{
    if (x >= 0.0) return true;
    if (x < -80.0) return u == 0.0;
    const double e = (double)__expf((float)x);
    const double gap = u - e;
    if (fabs(gap) > 2e-5 * e) return gap < 0.0;
    return u < exp(x);
}

// App. B "Improved equilibrium dynamics": at sweep t, slots (k, k+1) with k of
// the parity of t swap their replicas with probability min(1, exp((b_k -
// b_k+1)(E_k - E_k+1))), one PT draw per pair (FP64 arithmetic and 53-bit
// uniforms).  E is indexed by replica, rep_at / slot_of are this CTA's copies
// of the labels, beta_s the slots' FP64 inverse temperatures in shared memory
// (NULL: read from the plan).  The leader's counters are fire-and-forget
// atomics, so no read of global memory sits on its path.  The leader then writes the labels and energies back and, on
// measurement sweeps, adds e, e^2, |m|, m_x, m_y, m^2, m^4 and chi(k_min) of
// each slot (Sec. III) from the per-replica sums obs_s; dim = 3 (O(3) spins)
// adds the third component to m^2 and |F(k)|^2 and sums m_z.
__device__ __forceinline__ void pt_and_record(const DevPlan &P, const DevSample &d, const double *E, int *rep_at,
                                              int *slot_of, uint32_t t, uint32_t ops, bool leader, bool met,
                                              bool measure, const double *obs_s, const double *beta_s = nullptr,
                                              int dim = 2)
{
    const int R = d.R;
    if (ops & XYL_OP_PT) {
        for (int p = threadIdx.x; 2 * p + (int)(t & 1u) + 1 < R; p += blockDim.x) {
            const int k = 2 * p + (int)(t & 1u);
            const int a = rep_at[k], b = rep_at[k + 1];
            const double bk = beta_s ? beta_s[k] : P.beta[d.rep_off + k];
            const double bk1 = beta_s ? beta_s[k + 1] : P.beta[d.rep_off + k + 1];
            const double x = (bk - bk1) * (E[a] - E[b]);
            const Words4 w = philox_draw((uint32_t)k, t, kPurposePt, 0u, d.sample_id, P.key);
            const bool accept = pt_accept(uniform53(w.w0, w.w1), x);
            if (leader) atomicAdd(&P.pt_try[d.rep_off + k], 1ull);
            if (accept) {
                rep_at[k] = b;
                rep_at[k + 1] = a;
                slot_of[b] = k;
                slot_of[a] = k + 1;
                if (leader) atomicAdd(&P.pt_acc[d.rep_off + k], 1ull);
            }
        }
        __syncthreads();
    }
    if (!leader) return;
    const double invN = 1.0 / (double)d.N;
    for (int k = threadIdx.x; k < R; k += blockDim.x) {
        const int r = rep_at[k];
        P.rep_at[d.rep_off + k] = r;
        P.slot_of[d.rep_off + r] = k;
        P.last_E[d.rep_off + k] = E[k];
        if (met) atomicAdd(&P.met_try[d.rep_off + k], (unsigned long long)d.N);
        if (measure) {
            const double *o = obs_s + (size_t)r * kObsStride;
            const double e = E[r] * invN;
            const double mx = __ldcg(o + kObsMx) * invN, my = __ldcg(o + kObsMy) * invN;
            const double mz = dim == 3 ? __ldcg(o + kObsMz) * invN : 0.0;
            double m2 = mx * mx + my * my;
            double f1 = 0.0, f2 = 0.0;
#pragma unroll
            for (int f = kObsF1xRe; f <= kObsF1yIm; ++f) {
                const double z = __ldcg(o + f);
                f1 += z * z;
            }
#pragma unroll
            for (int f = kObsF2xRe; f <= kObsF2yIm; ++f) {
                const double z = __ldcg(o + f);
                f2 += z * z;
            }
            if (dim == 3) {
                m2 += mz * mz;
                const double a1 = __ldcg(o + kObsF1zRe), b1 = __ldcg(o + kObsF1zIm);
                const double a2 = __ldcg(o + kObsF2zRe), b2 = __ldcg(o + kObsF2zIm);
                f1 += a1 * a1 + b1 * b1;
                f2 += a2 * a2 + b2 * b2;
            }
            double *a = P.acc + (size_t)(d.rep_off + k) * kAccCount;
            a[XYL_ACC_N] += 1.0;
            a[XYL_ACC_E] += e;
            a[XYL_ACC_E2] += e * e;
            a[XYL_ACC_ABSM] += sqrt(m2);
            a[XYL_ACC_MX] += mx;
            a[XYL_ACC_MY] += my;
            a[XYL_ACC_M2] += m2;
            a[XYL_ACC_M4] += m2 * m2;
            a[XYL_ACC_CHIK] += (f1 + f2) * 0.5 * invN;
            if (dim == 3) a[XYL_ACC_MZ] += mz;
        }
    }
}

}  // namespace xyl
