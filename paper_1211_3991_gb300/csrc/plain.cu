// Plain engine: one launch per colour phase, one thread per (site, replica),
// replica-major spins ([sample][replica][site]).  This is the straightforward
// GPU form of the colour-sequential sweep of App. B ("generalised red-black
// Gauss-Seidel"): sites of one colour are mutually unlinked and update
// together; colours run one after another.  Instantiated in FP64 (the
// reference GPU kernel) and FP32.
#include <cuda_runtime.h>

#include <algorithm>

#include "engines.h"

namespace xyl {
namespace {

constexpr int kPlainBlock = 256;
constexpr int kGather = 4;  // neighbour loads in flight per thread

template <typename Real>
__device__ __forceinline__ Vec2<Real> make_vec2(Real x, Real y);
template <> __device__ __forceinline__ float2 make_vec2<float>(float x, float y) { return make_float2(x, y); }
template <> __device__ __forceinline__ double2 make_vec2<double>(double x, double y) { return make_double2(x, y); }

// One colour phase of the Metropolis (IS_MET) or overrelaxation pass.  With
// FUSE the replica's energy (links to lower colours, counted at their upper
// endpoint) is reduced into obs[0] on every sweep, and its magnetisation and
// Fourier sums on the sweeps that end with a measurement (every meas_every-th;
// meas_every = 0: none).  With
// DISORDER a neighbour id with its top bit set is a link with J = -1 (the
// neighbour's spin enters the local field negated, exactly J * S_j), and a
// site field, when the plan has one, is added after the neighbours.
template <typename Real, bool IS_MET, bool FUSE, bool DISORDER>
__global__ void __launch_bounds__(kPlainBlock) plain_phase_kernel(DevPlan P, int c, int meas_every)
{
    using V = Vec2<Real>;
    using V4 = Vec4<Real>;
    const int s = blockIdx.z, r = blockIdx.y;
    const DevSample d = P.samples[s];
    if (r >= d.R || c >= d.Q) return;
    int cb = P.color_ptr[d.color_off + c], ce = P.color_ptr[d.color_off + c + 1];
    checked_class(P, cb, ce, d.N);
    const int base = cb + (int)blockIdx.x * kPlainBlock;
    if (base >= ce) return;
    const int i = base + (int)threadIdx.x;
    const bool active = i < ce;
    V *sp = reinterpret_cast<V *>(P.spins) + d.spin_off + (int64_t)r * d.N;
    const int32_t *rp = P.row_ptr + d.row_off;
    const int32_t *cl = P.col + d.col_off;
    const int slot = P.slot_of[d.rep_off + r];

    Real nx = 0, ny = 0, lx = 0, ly = 0;
    bool accepted = false;
    if (active) {
        const V si = sp[i];
        Real hx = 0, hy = 0;
        const int rb = rp[i], re = rb + checked_id(P, rp[i + 1] - rp[i], d.max_deg + 1, 0);
        // neighbours in groups of kGather: every id of a group, then every spin,
        // are in flight together; the sums still run in row order
        for (int k0 = rb; k0 < re; k0 += kGather) {
            int raw[kGather];
            V sv[kGather];
#pragma unroll
            for (int q = 0; q < kGather; ++q) raw[q] = k0 + q < re ? cl[k0 + q] : 0;
#pragma unroll
            for (int q = 0; q < kGather; ++q)
                if (k0 + q < re) sv[q] = sp[checked_id(P, DISORDER ? (raw[q] & 0x7fffffff) : raw[q], d.N, 0)];
#pragma unroll
            for (int q = 0; q < kGather; ++q) {
                if (k0 + q >= re) break;
                const int j = DISORDER ? (raw[q] & 0x7fffffff) : raw[q];
                V sj = sv[q];
                if (DISORDER && raw[q] < 0) {
                    sj.x = -sj.x;
                    sj.y = -sj.y;
                }
                hx += sj.x;
                hy += sj.y;
                if (FUSE && j < cb) {
                    lx += sj.x;
                    ly += sj.y;
                }
            }
        }
        if (DISORDER && P.field) {
            // the site's own field after its neighbours; the fused energy takes -h_i . S_i once
            const V f = reinterpret_cast<const V *>(P.field)[d.site_off + i];
            hx += f.x;
            hy += f.y;
            if (FUSE) {
                lx += f.x;
                ly += f.y;
            }
        }
        if (IS_MET) {
            const uint32_t site = (uint32_t)P.perm[d.site_off + i];
            if constexpr (sizeof(Real) == 8) {
                const Words4 x = philox_draw(site, P.sweep[s], kPurposeMet, (uint32_t)r, d.sample_id, P.key);
                accepted = metropolis_step(P, si.x, si.y, hx, hy, P.beta[d.rep_off + slot], P.delta[d.rep_off + slot],
                                           x, nx, ny);
            } else {
                const Words4 x = met_block_f32(site, P.sweep[s], r, d.sample_id, P.key);
                accepted = metropolis_step_f32(si.x, si.y, hx, hy, (float)P.beta[d.rep_off + slot],
                                               (float)P.delta[d.rep_off + slot], (r & 1) ? x.w2 : x.w0,
                                               (r & 1) ? x.w3 : x.w1, nx, ny);
            }
            if (accepted) {
                sp[i] = make_vec2<Real>(nx, ny);
            } else {
                nx = si.x;
                ny = si.y;
            }
        } else {
            overrelax_step(si.x, si.y, hx, hy, nx, ny);
            sp[i] = make_vec2<Real>(nx, ny);
        }
    }
    if (IS_MET) {
        const unsigned int votes = __ballot_sync(0xffffffffu, accepted);
        if ((threadIdx.x & 31) == 0 && votes)
            atomicAdd(&P.met_acc[d.rep_off + slot], (unsigned long long)__popc(votes));
    }
    if (FUSE) {
        __shared__ double part[kPlainBlock / 32][kObsCount];
        const bool full = measurement_sweep(P.sweep[s], meas_every);
        const int nf = full ? kObsCount : 1;
        Real v[kObsCount];
        v[kObsE] = active ? -(nx * lx + ny * ly) : (Real)0;
        if (full) {
            V4 ph = {0, 0, 0, 0};
            if (active) ph = reinterpret_cast<const V4 *>(P.phase)[d.site_off + i];
            v[kObsMx] = nx;
            v[kObsMy] = ny;
            v[kObsF1xRe] = nx * ph.x; v[kObsF1xIm] = nx * ph.y;
            v[kObsF1yRe] = ny * ph.x; v[kObsF1yIm] = ny * ph.y;
            v[kObsF2xRe] = nx * ph.z; v[kObsF2xIm] = nx * ph.w;
            v[kObsF2yRe] = ny * ph.z; v[kObsF2yIm] = ny * ph.w;
        }
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
        for (int f = 0; f < kObsCount; ++f) {
            if (f >= nf) break;
            const Real w = warp_sum(v[f]);
            if (lane == 0) part[warp][f] = (double)w;
        }
        __syncthreads();
        if ((int)threadIdx.x < nf) {
            double total = 0.0;
#pragma unroll
            for (int w = 0; w < kPlainBlock / 32; ++w) total += part[w][threadIdx.x];
            atomicAdd(&P.obs[(size_t)(d.rep_off + r) * kObsStride + threadIdx.x], total);
        }
    }
}

template <typename Real, bool DISORDER>
cudaError_t sweep_impl(const DevPlan &P, const PlanShape &S, uint32_t ops, int measure_every, cudaStream_t st,
                       int64_t *launches)
{
    // each colour phase gets blocks for the largest class of that colour only
    auto grid = [&](int c) {
        const int sites = c < (int)S.class_max.size() ? S.class_max[c] : S.max_class;
        return dim3((unsigned)std::max(1, (sites + kPlainBlock - 1) / kPlainBlock), S.max_R, S.n_samples);
    };
    const bool met = ops & XYL_OP_MET, orx = ops & XYL_OP_OR;
    const int me = (ops & XYL_OP_MEASURE) ? measure_every : 0;
    int64_t n = 0;
    if (met) {
        for (int c = 0; c < S.max_Q; ++c) {
            if (orx)
                plain_phase_kernel<Real, true, false, DISORDER><<<grid(c), kPlainBlock, 0, st>>>(P, c, me);
            else
                plain_phase_kernel<Real, true, true, DISORDER><<<grid(c), kPlainBlock, 0, st>>>(P, c, me);
            ++n;
        }
    }
    if (orx) {
        for (int c = 0; c < S.max_Q; ++c) {
            plain_phase_kernel<Real, false, true, DISORDER><<<grid(c), kPlainBlock, 0, st>>>(P, c, me);
            ++n;
        }
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = launch_finalize(P, S, ops, measure_every, 1, 0, st);
    ++n;
    if (launches) *launches += n;
    return e;
}

}  // namespace

cudaError_t launch_plain_sweep(const DevPlan &P, const PlanShape &S, uint32_t ops, int measure_every,
                               cudaStream_t st, int64_t *launches)
{
    if (S.dim == 3) return launch_o3_sweep(P, S, ops, measure_every, st, launches);
    if (S.disorder)
        return S.fp64 ? sweep_impl<double, true>(P, S, ops, measure_every, st, launches)
                      : sweep_impl<float, true>(P, S, ops, measure_every, st, launches);
    return S.fp64 ? sweep_impl<double, false>(P, S, ops, measure_every, st, launches)
                  : sweep_impl<float, false>(P, S, ops, measure_every, st, launches);
}

}  // namespace xyl
