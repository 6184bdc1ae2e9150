// O(3) spins on the plain engines (App. B names O(3) among the continuous
// models the method carries over to).  Same Hamiltonian with unit 3-vectors,
// same colour-sequential sweep, parallel tempering and measurements; spins are
// stored replica-major as padded 4-vectors (float4 / double4_32a, w = 0), one
// thread per (site, replica) and one launch per colour phase.
//
// Proposal (the library's reading; the paper fixes no O(3) move): a point
// uniform on the spherical cap of angular radius Delta around S, built in the
// orthonormal frame of Duff et al. (JCGT 6(1), 2017) with its first vector
// times g = sign(z), so that the frame of -S is minus the frame of S and the
// move commutes with the gauge S -> -S bit for bit.  The FP64 steps are a
// fixed sequence of IEEE operations (this file compiles without contraction),
// the same as the oracle's.
#include <cuda_runtime.h>

#include <algorithm>

#include "engines.h"
#include "o3_f32.cuh"

namespace xyl {
namespace {

constexpr int kO3Block = 256;
constexpr int kGather = 4;  // neighbour loads in flight per thread
constexpr uint32_t kMetSecondBlock = 0x800000u;
constexpr double kPi = 3.14159265358979323846;
constexpr double kTwoPi = 6.283185307179586476925286766559;

template <typename Real> struct Vec3T;
template <> struct Vec3T<float> { using type = float4; };
template <> struct Vec3T<double> { using type = double4_32a; };
template <typename Real> using Vec3 = typename Vec3T<Real>::type;

__device__ __forceinline__ float4 make_v3(float x, float y, float z) { return make_float4(x, y, z, 0.0f); }
__device__ __forceinline__ double4_32a make_v3(double x, double y, double z)
{
    double4_32a v;
    v.x = x; v.y = y; v.z = z; v.w = 0.0;
    return v;
}

// Point of the cap around (x, y, z): 1 - cos theta = u * 2 sin^2(Delta / 2),
// azimuth 2 pi uphi - pi in the frame e1 = (g + x^2 a, b, -x),
// e2 = (b, g + y^2 a, -y), a = -1 / (g + z), b = x y a.
__device__ __forceinline__ void cap_propose(const DevPlan &P, double x, double y, double z, double half_width,
                                            double u, double uphi, double &nx, double &ny, double &nz)
{
    double sh, ch;
    sincos_series(P, 0.5 * half_width, &sh, &ch);
    const double w = u * (2.0 * (sh * sh));
    const double ct = 1.0 - w;
    const double st = sqrt(w * (2.0 - w));
    double sp, cp;
    sincos_series(P, kTwoPi * uphi - kPi, &sp, &cp);
    const double g = z >= 0.0 ? 1.0 : -1.0;
    const double a = -1.0 / (g + z);
    const double b = x * y * a;
    const double e1x = g + (x * x) * a, e1y = b, e1z = -x;
    const double e2x = b, e2y = g + (y * y) * a, e2z = -y;
    const double tx = cp * e1x + sp * e2x, ty = cp * e1y + sp * e2y, tz = cp * e1z + sp * e2z;
    nx = ct * x + st * tx;
    ny = ct * y + st * ty;
    nz = ct * z + st * tz;
}

__global__ void o3_init_kernel(DevPlan P, int fp64, int aligned)
{
    const int s = blockIdx.z, r = blockIdx.y;
    const DevSample d = P.samples[s];
    const int site = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= d.R || site >= d.N) return;
    double x = 1.0, y = 0.0, z = 0.0;
    if (!aligned) {
        const Words4 w = philox_draw((uint32_t)P.perm[d.site_off + site], 0u, kPurposeInit, (uint32_t)r,
                                     d.sample_id, P.key);
        const double u = fp64 ? uniform53(w.w0, w.w1) : (double)uniform24(w.w0);
        const double up = fp64 ? uniform53(w.w2, w.w3) : (double)uniform24(w.w1);
        z = 2.0 * u - 1.0;
        const double rho = sqrt((1.0 - z) * (1.0 + z));
        double sn, cs;
        sincos_series(P, kTwoPi * up - kPi, &sn, &cs);
        x = rho * cs;
        y = rho * sn;
    }
    const int64_t at = d.spin_off + (int64_t)r * d.N + site;
    if (fp64)
        reinterpret_cast<double4_32a *>(P.spins)[at] = make_v3(x, y, z);
    else
        reinterpret_cast<float4 *>(P.spins)[at] = make_v3((float)x, (float)y, (float)z);
}

// One colour phase of the Metropolis (IS_MET) or overrelaxation pass for O(3)
// spins; FUSE, DISORDER and the per-block reduction as in the XY plain kernel,
// with the z component's magnetisation and Fourier sums added.
template <typename Real, bool IS_MET, bool FUSE, bool DISORDER>
__global__ void __launch_bounds__(kO3Block) o3_phase_kernel(DevPlan P, int c, int meas_every)
{
    using V = Vec3<Real>;
    using V4 = Vec4<Real>;
    const int s = blockIdx.z, r = blockIdx.y;
    const DevSample d = P.samples[s];
    if (r >= d.R || c >= d.Q) return;
    int cb = P.color_ptr[d.color_off + c], ce = P.color_ptr[d.color_off + c + 1];
    checked_class(P, cb, ce, d.N);
    const int base = cb + (int)blockIdx.x * kO3Block;
    if (base >= ce) return;
    const int i = base + (int)threadIdx.x;
    const bool active = i < ce;
    V *sp = reinterpret_cast<V *>(P.spins) + d.spin_off + (int64_t)r * d.N;
    const int32_t *rp = P.row_ptr + d.row_off;
    const int32_t *cl = P.col + d.col_off;
    const int slot = P.slot_of[d.rep_off + r];

    Real nx = 0, ny = 0, nz = 0, lx = 0, ly = 0, lz = 0;
    bool accepted = false;
    if (active) {
        const V si = sp[i];
        Real hx = 0, hy = 0, hz = 0;
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
                    sj.z = -sj.z;
                }
                hx += sj.x;
                hy += sj.y;
                hz += sj.z;
                if (FUSE && j < cb) {
                    lx += sj.x;
                    ly += sj.y;
                    lz += sj.z;
                }
            }
        }
        if (DISORDER && P.field) {
            // the site's own field after its neighbours; the fused energy takes -h_i . S_i once
            const V4 f = reinterpret_cast<const V4 *>(P.field)[d.site_off + i];
            hx += f.x;
            hy += f.y;
            hz += f.z;
            if (FUSE) {
                lx += f.x;
                ly += f.y;
                lz += f.z;
            }
        }
        if (IS_MET) {
            const uint32_t site = (uint32_t)P.perm[d.site_off + i];
            const uint32_t t = P.sweep[s];
            const double beta = P.beta[d.rep_off + slot], half_width = P.delta[d.rep_off + slot];
            if constexpr (sizeof(Real) == 8) {
                const Words4 a = philox_draw(site, t, kPurposeMet, (uint32_t)r, d.sample_id, P.key);
                const Words4 b = philox_draw(site, t, kPurposeMet, kMetSecondBlock | (uint32_t)r, d.sample_id, P.key);
                cap_propose(P, si.x, si.y, si.z, half_width, uniform53(a.w0, a.w1), uniform53(b.w0, b.w1), nx, ny,
                            nz);
                const double dE = -((nx - si.x) * hx + (ny - si.y) * hy + (nz - si.z) * hz);
                accepted = dE <= 0.0 || uniform53(a.w2, a.w3) < exp(-beta * dE);
            } else {
                // the single-precision steps of o3_f32.cuh (hardware sincos/exp, proposal renormalised)
                const Words4 a = philox_draw(site, t, kPurposeMet, (uint32_t)r, d.sample_id, P.key);
                o3_cap_propose_f32(si.x, si.y, si.z, (float)half_width, uniform24(a.w0), uniform24(a.w1), nx, ny, nz);
                accepted = o3_accept_f32(si.x, si.y, si.z, nx, ny, nz, hx, hy, hz, (float)beta, uniform24(a.w2));
            }
            if (accepted) {
                sp[i] = make_v3(nx, ny, nz);
            } else {
                nx = si.x;
                ny = si.y;
                nz = si.z;
            }
        } else {
            if constexpr (sizeof(Real) == 4) {
                o3_reflect_f32(si.x, si.y, si.z, hx, hy, hz, nx, ny, nz);
            } else {
                const Real h2 = hx * hx + hy * hy + hz * hz;
                if (h2 > (Real)0) {
                    const Real k = (Real)2 * (si.x * hx + si.y * hy + si.z * hz) / h2;
                    nx = k * hx - si.x;
                    ny = k * hy - si.y;
                    nz = k * hz - si.z;
                } else {
                    nx = si.x;
                    ny = si.y;
                    nz = si.z;
                }
            }
            sp[i] = make_v3(nx, ny, nz);
        }
    }
    if (IS_MET) {
        const unsigned int votes = __ballot_sync(0xffffffffu, accepted);
        if ((threadIdx.x & 31) == 0 && votes)
            atomicAdd(&P.met_acc[d.rep_off + slot], (unsigned long long)__popc(votes));
    }
    if (FUSE) {
        __shared__ double part[kO3Block / 32][kObsCount3];
        const bool full = measurement_sweep(P.sweep[s], meas_every);
        const int nf = full ? kObsCount3 : 1;
        Real v[kObsCount3];
        v[kObsE] = active ? -(nx * lx + ny * ly + nz * lz) : (Real)0;
        if (full) {
            V4 ph = {0, 0, 0, 0};
            if (active) ph = reinterpret_cast<const V4 *>(P.phase)[d.site_off + i];
            v[kObsMx] = nx;
            v[kObsMy] = ny;
            v[kObsMz] = nz;
            v[kObsF1xRe] = nx * ph.x; v[kObsF1xIm] = nx * ph.y;
            v[kObsF1yRe] = ny * ph.x; v[kObsF1yIm] = ny * ph.y;
            v[kObsF1zRe] = nz * ph.x; v[kObsF1zIm] = nz * ph.y;
            v[kObsF2xRe] = nx * ph.z; v[kObsF2xIm] = nx * ph.w;
            v[kObsF2yRe] = ny * ph.z; v[kObsF2yIm] = ny * ph.w;
            v[kObsF2zRe] = nz * ph.z; v[kObsF2zIm] = nz * ph.w;
        }
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
        for (int f = 0; f < kObsCount3; ++f) {
            if (f >= nf) break;
            const Real w = warp_sum(v[f]);
            if (lane == 0) part[warp][f] = (double)w;
        }
        __syncthreads();
        if ((int)threadIdx.x < nf) {
            double total = 0.0;
#pragma unroll
            for (int w = 0; w < kO3Block / 32; ++w) total += part[w][threadIdx.x];
            atomicAdd(&P.obs[(size_t)(d.rep_off + r) * kObsStride + threadIdx.x], total);
        }
    }
}

template <typename T>
__device__ __forceinline__ T block_sum(T v, T *scratch)
{
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) scratch[warp] = v;
    __syncthreads();
    T total = 0;
    if (warp == 0) {
        total = (lane < (int)(blockDim.x >> 5)) ? scratch[lane] : (T)0;
        total = warp_sum(total);
    }
    return total;  // valid in thread 0
}

// One block per (sample, replica): optional renormalisation, then the FP64
// energy (each link once, from its higher colour-sorted endpoint),
// magnetisation and Fourier sums of all three components into obs[buffer].
__global__ void o3_recompute_kernel(DevPlan P, int fp64, int renormalise, int buffer_mode)
{
    __shared__ double scratch[32];
    const int s = blockIdx.y, r = blockIdx.x;
    const DevSample d = P.samples[s];
    if (r >= d.R) return;
    const int64_t off = d.spin_off + (int64_t)r * d.N;
    auto load = [&](int i, double &x, double &y, double &z) {
        if (fp64) {
            const double4_32a v = reinterpret_cast<const double4_32a *>(P.spins)[off + i];
            x = v.x; y = v.y; z = v.z;
        } else {
            const float4 v = reinterpret_cast<const float4 *>(P.spins)[off + i];
            x = v.x; y = v.y; z = v.z;
        }
    };
    if (renormalise) {
        for (int i = threadIdx.x; i < d.N; i += blockDim.x) {
            double x, y, z;
            load(i, x, y, z);
            const double n = sqrt(x * x + y * y + z * z);
            if (n <= 0.0) continue;
            if (fp64)
                reinterpret_cast<double4_32a *>(P.spins)[off + i] = make_v3(x / n, y / n, z / n);
            else
                reinterpret_cast<float4 *>(P.spins)[off + i] = make_v3((float)(x / n), (float)(y / n), (float)(z / n));
        }
        __syncthreads();
    }
    double acc[kObsCount3];
#pragma unroll
    for (int f = 0; f < kObsCount3; ++f) acc[f] = 0.0;
    for (int i = threadIdx.x; i < d.N; i += blockDim.x) {
        double sx, sy, sz;
        load(i, sx, sy, sz);
        double4_32a ph;
        if (fp64) {
            ph = reinterpret_cast<const double4_32a *>(P.phase)[d.site_off + i];
        } else {
            const float4 p = reinterpret_cast<const float4 *>(P.phase)[d.site_off + i];
            ph.x = p.x; ph.y = p.y; ph.z = p.z; ph.w = p.w;
        }
        double lx = 0.0, ly = 0.0, lz = 0.0;
        const int rb = P.row_ptr[d.row_off + i];
        const int re = rb + checked_id(P, P.row_ptr[d.row_off + i + 1] - rb, d.max_deg + 1, 0);
        for (int k = rb; k < re; ++k) {
            // a neighbour id with its top bit set is a link with J = -1
            const int raw = P.col[d.col_off + k];
            const int j = checked_id(P, raw & 0x7fffffff, d.N, 0);
            if (j >= i) continue;
            double vx, vy, vz;
            load(j, vx, vy, vz);
            if (raw < 0) { vx = -vx; vy = -vy; vz = -vz; }
            lx += vx; ly += vy; lz += vz;
        }
        if (P.field) {
            // random fields: -h_i . S_i once per site
            if (fp64) {
                const double4_32a f = reinterpret_cast<const double4_32a *>(P.field)[d.site_off + i];
                lx += f.x; ly += f.y; lz += f.z;
            } else {
                const float4 f = reinterpret_cast<const float4 *>(P.field)[d.site_off + i];
                lx += f.x; ly += f.y; lz += f.z;
            }
        }
        acc[kObsE] -= sx * lx + sy * ly + sz * lz;
        acc[kObsMx] += sx;
        acc[kObsMy] += sy;
        acc[kObsMz] += sz;
        acc[kObsF1xRe] += sx * ph.x; acc[kObsF1xIm] += sx * ph.y;
        acc[kObsF1yRe] += sy * ph.x; acc[kObsF1yIm] += sy * ph.y;
        acc[kObsF1zRe] += sz * ph.x; acc[kObsF1zIm] += sz * ph.y;
        acc[kObsF2xRe] += sx * ph.z; acc[kObsF2xIm] += sx * ph.w;
        acc[kObsF2yRe] += sy * ph.z; acc[kObsF2yIm] += sy * ph.w;
        acc[kObsF2zRe] += sz * ph.z; acc[kObsF2zIm] += sz * ph.w;
    }
    const uint32_t t = P.sweep[s];
    const int buf = buffer_mode ? (int)(t & 1u) : 0;
    double *o = P.obs + ((size_t)buf * P.total_R + d.rep_off + r) * kObsStride;
    for (int f = 0; f < kObsCount3; ++f) {
        const double v = block_sum(acc[f], scratch);
        if (threadIdx.x == 0) o[f] = v;
    }
    if (threadIdx.x == 0) {
        const double E = o[kObsE];
        const double diff = fabs(E - P.last_E[d.rep_off + r]);
        atomicMax(reinterpret_cast<unsigned long long *>(P.drift), (unsigned long long)__double_as_longlong(diff));
        P.last_E[d.rep_off + r] = E;
    }
}

template <typename Real, bool DISORDER>
cudaError_t o3_sweep_impl(const DevPlan &P, const PlanShape &S, uint32_t ops, int measure_every, cudaStream_t st,
                          int64_t *launches)
{
    // each colour phase gets blocks for the largest class of that colour only
    auto grid = [&](int c) {
        const int sites = c < (int)S.class_max.size() ? S.class_max[c] : S.max_class;
        return dim3((unsigned)std::max(1, (sites + kO3Block - 1) / kO3Block), S.max_R, S.n_samples);
    };
    const bool met = ops & XYL_OP_MET, orx = ops & XYL_OP_OR;
    const int me = (ops & XYL_OP_MEASURE) ? measure_every : 0;
    int64_t n = 0;
    if (met) {
        for (int c = 0; c < S.max_Q; ++c) {
            if (orx)
                o3_phase_kernel<Real, true, false, DISORDER><<<grid(c), kO3Block, 0, st>>>(P, c, me);
            else
                o3_phase_kernel<Real, true, true, DISORDER><<<grid(c), kO3Block, 0, st>>>(P, c, me);
            ++n;
        }
    }
    if (orx) {
        for (int c = 0; c < S.max_Q; ++c) {
            o3_phase_kernel<Real, false, true, DISORDER><<<grid(c), kO3Block, 0, st>>>(P, c, me);
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

cudaError_t launch_o3_init(const DevPlan &P, const PlanShape &S, int aligned, cudaStream_t st)
{
    dim3 grid((S.max_N + 255) / 256, S.max_R, S.n_samples);
    o3_init_kernel<<<grid, 256, 0, st>>>(P, S.fp64 ? 1 : 0, aligned);
    return cudaGetLastError();
}

cudaError_t launch_o3_sweep(const DevPlan &P, const PlanShape &S, uint32_t ops, int measure_every, cudaStream_t st,
                            int64_t *launches)
{
    if (S.coupled)
        return S.fp64 ? o3_sweep_impl<double, true>(P, S, ops, measure_every, st, launches)
                      : o3_sweep_impl<float, true>(P, S, ops, measure_every, st, launches);
    return S.fp64 ? o3_sweep_impl<double, false>(P, S, ops, measure_every, st, launches)
                  : o3_sweep_impl<float, false>(P, S, ops, measure_every, st, launches);
}

cudaError_t launch_o3_recompute(const DevPlan &P, const PlanShape &S, int renormalise, int buffer_mode,
                                cudaStream_t st)
{
    dim3 grid(S.max_R, S.n_samples);
    o3_recompute_kernel<<<grid, 256, 0, st>>>(P, S.fp64 ? 1 : 0, renormalise, buffer_mode);
    return cudaGetLastError();
}

}  // namespace xyl
