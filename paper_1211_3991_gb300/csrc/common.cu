// Kernels shared by every engine: spin initialisation, the end-of-sweep step
// (parallel tempering, measurement, counters) and the FP64 recomputation of
// each replica's energy and observables.
#include <cuda_runtime.h>

#include "engines.h"

namespace xyl {
namespace {

constexpr double kTwoPi = 6.283185307179586476925286766559;

__device__ __forceinline__ int64_t spin_index(const DevSample &d, int layout, int site, int r)
{
    return layout == kInterleaved ? d.spin_off + (int64_t)site * d.R + r : d.spin_off + (int64_t)r * d.N + site;
}

// theta = 2 pi u - pi from the INIT stream of (original site id, replica, sample).
__global__ void init_kernel(DevPlan P, int layout, int fp64, int aligned)
{
    const int s = blockIdx.z, r = blockIdx.y;
    const DevSample d = P.samples[s];
    const int site = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= d.R || site >= d.N) return;
    double cs = 1.0, sn = 0.0;
    if (!aligned) {
        const Words4 x = philox_draw((uint32_t)P.perm[d.site_off + site], 0u, kPurposeInit, (uint32_t)r,
                                     d.sample_id, P.key);
        const double u = fp64 ? uniform53(x.w0, x.w1) : (double)uniform24(x.w0);
        const double theta = kTwoPi * u - 3.14159265358979323846;
        if (fp64)
            sincos_series(P, theta, &sn, &cs);
        else
            sincos(theta, &sn, &cs);
    }
    const int64_t at = spin_index(d, layout, site, r);
    if (fp64)
        reinterpret_cast<double2 *>(P.spins)[at] = make_double2(cs, sn);
    else
        reinterpret_cast<float2 *>(P.spins)[at] = make_float2((float)cs, (float)sn);
}

// Identity labels, zero counters.
__global__ void reset_labels_kernel(DevPlan P)
{
    const int s = blockIdx.x;
    const DevSample d = P.samples[s];
    for (int k = threadIdx.x; k < d.R; k += blockDim.x) {
        P.slot_of[d.rep_off + k] = k;
        P.rep_at[d.rep_off + k] = k;
    }
    if (threadIdx.x == 0) P.sweep[s] = 0;
}

// One block per sample.  Reads the per-replica sums of the finished sweep from
// obs[buffer], attempts the PT swaps of pairs (k, k+1), k = t mod 2 (App. B:
// accept iff u < exp((beta_k - beta_k+1)(E_k - E_k+1)), FP64), adds one
// measurement per slot when due, updates the counters and clears the buffer.
__global__ void finalize_kernel(DevPlan P, uint32_t ops, int measure_every, int advance, int buffer_mode, int dim)
{
    extern __shared__ double sh[];
    const int s = blockIdx.x;
    const DevSample d = P.samples[s];
    const int R = d.R;
    double *E = sh;
    int *rep_at = reinterpret_cast<int *>(E + R);
    const uint32_t t = P.sweep[s];
    const int buf = buffer_mode ? (int)(t & 1u) : 0;
    double *obs = P.obs + ((size_t)buf * P.total_R + d.rep_off) * kObsStride;
    for (int k = threadIdx.x; k < R; k += blockDim.x) {
        E[k] = obs[(size_t)k * kObsStride + kObsE];
        rep_at[k] = P.rep_at[d.rep_off + k];
    }
    __syncthreads();
    if (ops & XYL_OP_PT) {
        for (int p = threadIdx.x; 2 * p + (int)(t & 1u) + 1 < R; p += blockDim.x) {
            const int k = 2 * p + (int)(t & 1u);
            const int a = rep_at[k], b = rep_at[k + 1];
            const double x = (P.beta[d.rep_off + k] - P.beta[d.rep_off + k + 1]) * (E[a] - E[b]);
            const Words4 w = philox_draw((uint32_t)k, t, kPurposePt, 0u, d.sample_id, P.key);
            const bool accept = uniform53(w.w0, w.w1) < exp(x);
            P.pt_try[d.rep_off + k] += 1ull;
            if (accept) {
                rep_at[k] = b;
                rep_at[k + 1] = a;
                P.pt_acc[d.rep_off + k] += 1ull;
            }
        }
        __syncthreads();
    }
    const bool measure = (ops & XYL_OP_MEASURE) && measure_every > 0 && ((t + 1u) % (uint32_t)measure_every) == 0u;
    const double invN = 1.0 / (double)d.N;
    for (int k = threadIdx.x; k < R; k += blockDim.x) {
        const int r = rep_at[k];
        P.rep_at[d.rep_off + k] = r;
        P.slot_of[d.rep_off + r] = k;
        if (ops & XYL_OP_MET) P.met_try[d.rep_off + k] += (unsigned long long)d.N;
        if (measure) {
            const double *o = obs + (size_t)r * kObsStride;
            const double e = o[kObsE] * invN;
            const double mx = o[kObsMx] * invN, my = o[kObsMy] * invN;
            double m2 = mx * mx + my * my;
            double f1 = o[kObsF1xRe] * o[kObsF1xRe] + o[kObsF1xIm] * o[kObsF1xIm] +
                        o[kObsF1yRe] * o[kObsF1yRe] + o[kObsF1yIm] * o[kObsF1yIm];
            double f2 = o[kObsF2xRe] * o[kObsF2xRe] + o[kObsF2xIm] * o[kObsF2xIm] +
                        o[kObsF2yRe] * o[kObsF2yRe] + o[kObsF2yIm] * o[kObsF2yIm];
            const double mz = dim == 3 ? o[kObsMz] * invN : 0.0;
            if (dim == 3) {
                // O(3) spins: the third component joins m^2 and |F(k)|^2
                m2 += mz * mz;
                f1 += o[kObsF1zRe] * o[kObsF1zRe] + o[kObsF1zIm] * o[kObsF1zIm];
                f2 += o[kObsF2zRe] * o[kObsF2zRe] + o[kObsF2zIm] * o[kObsF2zIm];
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
            a[XYL_ACC_MZ] += mz;
        }
    }
    __syncthreads();
    for (int k = threadIdx.x; k < R; k += blockDim.x) P.last_E[d.rep_off + k] = E[k];
    for (int q = threadIdx.x; q < R * kObsStride; q += blockDim.x) obs[q] = 0.0;
    if (advance && threadIdx.x == 0) P.sweep[s] = t + 1u;
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

// One block per (sample, replica): optional renormalisation |s| = 1, then the
// FP64 energy (each link once, from its higher colour-sorted endpoint),
// magnetisation and Fourier sums written to obs[buffer]; records the drift
// against the energy the last sweep produced.
__global__ void recompute_kernel(DevPlan P, int layout, int fp64, int renormalise, int buffer_mode)
{
    __shared__ double scratch[32];
    const int s = blockIdx.y, r = blockIdx.x;
    const DevSample d = P.samples[s];
    if (r >= d.R) return;
    if (renormalise && !fp64) {
        float2 *sp = reinterpret_cast<float2 *>(P.spins);
        for (int i = threadIdx.x; i < d.N; i += blockDim.x) {
            const int64_t at = spin_index(d, layout, i, r);
            const float2 v = sp[at];
            const double n = sqrt((double)v.x * v.x + (double)v.y * v.y);
            if (n > 0.0) sp[at] = make_float2((float)(v.x / n), (float)(v.y / n));
        }
        __syncthreads();
    } else if (renormalise) {
        double2 *sp = reinterpret_cast<double2 *>(P.spins);
        for (int i = threadIdx.x; i < d.N; i += blockDim.x) {
            const int64_t at = spin_index(d, layout, i, r);
            const double2 v = sp[at];
            const double n = sqrt(v.x * v.x + v.y * v.y);
            if (n > 0.0) sp[at] = make_double2(v.x / n, v.y / n);
        }
        __syncthreads();
    }
    double acc[kObsCount];
#pragma unroll
    for (int f = 0; f < kObsCount; ++f) acc[f] = 0.0;
    for (int i = threadIdx.x; i < d.N; i += blockDim.x) {
        double sx, sy;
        double4_32a ph;
        if (fp64) {
            const double2 v = reinterpret_cast<const double2 *>(P.spins)[spin_index(d, layout, i, r)];
            sx = v.x; sy = v.y;
            ph = reinterpret_cast<const double4_32a *>(P.phase)[d.site_off + i];
        } else {
            const float2 v = reinterpret_cast<const float2 *>(P.spins)[spin_index(d, layout, i, r)];
            sx = v.x; sy = v.y;
            const float4 p = reinterpret_cast<const float4 *>(P.phase)[d.site_off + i];
            ph = make_double4_32a(p.x, p.y, p.z, p.w);
        }
        double lx = 0.0, ly = 0.0;
        const int rb = P.row_ptr[d.row_off + i];
        const int re = rb + checked_id(P, P.row_ptr[d.row_off + i + 1] - rb, d.max_deg + 1, 0);
        for (int k = rb; k < re; ++k) {
            // a neighbour id with its top bit set is a link with J = -1 (random bonds)
            const int raw = P.col[d.col_off + k];
            const int j = checked_id(P, raw & 0x7fffffff, d.N, 0);
            if (j >= i) continue;
            double vx, vy;
            if (fp64) {
                const double2 v = reinterpret_cast<const double2 *>(P.spins)[spin_index(d, layout, j, r)];
                vx = v.x; vy = v.y;
            } else {
                const float2 v = reinterpret_cast<const float2 *>(P.spins)[spin_index(d, layout, j, r)];
                vx = v.x; vy = v.y;
            }
            if (raw < 0) { vx = -vx; vy = -vy; }
            lx += vx; ly += vy;
        }
        if (P.field) {
            // random fields: -h_i . S_i once per site
            if (fp64) {
                const double2 f = reinterpret_cast<const double2 *>(P.field)[d.site_off + i];
                lx += f.x; ly += f.y;
            } else {
                const float2 f = reinterpret_cast<const float2 *>(P.field)[d.site_off + i];
                lx += f.x; ly += f.y;
            }
        }
        acc[kObsE] -= sx * lx + sy * ly;
        acc[kObsMx] += sx;
        acc[kObsMy] += sy;
        acc[kObsF1xRe] += sx * ph.x; acc[kObsF1xIm] += sx * ph.y;
        acc[kObsF1yRe] += sy * ph.x; acc[kObsF1yIm] += sy * ph.y;
        acc[kObsF2xRe] += sx * ph.z; acc[kObsF2xIm] += sx * ph.w;
        acc[kObsF2yRe] += sy * ph.z; acc[kObsF2yIm] += sy * ph.w;
    }
    const uint32_t t = P.sweep[s];
    const int buf = buffer_mode ? (int)(t & 1u) : 0;
    double *o = P.obs + ((size_t)buf * P.total_R + d.rep_off + r) * kObsStride;
    for (int f = 0; f < kObsCount; ++f) {
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

// One block per sample: checks the device CSR the sweeps read.  Every
// colour class must be an independent set (App. B "Graph coloring": sites of
// one colour update together only because no link joins two of them), every
// neighbour id must lie in [0, N) and differ from the site, each row must be
// ascending, and every link must appear in both rows.  Violations are counted.
__global__ void check_kernel(DevPlan P, unsigned long long *violations)
{
    const int s = blockIdx.x;
    const DevSample d = P.samples[s];
    const int32_t *rp = P.row_ptr + d.row_off;
    const int32_t *cl = P.col + d.col_off;
    const int32_t *cp = P.color_ptr + d.color_off;
    unsigned long long bad = 0;
    for (int i = threadIdx.x; i < d.N; i += blockDim.x) {
        int c = 0;
        while (c + 1 < d.Q && cp[c + 1] <= i) ++c;
        const int cb = cp[c], ce = cp[c + 1];
        const int rb = rp[i], re = rp[i + 1];
        if (rb > re) { ++bad; continue; }
        int prev = -1;
        for (int k = rb; k < re; ++k) {
            const int j = cl[k] & 0x7fffffff;  // the top bit carries a coupling J = -1
            if (j < 0 || j >= d.N || j == i) { ++bad; continue; }
            if (j >= cb && j < ce) ++bad;      // a link inside a colour class
            if (j <= prev) ++bad;              // rows ascending, no repeated link
            prev = j;
            bool back = false;
            for (int q = rp[j]; q < rp[j + 1] && !back; ++q) back = (cl[q] & 0x7fffffff) == i;
            if (!back) ++bad;                  // the link must appear in row j too
        }
    }
    if (bad) atomicAdd(violations, bad);
}

}  // namespace

cudaError_t launch_check(const DevPlan &P, const PlanShape &S, unsigned long long *violations, cudaStream_t st)
{
    check_kernel<<<S.n_samples, 256, 0, st>>>(P, violations);
    return cudaGetLastError();
}

cudaError_t launch_init(const DevPlan &P, const PlanShape &S, int aligned, cudaStream_t st)
{
    dim3 grid((S.max_N + 255) / 256, S.max_R, S.n_samples);
    if (S.dim == 3) {
        const cudaError_t e = launch_o3_init(P, S, aligned, st);
        if (e != cudaSuccess) return e;
    } else {
        init_kernel<<<grid, 256, 0, st>>>(P, S.layout, S.fp64 ? 1 : 0, aligned);
    }
    reset_labels_kernel<<<S.n_samples, 128, 0, st>>>(P);
    return cudaGetLastError();
}

cudaError_t launch_finalize(const DevPlan &P, const PlanShape &S, uint32_t ops, int measure_every, int advance,
                            int buffer_mode, cudaStream_t st)
{
    const size_t smem = (size_t)S.max_R * (sizeof(double) + sizeof(int));
    finalize_kernel<<<S.n_samples, 128, smem, st>>>(P, ops, measure_every, advance, buffer_mode, S.dim);
    return cudaGetLastError();
}

cudaError_t launch_recompute(const DevPlan &P, const PlanShape &S, int renormalise, int buffer_mode, cudaStream_t st)
{
    if (S.dim == 3) return launch_o3_recompute(P, S, renormalise, buffer_mode, st);
    dim3 grid(S.max_R, S.n_samples);
    recompute_kernel<<<grid, 256, 0, st>>>(P, S.layout, S.fp64 ? 1 : 0, renormalise, buffer_mode);
    return cudaGetLastError();
}

}  // namespace xyl
