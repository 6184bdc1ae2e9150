// Resident FP32 engine for O(3) spins (App. B names O(3) among the continuous
// models the method carries over to): the batched sampler with three-component
// spins held in shared memory for the whole launch.
//
// Work decomposition.  The replicas of a sample are split into groups of Rg
// (a power of two); one CTA owns a group and keeps its spins of every site in
// shared memory as three single-precision component arrays, [site][replica]
// each (12 bytes a site and replica), plus one zero row that padded CSR
// entries point at.  One thread updates one (site, replica): with a block
// size that is a multiple of Rg a thread keeps its replica for the whole
// launch.  Colour phases are separated by __syncthreads.  A cluster holds the
// groups of a sample when they are at most 16, and they meet once per sweep
// at a cluster barrier; otherwise every group is a cluster of its own and the
// groups of a sample meet at a bounded global barrier.  Then every CTA reads
// the sample's replica energies and takes the same parallel-tempering
// decisions; the first CTA of the first group records the measurement.
//
// The per-spin arithmetic is that of the plain engine (o3_f32.cuh, the same
// Philox block per replica, neighbour sums in row order), so both give
// bit-identical spins from the same state.  Spins live replica-major in
// global memory (padded float4), read at launch start and written back at the
// end.  CSR rows of up to eight neighbours (16-bit ids) and the random-stream
// site ids are staged beside the spins when they fit, else read from global
// memory one item ahead.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include "engines.h"
#include "o3_f32.cuh"
#include "sweep_tail.cuh"

namespace cg = cooperative_groups;

namespace xyl {
namespace {

constexpr int kO3Sums = kObsCount3;
constexpr unsigned int kO3BarrierPolls = 1u << 21;  // about a second of polling

struct O3Params {
    const int2 *units;   // (sample, group), sample-major
    int unit_begin;
    int gpc;             // replica groups per cluster
    int Rg, log2rg;
    int n_sweeps;
    uint32_t ops;
    int measure_every;
    int n_warps;
    int comp;            // floats in each spin component array ((N + 1) * Rg, padded)
    int off_part, off_met, off_beta, off_ids, off_col;  // dynamic shared memory (bytes)
    int csr_w;           // staged row width (6 or 8), 0 = rows read from global memory
    int ids;             // random-stream site ids staged as 16-bit values
};

struct O3Shared {
    double E[kMaxReplicas];
    float beta[kMaxReplicas];
    float delta[kMaxReplicas];
    int slot_of[kMaxReplicas];
    int rep_at[kMaxReplicas];
    int cls_cb[kMaxColorsBatched + 1];
    int abort_flag;
};

template <int DEG>
struct O3Row {
    int nb[DEG > 0 ? DEG : 8];  // missing entries of a shorter row point at the zero row N
    int rb, deg;                 // DEG = 0: the row's place in the global CSR
    uint32_t key;
    uint32_t neg;                // random bonds: bit k set for a link with J = -1
};

template <int DEG, bool IS_MET, bool DISORDER>
__device__ __forceinline__ void o3_fetch_row(const DevPlan &P, const DevSample &d, const O3Params &op,
                                             const uint16_t *col, const uint16_t *ids, int i, O3Row<DEG> &row)
{
    constexpr int W = DEG > 0 ? DEG : 8;
    row.neg = 0u;
    if constexpr (DEG == 0) {
        row.rb = __ldg(P.row_ptr + d.row_off + i);
        row.deg = checked_id(P, __ldg(P.row_ptr + d.row_off + i + 1) - row.rb, d.max_deg + 1, 0);
    } else if (col) {
        const uint32_t *c = reinterpret_cast<const uint32_t *>(col + (size_t)i * W);
#pragma unroll
        for (int k = 0; k < W / 2; ++k) {
            const uint32_t w = c[k];
            if (DISORDER) {
                row.nb[2 * k] = (int)(w & 0x7fffu);
                row.nb[2 * k + 1] = (int)((w >> 16) & 0x7fffu);
                row.neg |= ((w >> 15) & 1u) << (2 * k) | ((w >> 31) & 1u) << (2 * k + 1);
            } else {
                row.nb[2 * k] = (int)(w & 0xffffu);
                row.nb[2 * k + 1] = (int)(w >> 16);
            }
        }
    } else {
        const int32_t *cl = P.col + d.col_off;
        int rb, deg;
        if (DEG > 0) {
            rb = i * DEG;
            deg = DEG;
        } else {
            rb = __ldg(P.row_ptr + d.row_off + i);
            deg = __ldg(P.row_ptr + d.row_off + i + 1) - rb;
        }
#pragma unroll
        for (int k = 0; k < W; ++k) row.nb[k] = (DEG > 0 || k < deg) ? __ldg(cl + rb + k) : d.N;
        if (DISORDER) {
#pragma unroll
            for (int k = 0; k < W; ++k) {
                row.neg |= (row.nb[k] < 0 ? 1u : 0u) << k;
                row.nb[k] &= 0x7fffffff;
            }
        }
    }
    if (IS_MET) row.key = ids ? (uint32_t)ids[i] : (uint32_t)__ldg(P.perm + d.site_off + i);
}

// One colour phase over class c for this thread's replica: sx, sy, sz are the
// component arrays offset by the thread's replica lane.
template <bool IS_MET, bool FUSE_E, int DEG, bool DISORDER>
__device__ __forceinline__ void o3_phase(const DevPlan &P, const DevSample &d, const O3Shared &sh, const O3Params &op,
                                         const uint16_t *col, const uint16_t *ids, float *sx, float *sy, float *sz,
                                         int c, uint32_t t, int r, float beta, float half_width, float &e,
                                         unsigned &acc)
{
    constexpr int W = DEG > 0 ? DEG : 8;
    const int cb = sh.cls_cb[c];
    const int items = (sh.cls_cb[c + 1] - cb) << op.log2rg;
    const int Rg = op.Rg;
    int q = threadIdx.x;
    if (q >= items) return;
    O3Row<DEG> cur;
    o3_fetch_row<DEG, IS_MET, DISORDER>(P, d, op, col, ids, cb + (q >> op.log2rg), cur);
    for (; q < items; q += blockDim.x) {
        const int i = cb + (q >> op.log2rg);
        O3Row<DEG> nxt;
        const int qn = q + (int)blockDim.x;
        if (qn < items) o3_fetch_row<DEG, IS_MET, DISORDER>(P, d, op, col, ids, cb + (qn >> op.log2rg), nxt);
        const float x = sx[i * Rg], y = sy[i * Rg], z = sz[i * Rg];
        float hx = 0.f, hy = 0.f, hz = 0.f, lx = 0.f, ly = 0.f, lz = 0.f;
        auto add = [&](int j_raw, bool neg) {
            const int j = checked_id(P, j_raw, d.N + 1, d.N);  // N: the zero row
            float vx = sx[j * Rg], vy = sy[j * Rg], vz = sz[j * Rg];
            if (DISORDER && neg) {
                vx = -vx;
                vy = -vy;
                vz = -vz;
            }
            hx = __fadd_rn(hx, vx);
            hy = __fadd_rn(hy, vy);
            hz = __fadd_rn(hz, vz);
            if (FUSE_E && j < cb) {
                lx += vx;
                ly += vy;
                lz += vz;
            }
        };
        if constexpr (DEG == 0) {
            const int32_t *cl = P.col + d.col_off + cur.rb;
            for (int k = 0; k < cur.deg; ++k) {
                const int raw = __ldg(cl + k);
                add(DISORDER ? (raw & 0x7fffffff) : raw, DISORDER && raw < 0);
            }
        } else {
#pragma unroll
            for (int k = 0; k < W; ++k) add(cur.nb[k], DISORDER && ((cur.neg >> k) & 1u));
        }
        if (DISORDER && P.field) {
            // the site's own field after its neighbours; the fused energy takes -h_i . S_i once
            const float4 f = __ldg(reinterpret_cast<const float4 *>(P.field) + d.site_off + i);
            hx = __fadd_rn(hx, f.x);
            hy = __fadd_rn(hy, f.y);
            hz = __fadd_rn(hz, f.z);
            if (FUSE_E) {
                lx += f.x;
                ly += f.y;
                lz += f.z;
            }
        }
        float nx, ny, nz;
        if (IS_MET) {
            const Words4 w = philox_draw(cur.key, t, kPurposeMet, (uint32_t)r, d.sample_id, P.key);
            o3_cap_propose_f32(x, y, z, half_width, uniform24(w.w0), uniform24(w.w1), nx, ny, nz);
            const bool ok = o3_accept_f32(x, y, z, nx, ny, nz, hx, hy, hz, beta, uniform24(w.w2));
            acc += ok ? 1u : 0u;
            if (ok) {
                sx[i * Rg] = nx;
                sy[i * Rg] = ny;
                sz[i * Rg] = nz;
            } else {
                nx = x;
                ny = y;
                nz = z;
            }
        } else {
            o3_reflect_f32(x, y, z, hx, hy, hz, nx, ny, nz);
            sx[i * Rg] = nx;
            sy[i * Rg] = ny;
            sz[i * Rg] = nz;
        }
        if (FUSE_E) e -= nx * lx + ny * ly + nz * lz;
        cur = nxt;
    }
}

// Sum over the lanes of a warp that hold the same replica (lanes l and l ^ o, o >= Rg).
__device__ __forceinline__ float o3_warp_reduce(const O3Params &op, float x)
{
    for (int o = 16; o >= op.Rg; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

__device__ __forceinline__ unsigned o3_warp_reduce(const O3Params &op, unsigned x)
{
    for (int o = 16; o >= op.Rg; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

template <int DEG, bool DISORDER>
__device__ __forceinline__ void o3_body(const DevPlan &P, const O3Params &op)
{
    __shared__ O3Shared sh;
    extern __shared__ __align__(16) unsigned char dyn[];
    cg::cluster_group cluster = cg::this_cluster();
    const int rank = (int)cluster.block_rank();
    const int unit = op.unit_begin + (int)blockIdx.x;
    const int2 ug = op.units[unit];
    const int s = ug.x, group = ug.y;
    const DevSample d = P.samples[s];
    const int R = d.R, Rg = op.Rg, N = d.N;
    const int n_groups = R / Rg;
    const bool global_barrier = op.gpc < n_groups;
    const bool leader = group == 0;
    const int rl = (int)(threadIdx.x & (unsigned)(Rg - 1));
    const int r = group * Rg + rl;
    const int warp = (int)(threadIdx.x >> 5), lane = (int)(threadIdx.x & 31u);
    const bool owner_lane = lane < Rg;

    double *beta64 = reinterpret_cast<double *>(dyn + op.off_beta);
    for (int k = threadIdx.x; k < R; k += blockDim.x) {
        sh.slot_of[k] = P.slot_of[d.rep_off + k];
        sh.rep_at[k] = P.rep_at[d.rep_off + k];
        sh.beta[k] = (float)P.beta[d.rep_off + k];
        sh.delta[k] = (float)P.delta[d.rep_off + k];
        beta64[k] = P.beta[d.rep_off + k];
    }
    for (int c = threadIdx.x; c <= d.Q; c += blockDim.x)
        sh.cls_cb[c] = checked_id(P, P.color_ptr[d.color_off + c], d.N + 1, 0);
    if (threadIdx.x == 0) sh.abort_flag = 0;
    // spins of the group (replica-major float4 in global memory), then the zero row
    float *xs = reinterpret_cast<float *>(dyn);
    float *ys = xs + op.comp;
    float *zs = ys + op.comp;
    const float4 *gsp = reinterpret_cast<const float4 *>(P.spins) + d.spin_off;
    for (int k = threadIdx.x; k < N * Rg; k += blockDim.x) {
        const int i = k >> op.log2rg, q = k & (Rg - 1);
        const float4 v = __ldcg(gsp + (int64_t)(group * Rg + q) * N + i);
        xs[k] = v.x;
        ys[k] = v.y;
        zs[k] = v.z;
    }
    for (int k = threadIdx.x; k < Rg; k += blockDim.x) xs[N * Rg + k] = ys[N * Rg + k] = zs[N * Rg + k] = 0.f;
    uint16_t *ids = op.ids ? reinterpret_cast<uint16_t *>(dyn + op.off_ids) : nullptr;
    uint16_t *col = op.csr_w ? reinterpret_cast<uint16_t *>(dyn + op.off_col) : nullptr;
    if (ids || col) {
        const int Wd = op.csr_w;
        for (int i = threadIdx.x; i < N; i += blockDim.x) {
            if (ids) ids[i] = (uint16_t)P.perm[d.site_off + i];
            if (col) {
                const int rb = P.row_ptr[d.row_off + i], re = P.row_ptr[d.row_off + i + 1];
                for (int k = 0; k < Wd; ++k) {
                    const int raw = k < re - rb ? P.col[d.col_off + rb + k] : N;
                    // with random bonds the id keeps 15 bits and bit 15 holds J = -1
                    col[(size_t)i * Wd + k] = DISORDER ? (uint16_t)((raw & 0x7fff) | (raw < 0 ? 0x8000 : 0))
                                                       : (uint16_t)raw;
                }
            }
        }
    }
    float *part = reinterpret_cast<float *>(dyn + op.off_part);
    unsigned *part_met = reinterpret_cast<unsigned *>(dyn + op.off_met);
    __syncthreads();

    float *sx = xs + rl, *sy = ys + rl, *sz = zs + rl;
    uint32_t t = P.sweep[s];
    const bool met = op.ops & XYL_OP_MET, orx = op.ops & XYL_OP_OR;
    for (int it = 0; it < op.n_sweeps; ++it) {
        const bool measure = (op.ops & XYL_OP_MEASURE) && op.measure_every > 0 &&
                             ((t + 1u) % (uint32_t)op.measure_every) == 0u;
        const int slot = sh.slot_of[r];
        const float beta = sh.beta[slot], half_width = sh.delta[slot];
        float e = 0.f;
        unsigned acc = 0u;
        if (met) {
            for (int c = 0; c < d.Q; ++c) {
                if (orx) o3_phase<true, false, DEG, DISORDER>(P, d, sh, op, col, ids, sx, sy, sz, c, t, r, beta,
                                                              half_width, e, acc);
                else o3_phase<true, true, DEG, DISORDER>(P, d, sh, op, col, ids, sx, sy, sz, c, t, r, beta,
                                                         half_width, e, acc);
                __syncthreads();
            }
        }
        if (orx) {
            for (int c = 0; c < d.Q; ++c) {
                o3_phase<false, true, DEG, DISORDER>(P, d, sh, op, col, ids, sx, sy, sz, c, t, r, beta, half_width, e,
                                                     acc);
                __syncthreads();
            }
        }
        // per-warp partials: fused energy, accepted moves and, on measurement
        // sweeps, magnetisation and Fourier sums of every site of this replica
        float m[kO3Sums - 1];
#pragma unroll
        for (int f = 0; f < kO3Sums - 1; ++f) m[f] = 0.f;
        if (measure) {
            for (int q = threadIdx.x; q < N * Rg; q += blockDim.x) {
                const int i = q >> op.log2rg;
                const float vx = sx[i * Rg], vy = sy[i * Rg], vz = sz[i * Rg];
                const float4 ph = __ldg(reinterpret_cast<const float4 *>(P.phase) + d.site_off + i);
                m[kObsMx - 1] += vx;
                m[kObsMy - 1] += vy;
                m[kObsMz - 1] += vz;
                m[kObsF1xRe - 1] += vx * ph.x; m[kObsF1xIm - 1] += vx * ph.y;
                m[kObsF1yRe - 1] += vy * ph.x; m[kObsF1yIm - 1] += vy * ph.y;
                m[kObsF1zRe - 1] += vz * ph.x; m[kObsF1zIm - 1] += vz * ph.y;
                m[kObsF2xRe - 1] += vx * ph.z; m[kObsF2xIm - 1] += vx * ph.w;
                m[kObsF2yRe - 1] += vy * ph.z; m[kObsF2yIm - 1] += vy * ph.w;
                m[kObsF2zRe - 1] += vz * ph.z; m[kObsF2zIm - 1] += vz * ph.w;
            }
        }
        const int nf = measure ? kO3Sums : 1;
        {
            const float ew = o3_warp_reduce(op, e);
            if (owner_lane) part[((size_t)0 * op.n_warps + warp) * Rg + rl] = ew;
            if (met) {
                const unsigned a = o3_warp_reduce(op, acc);
                if (owner_lane) part_met[warp * Rg + rl] = a;
            }
            if (measure) {
#pragma unroll
                for (int f = 1; f < kO3Sums; ++f) {
                    const float x = o3_warp_reduce(op, m[f - 1]);
                    if (owner_lane) part[((size_t)f * op.n_warps + warp) * Rg + rl] = x;
                }
            }
        }
        __syncthreads();
        // CTA sums in a fixed shuffle tree (lane w holds warp w's partial); one
        // CTA covers its replicas' sites, so the sums are stored
        const int buf = (int)(t & 1u);
        double *obs_s = P.obs + ((size_t)buf * P.total_R + d.rep_off) * kObsStride;
        for (int q = warp; q < Rg * nf; q += op.n_warps) {
            const int ql = q / nf, f = q % nf;
            float v = lane < op.n_warps ? part[((size_t)f * op.n_warps + lane) * Rg + ql] : 0.f;
            v = warp_sum(v);
            if (lane == 0) __stcg(obs_s + (size_t)(group * Rg + ql) * kObsStride + f, (double)v);
        }
        if (met) {
            for (int ql = warp; ql < Rg; ql += op.n_warps) {
                unsigned n = lane < op.n_warps ? part_met[lane * Rg + ql] : 0u;
                n = warp_sum(n);
                if (lane == 0 && n)
                    atomicAdd(&P.met_acc[d.rep_off + sh.slot_of[group * Rg + ql]], (unsigned long long)n);
            }
        }
        if (global_barrier) {
            // every group signs in once its sums are out and waits (bounded)
            // for the others; the outcome reaches the CTA through shared memory
            __threadfence();
            __syncthreads();
            if (threadIdx.x == 0) {
                atomicAdd(&P.barrier[s], 1u);
                int failed = 0;
                if (!wait_counter_at_least(&P.barrier[s], (unsigned int)(n_groups * (it + 1)), kO3BarrierPolls)) {
                    atomicExch(P.status, XYL_ETIMEOUT);
                    failed = 1;
                }
                __threadfence();
                sh.abort_flag = failed;
            }
        }
        // every group's sums are out before any CTA reads them
        cluster_arrive();
        cluster_wait();
        if (global_barrier && *(volatile int *)&sh.abort_flag) break;
        for (int k = threadIdx.x; k < R; k += blockDim.x) sh.E[k] = __ldcg(obs_s + (size_t)k * kObsStride + kObsE);
        __syncthreads();
        pt_and_record(P, d, sh.E, sh.rep_at, sh.slot_of, t, op.ops, leader && rank == 0, met, measure, obs_s, beta64,
                      3);
        ++t;
        __syncthreads();
    }
    if (leader && rank == 0 && threadIdx.x == 0) P.sweep[s] = t;
    // write the group's spins back
    float4 *gspw = reinterpret_cast<float4 *>(P.spins) + d.spin_off;
    for (int k = threadIdx.x; k < N * Rg; k += blockDim.x) {
        const int i = k >> op.log2rg, q = k & (Rg - 1);
        __stcg(gspw + (int64_t)(group * Rg + q) * N + i, make_float4(xs[k], ys[k], zs[k], 0.f));
    }
}

// Up to 672 threads with 96 registers each, or up to 1024 with 64.
template <int DEG, bool DISORDER>
__global__ void __maxnreg__(96) resident_o3_kernel(DevPlan P, O3Params op)
{
    o3_body<DEG, DISORDER>(P, op);
}

template <int DEG, bool DISORDER>
__global__ void __launch_bounds__(1024, 1) resident_o3_kernel_wide(DevPlan P, O3Params op)
{
    o3_body<DEG, DISORDER>(P, op);
}

using O3KernelFn = void (*)(DevPlan, O3Params);

template <bool DISORDER>
O3KernelFn pick_o3_d(const BatchedShape &B)
{
    const bool wide = B.block > kResidentNarrowMaxThreads;
    if (B.fixed_deg == 6) return wide ? resident_o3_kernel_wide<6, DISORDER> : resident_o3_kernel<6, DISORDER>;
    if (B.max_deg > 8) return wide ? resident_o3_kernel_wide<0, DISORDER> : resident_o3_kernel<0, DISORDER>;
    return wide ? resident_o3_kernel_wide<-8, DISORDER> : resident_o3_kernel<-8, DISORDER>;
}

O3KernelFn pick_o3(const BatchedShape &B) { return B.disorder ? pick_o3_d<true>(B) : pick_o3_d<false>(B); }

cudaLaunchConfig_t o3_config(const BatchedShape &B, unsigned n_ctas, cudaLaunchAttribute *attr)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(n_ctas, 1, 1);
    cfg.blockDim = dim3((unsigned)B.block, 1, 1);
    cfg.dynamicSmemBytes = B.smem_bytes;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)B.cpc;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cfg;
}

}  // namespace

cudaError_t resident_o3_max_active_clusters(const BatchedShape &B, int *clusters)
{
    const O3KernelFn kernel = pick_o3(B);
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kResidentDynLimitBytes);
    if (e != cudaSuccess) return e;
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = o3_config(B, (unsigned)B.cpc, attr);
    return cudaOccupancyMaxActiveClusters(clusters, kernel, &cfg);
}

cudaError_t launch_resident_o3(const DevPlan &P, const BatchedShape &B, const int2 *d_units, int unit_begin,
                               int unit_count, int n_sweeps, uint32_t ops, int measure_every, cudaStream_t st)
{
    if (unit_count <= 0) return cudaSuccess;
    O3Params op;
    op.units = d_units;
    op.unit_begin = unit_begin;
    op.gpc = B.gpc;
    op.Rg = B.Rg;
    op.log2rg = 0;
    while ((1 << op.log2rg) < B.Rg) ++op.log2rg;
    op.n_sweeps = n_sweeps;
    op.ops = ops;
    op.measure_every = measure_every;
    op.n_warps = B.block / 32;
    op.comp = B.o3_comp;
    op.off_part = (int)B.rs_off_part;
    op.off_met = (int)B.rs_off_met;
    op.off_beta = (int)B.rs_off_beta;
    op.off_ids = (int)B.rs_off_ids;
    op.off_col = (int)B.rs_off_col;
    op.csr_w = B.rs_csr_w;
    op.ids = B.rs_ids ? 1 : 0;
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = o3_config(B, (unsigned)unit_count, attr);
    cfg.stream = st;
    return cudaLaunchKernelEx(&cfg, pick_o3(B), P, op);
}

}  // namespace xyl
