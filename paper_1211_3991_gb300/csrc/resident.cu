// Resident FP32 engine: the batched sampler with each CTA's replicas held in
// shared memory for the whole launch.
//
// Work decomposition.  The replicas of a sample are split into groups of Rg
// (a power of two); one CTA owns a group and keeps the group's spins of every
// site, [site][replica] float2, in shared memory from the start of the launch
// to its end, so a colour phase reads and writes nothing but shared memory and
// phases are separated by __syncthreads alone.  The CTAs of all groups of a
// sample form one thread-block cluster: once per sweep they publish their
// replicas' energies (and, on measurement sweeps, the magnetisation and
// Fourier sums) and meet at a cluster barrier, after which every CTA takes the
// same parallel-tempering decisions and the first CTA records the
// measurement.  Clusters never wait on one another.
//
// The per-spin arithmetic, the random streams and the order of every field
// sum are those of the global-memory batched kernel, so both give bit-equal
// spins from the same state; only the order of the energy sums differs.
// The CSR rows (as 16-bit ids) and the random-stream site ids are staged in
// shared memory when they fit beside the spins; otherwise they are read
// through the read-only path, one item ahead.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include "engines.h"
#include "sweep_tail.cuh"

namespace cg = cooperative_groups;

namespace xyl {
namespace {

constexpr int kSums = kObsCount;

struct ResidentParams {
    int sample_begin;
    int cpc;             // CTAs per cluster = replica groups per sample
    int Rg;
    int log2lps;         // log2 of the lanes that share a site (Rg / RV)
    int n_sweeps;
    uint32_t ops;
    int measure_every;
    int n_warps;
    // dynamic shared memory layout (byte offsets; 0 size = not staged)
    int off_ids, off_col, off_part, off_met;
    int csr_w;           // staged CSR row width (6 or 8), 0 = rows read from global memory
    int ids;             // random-stream site ids staged as 16-bit values
};

struct ResidentShared {
    double E[kMaxReplicas];          // energies of every replica of the sample
    float beta[kMaxReplicas];        // per slot
    float delta[kMaxReplicas];       // per slot
    int slot_of[kMaxReplicas];
    int rep_at[kMaxReplicas];
    int cls_cb[kMaxColorsBatched + 1];
};
static_assert(sizeof(ResidentShared) + kResidentDynLimitBytes <= 232448, "resident shared memory above 227 KB");

// Neighbour ids and random-stream key of one site.
template <int DEG>
struct Row {
    int nb[DEG > 0 ? DEG : 8];  // missing entries of a shorter row point at the zero spin N
    uint32_t key;
};

struct Stage {
    const uint16_t *col;   // [N][csr_w] colour-sorted ids, padding -> N (a zero spin)
    const uint16_t *ids;   // [N] original ids
};

template <int DEG, bool IS_MET>
__device__ __forceinline__ void fetch_row(const DevPlan &P, const DevSample &d, const ResidentParams &rp,
                                          const Stage &stg, int i, Row<DEG> &row)
{
    constexpr int W = DEG > 0 ? DEG : 8;
    if (stg.col) {
        // rows of W 16-bit ids, 4-byte aligned (W even)
        const uint32_t *c = reinterpret_cast<const uint32_t *>(stg.col + (size_t)i * W);
#pragma unroll
        for (int k = 0; k < W / 2; ++k) {
            const uint32_t w = c[k];
            row.nb[2 * k] = (int)(w & 0xffffu);
            row.nb[2 * k + 1] = (int)(w >> 16);
        }
    } else {
        const int32_t *cl = P.col + d.col_off;
        int rb, deg;
        if (DEG > 0) {
            rb = i * DEG;  // every row has DEG entries
            deg = DEG;
        } else {
            rb = __ldg(P.row_ptr + d.row_off + i);
            deg = __ldg(P.row_ptr + d.row_off + i + 1) - rb;
        }
#pragma unroll
        for (int k = 0; k < W; ++k) row.nb[k] = (DEG > 0 || k < deg) ? __ldg(cl + rb + k) : d.N;
    }
    if (IS_MET) row.key = stg.ids ? (uint32_t)stg.ids[i] : (uint32_t)__ldg(P.perm + d.site_off + i);
}

template <int RV>
__device__ __forceinline__ void lds_spins(const float2 *p, float2 (&v)[RV])
{
    if constexpr (RV == 2) {
        const float4 q = *reinterpret_cast<const float4 *>(p);
        v[0] = make_float2(q.x, q.y);
        v[1] = make_float2(q.z, q.w);
    } else {
        v[0] = *p;
    }
}

template <int RV>
__device__ __forceinline__ void sts_spins(float2 *p, const float2 (&v)[RV])
{
    if constexpr (RV == 2)
        *reinterpret_cast<float4 *>(p) = make_float4(v[0].x, v[0].y, v[1].x, v[1].y);
    else
        *p = v[0];
}

template <int RV>
struct RLane {
    int r0;              // first replica this thread updates (absolute within the sample)
    int lane_rep;        // its offset within the group
    float beta[RV], delta[RV];
    float e[RV];
    unsigned int acc[RV];
};

// One colour phase over every site of colour c for this CTA's replicas: one
// thread per (site, block of RV consecutive replicas).  sp points at the
// group's spins in shared memory.
template <bool IS_MET, bool FUSE_E, int RV, int DEG>
__device__ __forceinline__ void rphase(const DevPlan &P, const DevSample &d, const ResidentShared &sh,
                                       const ResidentParams &rp, const Stage &stg, float2 *sp, int c, uint32_t t,
                                       RLane<RV> &ln)
{
    constexpr int W = DEG > 0 ? DEG : 8;
    const int cb = sh.cls_cb[c], ce = sh.cls_cb[c + 1];
    const int items = (ce - cb) << rp.log2lps;
    const int Rg = rp.Rg;
    float2 *spl = sp + ln.lane_rep;
    int q = threadIdx.x;
    if (q >= items) return;
    Row<DEG> cur;
    fetch_row<DEG, IS_MET>(P, d, rp, stg, cb + (q >> rp.log2lps), cur);
    for (; q < items; q += blockDim.x) {
        const int i = cb + (q >> rp.log2lps);
        Row<DEG> nxt;
        const int qn = q + (int)blockDim.x;
        if (qn < items) fetch_row<DEG, IS_MET>(P, d, rp, stg, cb + (qn >> rp.log2lps), nxt);
        float2 s[RV];
        lds_spins<RV>(spl + i * Rg, s);
        float hx[RV], hy[RV], lx[RV], ly[RV];
#pragma unroll
        for (int v = 0; v < RV; ++v) hx[v] = hy[v] = lx[v] = ly[v] = 0.f;
#pragma unroll
        for (int k = 0; k < W; ++k) {
            const int j = cur.nb[k];
            float2 sj[RV];
            lds_spins<RV>(spl + j * Rg, sj);
            const bool lower = FUSE_E && j < cb;
#pragma unroll
            for (int v = 0; v < RV; ++v) {
                hx[v] += sj[v].x;
                hy[v] += sj[v].y;
                if (lower) {
                    lx[v] += sj[v].x;
                    ly[v] += sj[v].y;
                }
            }
        }
        float2 n[RV];
        if (IS_MET) {
            const Words4 x = met_block_f32(cur.key, t, ln.r0, d.sample_id, P.key);
            bool any = false;
#pragma unroll
            for (int v = 0; v < RV; ++v) {
                // replica r0 + v: even replicas take (w0, w1), odd ones (w2, w3)
                const bool odd = ((ln.r0 + v) & 1) != 0;
                const bool ok = metropolis_step_f32(s[v].x, s[v].y, hx[v], hy[v], ln.beta[v], ln.delta[v],
                                                    odd ? x.w2 : x.w0, odd ? x.w3 : x.w1, n[v].x, n[v].y);
                if (!ok) n[v] = s[v];
                ln.acc[v] += ok ? 1u : 0u;
                any |= ok;
            }
            if (any) sts_spins<RV>(spl + i * Rg, n);
        } else {
#pragma unroll
            for (int v = 0; v < RV; ++v) overrelax_step(s[v].x, s[v].y, hx[v], hy[v], n[v].x, n[v].y);
            sts_spins<RV>(spl + i * Rg, n);
        }
        if (FUSE_E) {
#pragma unroll
            for (int v = 0; v < RV; ++v) ln.e[v] -= n[v].x * lx[v] + n[v].y * ly[v];
        }
        cur = nxt;
    }
}

// Warp partial of a per-thread value of group replica rl (lanes l and l ^ o,
// o >= lanes per site, hold the same replicas), one slot per warp so the CTA
// sum is taken in a fixed order.
__device__ __forceinline__ float warp_reduce_rep(const ResidentParams &rp, float x)
{
    for (int o = 16; o >= (1 << rp.log2lps); o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

__device__ __forceinline__ unsigned warp_reduce_rep(const ResidentParams &rp, unsigned x)
{
    for (int o = 16; o >= (1 << rp.log2lps); o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

template <int RV, int DEG>
__device__ __forceinline__ void resident_sweeps(const DevPlan &P, const ResidentParams &rp, ResidentShared &sh,
                                                const Stage &stg, float2 *sp, float *part, unsigned *part_met,
                                                int s, int group)
{
    const DevSample d = P.samples[s];
    const int R = d.R, Rg = rp.Rg;
    const bool leader = group == 0;
    const int warp = (int)(threadIdx.x >> 5);
    RLane<RV> ln;
    ln.lane_rep = (int)(threadIdx.x & ((1u << rp.log2lps) - 1u)) * RV;
    ln.r0 = group * Rg + ln.lane_rep;
    const bool owner_lane = (threadIdx.x & 31u) < (1u << rp.log2lps);
    uint32_t t = P.sweep[s];
    const bool met = rp.ops & XYL_OP_MET, orx = rp.ops & XYL_OP_OR;
    for (int it = 0; it < rp.n_sweeps; ++it) {
        const bool measure = (rp.ops & XYL_OP_MEASURE) && rp.measure_every > 0 &&
                             ((t + 1u) % (uint32_t)rp.measure_every) == 0u;
#pragma unroll
        for (int v = 0; v < RV; ++v) {
            const int slot = sh.slot_of[ln.r0 + v];
            ln.beta[v] = sh.beta[slot];
            ln.delta[v] = sh.delta[slot];
            ln.e[v] = 0.f;
            ln.acc[v] = 0u;
        }
        if (met) {
            for (int c = 0; c < d.Q; ++c) {
                if (orx) rphase<true, false, RV, DEG>(P, d, sh, rp, stg, sp, c, t, ln);
                else rphase<true, true, RV, DEG>(P, d, sh, rp, stg, sp, c, t, ln);
                __syncthreads();
            }
        }
        if (orx) {
            for (int c = 0; c < d.Q; ++c) {
                rphase<false, true, RV, DEG>(P, d, sh, rp, stg, sp, c, t, ln);
                __syncthreads();
            }
        }
        // per-warp partials: fused energy, accepted moves and, on measurement
        // sweeps, magnetisation and Fourier sums of the final spins
        float m[RV][kSums - 1];
#pragma unroll
        for (int v = 0; v < RV; ++v)
#pragma unroll
            for (int f = 0; f < kSums - 1; ++f) m[v][f] = 0.f;
        if (measure) {
            const int items = d.N << rp.log2lps;
            for (int q = threadIdx.x; q < items; q += blockDim.x) {
                const int i = q >> rp.log2lps;
                float2 sv[RV];
                lds_spins<RV>(sp + ln.lane_rep + i * Rg, sv);
                const float4 ph = __ldg(reinterpret_cast<const float4 *>(P.phase) + d.site_off + i);
#pragma unroll
                for (int v = 0; v < RV; ++v) {
                    m[v][kObsMx - 1] += sv[v].x;
                    m[v][kObsMy - 1] += sv[v].y;
                    m[v][kObsF1xRe - 1] += sv[v].x * ph.x; m[v][kObsF1xIm - 1] += sv[v].x * ph.y;
                    m[v][kObsF1yRe - 1] += sv[v].y * ph.x; m[v][kObsF1yIm - 1] += sv[v].y * ph.y;
                    m[v][kObsF2xRe - 1] += sv[v].x * ph.z; m[v][kObsF2xIm - 1] += sv[v].x * ph.w;
                    m[v][kObsF2yRe - 1] += sv[v].y * ph.z; m[v][kObsF2yIm - 1] += sv[v].y * ph.w;
                }
            }
        }
        const int nf = measure ? kSums : 1;
#pragma unroll
        for (int v = 0; v < RV; ++v) {
            const int rl = ln.lane_rep + v;
            const float e = warp_reduce_rep(rp, ln.e[v]);
            if (owner_lane) part[((size_t)0 * rp.n_warps + warp) * Rg + rl] = e;
            if (met) {
                const unsigned a = warp_reduce_rep(rp, ln.acc[v]);
                if (owner_lane) part_met[warp * Rg + rl] = a;
            }
            if (measure) {
#pragma unroll
                for (int f = 1; f < kSums; ++f) {
                    const float x = warp_reduce_rep(rp, m[v][f - 1]);
                    if (owner_lane) part[((size_t)f * rp.n_warps + warp) * Rg + rl] = x;
                }
            }
        }
        __syncthreads();
        // CTA sums in warp order, in FP64; this CTA alone owns its replicas' slots
        const int buf = (int)(t & 1u);
        double *obs_s = P.obs + ((size_t)buf * P.total_R + d.rep_off) * kObsStride;
        for (int q = threadIdx.x; q < Rg * nf; q += blockDim.x) {
            const int rl = q / nf, f = q % nf;
            double v = 0.0;
            for (int w = 0; w < rp.n_warps; ++w) v += (double)part[((size_t)f * rp.n_warps + w) * Rg + rl];
            __stcg(obs_s + (size_t)(group * Rg + rl) * kObsStride + f, v);
        }
        if (met && threadIdx.x < Rg) {
            const int r = group * Rg + threadIdx.x;
            unsigned int n = 0;
            for (int w = 0; w < rp.n_warps; ++w) n += part_met[w * Rg + threadIdx.x];
            if (n) atomicAdd(&P.met_acc[d.rep_off + sh.slot_of[r]], (unsigned long long)n);
        }
        // every group's sums are out before any CTA reads them
        cluster_arrive();
        cluster_wait();
        for (int k = threadIdx.x; k < R; k += blockDim.x) sh.E[k] = __ldcg(obs_s + (size_t)k * kObsStride + kObsE);
        __syncthreads();
        pt_and_record(P, d, sh.E, sh.rep_at, sh.slot_of, t, rp.ops, leader, met, measure, obs_s);
        ++t;
        __syncthreads();
    }
    if (leader && threadIdx.x == 0) P.sweep[s] = t;
}

template <int RV, int DEG>
__global__ void __maxnreg__(96) resident_kernel(DevPlan P, ResidentParams rp)
{
    __shared__ ResidentShared sh;
    extern __shared__ __align__(16) unsigned char dyn[];
    cg::cluster_group cluster = cg::this_cluster();
    const int group = (int)cluster.block_rank();
    const int s = rp.sample_begin + (int)(blockIdx.x / (unsigned)rp.cpc);
    const DevSample d = P.samples[s];
    const int R = d.R, Rg = rp.Rg, N = d.N;

    for (int k = threadIdx.x; k < R; k += blockDim.x) {
        sh.slot_of[k] = P.slot_of[d.rep_off + k];
        sh.rep_at[k] = P.rep_at[d.rep_off + k];
        sh.beta[k] = (float)P.beta[d.rep_off + k];
        sh.delta[k] = (float)P.delta[d.rep_off + k];
    }
    for (int c = threadIdx.x; c <= d.Q; c += blockDim.x) sh.cls_cb[c] = P.color_ptr[d.color_off + c];

    // the group's spins of every site, then one zero row (target of padded CSR entries)
    float2 *sp = reinterpret_cast<float2 *>(dyn);
    const float2 *gsp = reinterpret_cast<const float2 *>(P.spins) + d.spin_off + group * Rg;
    for (int k = threadIdx.x; k < N * Rg; k += blockDim.x) {
        const int i = k / Rg, rl = k - i * Rg;
        sp[k] = __ldcg(gsp + (size_t)i * R + rl);
    }
    for (int k = threadIdx.x; k < Rg; k += blockDim.x) sp[(size_t)N * Rg + k] = make_float2(0.f, 0.f);
    Stage stg{nullptr, nullptr};
    if (rp.ids) {
        uint16_t *ids = reinterpret_cast<uint16_t *>(dyn + rp.off_ids);
        for (int i = threadIdx.x; i < N; i += blockDim.x) ids[i] = (uint16_t)P.perm[d.site_off + i];
        stg.ids = ids;
    }
    if (rp.csr_w) {
        uint16_t *col = reinterpret_cast<uint16_t *>(dyn + rp.off_col);
        const int W = rp.csr_w;
        for (int q = threadIdx.x; q < N * W; q += blockDim.x) {
            const int i = q / W, k = q - i * W;
            const int rb = P.row_ptr[d.row_off + i], re = P.row_ptr[d.row_off + i + 1];
            col[q] = (uint16_t)(k < re - rb ? P.col[d.col_off + rb + k] : N);
        }
        stg.col = col;
    }
    float *part = reinterpret_cast<float *>(dyn + rp.off_part);
    unsigned *part_met = reinterpret_cast<unsigned *>(dyn + rp.off_met);
    __syncthreads();
    resident_sweeps<RV, DEG>(P, rp, sh, stg, sp, part, part_met, s, group);
    // write the spins back
    float2 *gspw = reinterpret_cast<float2 *>(P.spins) + d.spin_off + group * Rg;
    for (int k = threadIdx.x; k < N * Rg; k += blockDim.x) {
        const int i = k / Rg, rl = k - i * Rg;
        __stcg(gspw + (size_t)i * R + rl, sp[k]);
    }
}

using KernelFn = void (*)(DevPlan, ResidentParams);

KernelFn pick_resident(const BatchedShape &B)
{
    const bool rv2 = B.Rg >= 2;
    if (B.fixed_deg == 6) return rv2 ? resident_kernel<2, 6> : resident_kernel<1, 6>;
    return rv2 ? resident_kernel<2, -8> : resident_kernel<1, -8>;
}

cudaError_t set_resident_attributes(KernelFn k)
{
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kResidentDynLimitBytes);
    return e;
}

cudaLaunchConfig_t resident_config(const BatchedShape &B, unsigned n_ctas, cudaLaunchAttribute *attr)
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

size_t resident_static_smem_bytes() { return sizeof(ResidentShared); }

cudaError_t resident_max_active_clusters(const BatchedShape &B, int *clusters)
{
    const KernelFn kernel = pick_resident(B);
    cudaError_t e = set_resident_attributes(kernel);
    if (e != cudaSuccess) return e;
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = resident_config(B, (unsigned)B.cpc, attr);
    return cudaOccupancyMaxActiveClusters(clusters, kernel, &cfg);
}

cudaError_t launch_resident(const DevPlan &P, const BatchedShape &B, int sample_begin, int sample_count,
                            int n_sweeps, uint32_t ops, int measure_every, cudaStream_t st)
{
    if (sample_count <= 0) return cudaSuccess;
    ResidentParams rp;
    rp.sample_begin = sample_begin;
    rp.cpc = B.cpc;
    rp.Rg = B.Rg;
    const int rv = B.Rg >= 2 ? 2 : 1;
    rp.log2lps = 0;
    while ((1 << rp.log2lps) < B.Rg / rv) ++rp.log2lps;
    rp.n_sweeps = n_sweeps;
    rp.ops = ops;
    rp.measure_every = measure_every;
    rp.n_warps = B.block / 32;
    rp.off_ids = (int)B.rs_off_ids;
    rp.off_col = (int)B.rs_off_col;
    rp.off_part = (int)B.rs_off_part;
    rp.off_met = (int)B.rs_off_met;
    rp.csr_w = B.rs_csr_w;
    rp.ids = B.rs_ids ? 1 : 0;
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = resident_config(B, (unsigned)(sample_count * B.cpc), attr);
    cfg.stream = st;
    return cudaLaunchKernelEx(&cfg, pick_resident(B), P, rp);
}

}  // namespace xyl
