// Resident FP32 engine: the batched sampler with the spins held in shared
// memory for the whole launch.
//
// Work decomposition.  The replicas of a sample are split into groups of Rg
// (a power of two).  G CTAs (G >= 1) share a group: each keeps a full copy of
// the group's spins of every site, [site][replica] float2, in its shared
// memory from the start of the launch to its end, and updates its own chunk
// of every colour class (chunk k of a class is its k-th contiguous 1/G).  A
// colour phase therefore reads nothing but shared memory.  With G > 1 a CTA
// writes each spin it changes into its own copy and into the copies of the
// CTAs whose chunks have a link to that site (a per-site mask of peers, built
// on the host), and the phases are separated by cluster barriers; with G = 1
// __syncthreads separates them.
//
// A cluster holds gpc groups x G CTAs.  When all groups of a sample fit in one
// cluster (gpc = R / Rg) the sample's CTAs meet once per sweep at a cluster
// barrier; otherwise (gpc = 1) at a bounded global barrier like the
// global-memory kernel's.  After the barrier every CTA reads all replica
// energies, takes the same parallel-tempering decisions, and the first CTA of
// the first group records the measurement.
//
// The per-spin arithmetic, the random streams and the order of every field
// sum are those of the global-memory batched kernel, so both give bit-equal
// spins from the same state; only the order of the energy sums differs.  The
// CSR rows of a CTA's own sites (16-bit ids) and their random-stream site ids
// are staged in shared memory when they fit beside the spins; otherwise they
// are read through the read-only path, one item ahead.  Rows longer than eight
// (the paper's 2N-bond graphs) are read from the global CSR entry by entry.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include "engines.h"
#include "sweep_tail.cuh"

namespace cg = cooperative_groups;

namespace xyl {
namespace {

constexpr int kSums = kObsCount;
constexpr unsigned int kResidentBarrierPolls = 1u << 21;  // about a second of polling

struct ResidentParams {
    const int2 *units;   // (sample, group), sample-major
    int unit_begin;
    int G;               // CTAs that share one replica group
    int gpc;             // replica groups per cluster
    int Rg;
    int log2lps;         // log2 of the lanes that share a site (Rg / RV)
    int n_sweeps;
    uint32_t ops;
    int measure_every;
    int n_warps;
    // dynamic shared memory layout (byte offsets)
    int off_ids, off_col, off_part, off_met, off_peers;  // off_peers 0: masks read from global memory
    int off_beta;        // FP64 slot inverse temperatures (parallel tempering)
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
    int cls_lo[kMaxColorsBatched];   // this CTA's chunk of each class: [lo, hi)
    int cls_hi[kMaxColorsBatched];
    int cls_base[kMaxColorsBatched]; // first staged row of the chunk
    int abort_flag;
};
static_assert(sizeof(ResidentShared) + kResidentDynLimitBytes <= 232448, "resident shared memory above 227 KB");

// Neighbour ids, random-stream key and peer mask of one site; with random
// bonds, bit k of neg marks a link with J = -1.
template <int DEG>
struct Row {
    int nb[DEG > 0 ? DEG : 8];  // missing entries of a shorter row point at the zero spin N
    uint32_t key;
    uint32_t peers;
    uint32_t neg;
};

// DEG = 0 (any degree): the row's place in the global CSR, read entry by entry.
template <>
struct Row<0> {
    int rb, deg;
    uint32_t key;
    uint32_t peers;
    uint32_t neg;
};

struct Stage {
    const uint16_t *col;    // [owned][csr_w] colour-sorted ids, padding -> N (a zero spin); J = -1 in bit 15 (DISORDER)
    const uint16_t *ids;    // [owned] original ids
    const uint16_t *peers;  // [owned] peer masks (site split)
};

// i: colour-sorted site id; l: its staged row.  With DISORDER the sign of each
// link comes from bit 15 of a staged id or bit 31 of a global one.
template <int DEG, bool IS_MET, bool SPLIT, bool DISORDER>
__device__ __forceinline__ void fetch_row(const DevPlan &P, const DevSample &d, const Stage &stg, int i, int l,
                                          Row<DEG> &row)
{
    constexpr int W = DEG > 0 ? DEG : 8;
    row.neg = 0u;
    if constexpr (DEG == 0) {
        row.rb = __ldg(P.row_ptr + d.row_off + i);
        row.deg = checked_id(P, __ldg(P.row_ptr + d.row_off + i + 1) - row.rb, d.max_deg + 1, 0);
    } else if (stg.col) {
        // rows of W 16-bit ids, 4-byte aligned (W even)
        const uint32_t *c = reinterpret_cast<const uint32_t *>(stg.col + (size_t)l * W);
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
            rb = i * DEG;  // every row has DEG entries
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
    if (IS_MET) row.key = stg.ids ? (uint32_t)stg.ids[l] : (uint32_t)__ldg(P.perm + d.site_off + i);
    if (SPLIT) row.peers = stg.peers ? stg.peers[l] : __ldg(P.push + d.site_off + i);
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

// Where this CTA sits: its group within the cluster and its chunk rank.
struct Place {
    int gi;              // group within the cluster
    int sr;              // chunk rank within the group (0..G-1)
};

// The new spins of site i go to this CTA's copy and, with a site split, to
// the copies of the peers that read the site: the same shared-memory offset in
// the peer, addressed through mapa and written with st.shared::cluster.
template <int RV, bool SPLIT>
__device__ __forceinline__ void put_spins(cg::cluster_group &cluster, const ResidentParams &rp, const Place &pl,
                                          float2 *p, uint32_t peers, const float2 (&n)[RV])
{
    (void)cluster;
    sts_spins<RV>(p, n);
    if (SPLIT) {
        const uint32_t local = (uint32_t)__cvta_generic_to_shared(p);
        const uint32_t first = (uint32_t)(pl.gi * rp.G);
        while (peers) {
            const uint32_t r = (uint32_t)__ffs(peers) - 1u;
            peers &= peers - 1u;
            uint32_t remote;
            asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(remote) : "r"(local), "r"(first + r));
            if constexpr (RV == 2)
                asm volatile("st.shared::cluster.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(remote), "f"(n[0].x), "f"(n[0].y),
                             "f"(n[RV - 1].x), "f"(n[RV - 1].y) : "memory");
            else
                asm volatile("st.shared::cluster.v2.f32 [%0], {%1, %2};" ::"r"(remote), "f"(n[0].x), "f"(n[0].y) : "memory");
        }
    }
}

// One colour phase over this CTA's chunk of colour c for its replicas: one
// thread per (site, block of RV consecutive replicas).  sp points at the
// group's spins in shared memory.
template <bool IS_MET, bool FUSE_E, int RV, int DEG, bool SPLIT, bool DISORDER>
__device__ __forceinline__ void rphase(const DevPlan &P, const DevSample &d, const ResidentShared &sh,
                                       const ResidentParams &rp, const Stage &stg, cg::cluster_group &cluster,
                                       const Place &pl, float2 *sp, int c, uint32_t t, RLane<RV> &ln)
{
    constexpr int W = DEG > 0 ? DEG : 8;
    const int cb = sh.cls_cb[c], lo = sh.cls_lo[c], base = sh.cls_base[c];
    const int items = (sh.cls_hi[c] - lo) << rp.log2lps;
    const int Rg = rp.Rg;
    float2 *spl = sp + ln.lane_rep;
    int q = threadIdx.x;
    if (q >= items) return;
    Row<DEG> cur;
    fetch_row<DEG, IS_MET, SPLIT, DISORDER>(P, d, stg, lo + (q >> rp.log2lps), base + (q >> rp.log2lps), cur);
    for (; q < items; q += blockDim.x) {
        const int i = lo + (q >> rp.log2lps);
        Row<DEG> nxt;
        const int qn = q + (int)blockDim.x;
        if (qn < items)
            fetch_row<DEG, IS_MET, SPLIT, DISORDER>(P, d, stg, lo + (qn >> rp.log2lps), base + (qn >> rp.log2lps), nxt);
        float2 s[RV];
        lds_spins<RV>(spl + i * Rg, s);
        float hx[RV], hy[RV], lx[RV], ly[RV];
#pragma unroll
        for (int v = 0; v < RV; ++v) hx[v] = hy[v] = lx[v] = ly[v] = 0.f;
        if constexpr (DEG == 0) {
            // any degree: ids from the global CSR in groups of four, sums in row order
            const int32_t *cl = P.col + d.col_off + cur.rb;
            for (int k0 = 0; k0 < cur.deg; k0 += 4) {
                int raw[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) raw[q] = k0 + q < cur.deg ? __ldg(cl + k0 + q) : 0;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    if (k0 + q >= cur.deg) break;
                    const int j = checked_id(P, DISORDER ? (raw[q] & 0x7fffffff) : raw[q], d.N + 1, d.N);
                    float2 sj[RV];
                    lds_spins<RV>(spl + j * Rg, sj);
                    if (DISORDER && raw[q] < 0) {
#pragma unroll
                        for (int v = 0; v < RV; ++v) sj[v] = make_float2(-sj[v].x, -sj[v].y);
                    }
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
            }
        } else {
#pragma unroll
            for (int k = 0; k < W; ++k) {
                const int j = checked_id(P, cur.nb[k], d.N + 1, d.N);  // N: the zero row
                float2 sj[RV];
                lds_spins<RV>(spl + j * Rg, sj);
                if (DISORDER && ((cur.neg >> k) & 1u)) {
#pragma unroll
                    for (int v = 0; v < RV; ++v) sj[v] = make_float2(-sj[v].x, -sj[v].y);
                }
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
        }
        if (DISORDER && P.field) {
            // the site's own field after its neighbours; the fused energy takes -h_i . S_i once
            const float2 f = __ldg(reinterpret_cast<const float2 *>(P.field) + d.site_off + i);
#pragma unroll
            for (int v = 0; v < RV; ++v) {
                hx[v] += f.x;
                hy[v] += f.y;
                if (FUSE_E) {
                    lx[v] += f.x;
                    ly[v] += f.y;
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
            if (any) put_spins<RV, SPLIT>(cluster, rp, pl, spl + i * Rg, cur.peers, n);
        } else {
#pragma unroll
            for (int v = 0; v < RV; ++v) overrelax_step(s[v].x, s[v].y, hx[v], hy[v], n[v].x, n[v].y);
            put_spins<RV, SPLIT>(cluster, rp, pl, spl + i * Rg, cur.peers, n);
        }
        if (FUSE_E) {
#pragma unroll
            for (int v = 0; v < RV; ++v) ln.e[v] -= n[v].x * lx[v] + n[v].y * ly[v];
        }
        cur = nxt;
    }
}

// Phases end at a cluster barrier when peers read this CTA's writes.
template <bool SPLIT>
__device__ __forceinline__ void phase_barrier()
{
    if (SPLIT) {
        cluster_arrive();
        cluster_wait();
    } else {
        __syncthreads();
    }
}

// Sum over the lanes of a warp that hold the same replicas (lanes l and
// l ^ o, o >= lanes per site).
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

template <int RV, int DEG, bool SPLIT, bool DISORDER>
__device__ __forceinline__ void resident_sweeps(const DevPlan &P, const ResidentParams &rp, ResidentShared &sh,
                                                const Stage &stg, cg::cluster_group &cluster, const Place &pl,
                                                float2 *sp, float *part, unsigned *part_met, const double *beta64,
                                                int s, int group)
{
    const DevSample d = P.samples[s];
    const int R = d.R, Rg = rp.Rg;
    const int n_groups = R / Rg;
    const bool global_barrier = rp.gpc < n_groups;
    const int rank = (int)cluster.block_rank();
    const bool leader = group == 0 && pl.sr == 0;
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
                if (orx) rphase<true, false, RV, DEG, SPLIT, DISORDER>(P, d, sh, rp, stg, cluster, pl, sp, c, t, ln);
                else rphase<true, true, RV, DEG, SPLIT, DISORDER>(P, d, sh, rp, stg, cluster, pl, sp, c, t, ln);
                phase_barrier<SPLIT>();
            }
        }
        if (orx) {
            for (int c = 0; c < d.Q; ++c) {
                rphase<false, true, RV, DEG, SPLIT, DISORDER>(P, d, sh, rp, stg, cluster, pl, sp, c, t, ln);
                phase_barrier<SPLIT>();
            }
        }
        // per-warp partials: fused energy, accepted moves and, on measurement
        // sweeps, magnetisation and Fourier sums of this CTA's final sites
        float m[RV][kSums - 1];
#pragma unroll
        for (int v = 0; v < RV; ++v)
#pragma unroll
            for (int f = 0; f < kSums - 1; ++f) m[v][f] = 0.f;
        if (measure) {
            for (int c = 0; c < d.Q; ++c) {
                const int lo = sh.cls_lo[c];
                const int items = (sh.cls_hi[c] - lo) << rp.log2lps;
                for (int q = threadIdx.x; q < items; q += blockDim.x) {
                    const int i = lo + (q >> rp.log2lps);
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
        // CTA sums: one warp per (replica, field) adds the warp partials in a
        // fixed shuffle tree (lane w holds warp w's); stored when this CTA
        // alone covers its replicas' sites, else added across the G CTAs
        const int buf = (int)(t & 1u);
        double *obs_s = P.obs + ((size_t)buf * P.total_R + d.rep_off) * kObsStride;
        const int lane = (int)(threadIdx.x & 31u);
        for (int q = warp; q < Rg * nf; q += rp.n_warps) {
            const int rl = q / nf, f = q % nf;
            float v = lane < rp.n_warps ? part[((size_t)f * rp.n_warps + lane) * Rg + rl] : 0.f;
            v = warp_sum(v);
            double *dst = obs_s + (size_t)(group * Rg + rl) * kObsStride + f;
            if (lane == 0) {
                if (SPLIT) atomicAdd(dst, (double)v);
                else __stcg(dst, (double)v);
            }
        }
        if (met) {
            for (int rl = warp; rl < Rg; rl += rp.n_warps) {
                unsigned n = lane < rp.n_warps ? part_met[lane * Rg + rl] : 0u;
                n = warp_sum(n);
                if (lane == 0 && n) atomicAdd(&P.met_acc[d.rep_off + sh.slot_of[group * Rg + rl]], (unsigned long long)n);
            }
        }
        if (global_barrier) {
            // every CTA of the sample signs in once its sums are out; the first
            // CTA of each cluster waits for all of them (bounded) and tells the
            // other CTAs of its cluster the outcome through their shared memory
            __threadfence();
            __syncthreads();
            if (threadIdx.x == 0) atomicAdd(&P.barrier[s], 1u);
            if (rank == 0 && threadIdx.x == 0) {
                int failed = 0;
                const unsigned int target = (unsigned int)(rp.G * n_groups * (it + 1));
                if (!wait_counter_at_least(&P.barrier[s], target, kResidentBarrierPolls)) {
                    atomicExch(P.status, XYL_ETIMEOUT);
                    failed = 1;
                }
                __threadfence();
                for (int k = 0; k < rp.G * rp.gpc; ++k) *cluster.map_shared_rank(&sh.abort_flag, k) = failed;
            }
        }
        // every group's sums are out before any CTA reads them
        cluster_arrive();
        cluster_wait();
        if (global_barrier && *(volatile int *)&sh.abort_flag) break;
        for (int k = threadIdx.x; k < R; k += blockDim.x) sh.E[k] = __ldcg(obs_s + (size_t)k * kObsStride + kObsE);
        __syncthreads();
        pt_and_record(P, d, sh.E, sh.rep_at, sh.slot_of, t, rp.ops, leader, met, measure, obs_s, beta64);
        if (SPLIT && pl.sr == 0) {
            // clear this group's slots of the buffer the next sweep adds into:
            // every reader of it finished before the barrier just passed
            double *nxt = P.obs + ((size_t)(buf ^ 1) * P.total_R + d.rep_off + group * Rg) * kObsStride;
            for (int q = threadIdx.x; q < Rg * kObsStride; q += blockDim.x) nxt[q] = 0.0;
        }
        ++t;
        __syncthreads();
    }
    if (leader && threadIdx.x == 0) P.sweep[s] = t;
}

template <int RV, int DEG, bool SPLIT, bool DISORDER>
__device__ __forceinline__ void resident_body(const DevPlan &P, const ResidentParams &rp)
{
    __shared__ ResidentShared sh;
    extern __shared__ __align__(16) unsigned char dyn[];
    cg::cluster_group cluster = cg::this_cluster();
    const int rank = (int)cluster.block_rank();
    Place pl;
    pl.gi = rank / rp.G;
    pl.sr = rank - pl.gi * rp.G;
    const int unit = rp.unit_begin + (int)(blockIdx.x / (unsigned)(rp.G * rp.gpc)) * rp.gpc + pl.gi;
    const int2 ug = rp.units[unit];
    const int s = ug.x, group = ug.y;
    const DevSample d = P.samples[s];
    const int R = d.R, Rg = rp.Rg, N = d.N;

    double *beta64 = reinterpret_cast<double *>(dyn + rp.off_beta);
    for (int k = threadIdx.x; k < R; k += blockDim.x) {
        sh.slot_of[k] = P.slot_of[d.rep_off + k];
        sh.rep_at[k] = P.rep_at[d.rep_off + k];
        sh.beta[k] = (float)P.beta[d.rep_off + k];
        sh.delta[k] = (float)P.delta[d.rep_off + k];
        beta64[k] = P.beta[d.rep_off + k];
    }
    if (threadIdx.x == 0) {
        sh.abort_flag = 0;
        // this CTA's chunk of every colour class
        int base = 0;
        for (int c = 0; c < d.Q; ++c) {
            int cb = P.color_ptr[d.color_off + c], ce = P.color_ptr[d.color_off + c + 1];
            checked_class(P, cb, ce, d.N);
            const int chunk = (ce - cb + rp.G - 1) / rp.G;
            const int lo = min(ce, cb + pl.sr * chunk), hi = min(ce, lo + chunk);
            sh.cls_cb[c] = cb;
            sh.cls_lo[c] = lo;
            sh.cls_hi[c] = hi;
            sh.cls_base[c] = base;
            base += hi - lo;
        }
        sh.cls_cb[d.Q] = P.color_ptr[d.color_off + d.Q];
    }

    // the group's spins of every site, then one zero row (target of padded CSR entries)
    float2 *sp = reinterpret_cast<float2 *>(dyn);
    const float2 *gsp = reinterpret_cast<const float2 *>(P.spins) + d.spin_off + group * Rg;
    for (int k = threadIdx.x; k < N * Rg; k += blockDim.x) {
        const int i = k / Rg, rl = k - i * Rg;
        sp[k] = __ldcg(gsp + (size_t)i * R + rl);
    }
    for (int k = threadIdx.x; k < Rg; k += blockDim.x) sp[(size_t)N * Rg + k] = make_float2(0.f, 0.f);
    __syncthreads();
    // rows, site ids and peer masks of this CTA's own sites
    Stage stg{nullptr, nullptr, nullptr};
    uint16_t *ids = rp.ids ? reinterpret_cast<uint16_t *>(dyn + rp.off_ids) : nullptr;
    uint16_t *col = rp.csr_w ? reinterpret_cast<uint16_t *>(dyn + rp.off_col) : nullptr;
    uint16_t *peers = (SPLIT && rp.off_peers) ? reinterpret_cast<uint16_t *>(dyn + rp.off_peers) : nullptr;
    if (ids || col || peers) {
        const int W = rp.csr_w;
        for (int c = 0; c < d.Q; ++c) {
            const int lo = sh.cls_lo[c], n = sh.cls_hi[c] - lo, base = sh.cls_base[c];
            for (int q = threadIdx.x; q < n; q += blockDim.x) {
                const int i = lo + q, l = base + q;
                if (ids) ids[l] = (uint16_t)P.perm[d.site_off + i];
                if (peers) peers[l] = P.push[d.site_off + i];
                if (col) {
                    const int rb = P.row_ptr[d.row_off + i], re = P.row_ptr[d.row_off + i + 1];
                    for (int k = 0; k < W; ++k) {
                        const int raw = k < re - rb ? P.col[d.col_off + rb + k] : N;
                        // with random bonds the id keeps 15 bits and bit 15 holds J = -1
                        col[(size_t)l * W + k] = DISORDER ? (uint16_t)((raw & 0x7fff) | (raw < 0 ? 0x8000 : 0))
                                                         : (uint16_t)raw;
                    }
                }
            }
        }
    }
    stg.ids = ids;
    stg.col = col;
    stg.peers = peers;
    float *part = reinterpret_cast<float *>(dyn + rp.off_part);
    unsigned *part_met = reinterpret_cast<unsigned *>(dyn + rp.off_met);
    // peers write into this CTA's copy only after it holds the starting spins
    if (SPLIT) cluster.sync();
    else __syncthreads();
    resident_sweeps<RV, DEG, SPLIT, DISORDER>(P, rp, sh, stg, cluster, pl, sp, part, part_met, beta64, s, group);
    // write this CTA's own sites back (every copy agrees after the last barrier)
    float2 *gspw = reinterpret_cast<float2 *>(P.spins) + d.spin_off + group * Rg;
    for (int c = 0; c < d.Q; ++c) {
        const int lo = sh.cls_lo[c], n = (sh.cls_hi[c] - lo) * Rg;
        for (int k = threadIdx.x; k < n; k += blockDim.x) {
            const int i = lo + k / Rg, rl = k % Rg;
            __stcg(gspw + (size_t)i * R + rl, sp[(size_t)i * Rg + rl]);
        }
    }
}

// Up to 672 threads with 96 registers each, or up to 1024 with 64.
template <int RV, int DEG, bool SPLIT, bool DISORDER>
__global__ void __maxnreg__(96) resident_kernel(DevPlan P, ResidentParams rp)
{
    resident_body<RV, DEG, SPLIT, DISORDER>(P, rp);
}

template <int RV, int DEG, bool SPLIT, bool DISORDER>
__global__ void __launch_bounds__(1024, 1) resident_kernel_wide(DevPlan P, ResidentParams rp)
{
    resident_body<RV, DEG, SPLIT, DISORDER>(P, rp);
}

using KernelFn = void (*)(DevPlan, ResidentParams);

template <int RV, int DEG, bool SPLIT, bool DISORDER>
KernelFn pick_width(const BatchedShape &B)
{
    return B.block > kResidentNarrowMaxThreads ? resident_kernel_wide<RV, DEG, SPLIT, DISORDER>
                                               : resident_kernel<RV, DEG, SPLIT, DISORDER>;
}

template <bool SPLIT, bool DISORDER>
KernelFn pick_split(const BatchedShape &B)
{
    const bool rv2 = B.Rg >= 2;
    if (B.fixed_deg == 6) return rv2 ? pick_width<2, 6, SPLIT, DISORDER>(B) : pick_width<1, 6, SPLIT, DISORDER>(B);
    if (B.max_deg > 8) return rv2 ? pick_width<2, 0, SPLIT, DISORDER>(B) : pick_width<1, 0, SPLIT, DISORDER>(B);
    return rv2 ? pick_width<2, -8, SPLIT, DISORDER>(B) : pick_width<1, -8, SPLIT, DISORDER>(B);
}

KernelFn pick_resident(const BatchedShape &B)
{
    if (B.disorder) return B.G > 1 ? pick_split<true, true>(B) : pick_split<false, true>(B);
    return B.G > 1 ? pick_split<true, false>(B) : pick_split<false, false>(B);
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

cudaError_t launch_resident(const DevPlan &P, const BatchedShape &B, const int2 *d_units, int unit_begin,
                            int unit_count, int n_sweeps, uint32_t ops, int measure_every, cudaStream_t st)
{
    if (unit_count <= 0) return cudaSuccess;
    ResidentParams rp;
    rp.units = d_units;
    rp.unit_begin = unit_begin;
    rp.G = B.G;
    rp.gpc = B.gpc;
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
    rp.off_beta = (int)B.rs_off_beta;
    rp.off_peers = (int)B.rs_off_peers;
    rp.csr_w = B.rs_csr_w;
    rp.ids = B.rs_ids ? 1 : 0;
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = resident_config(B, (unsigned)(unit_count / B.gpc * B.cpc), attr);
    cfg.stream = st;
    return cudaLaunchKernelEx(&cfg, pick_resident(B), P, rp);
}

}  // namespace xyl
