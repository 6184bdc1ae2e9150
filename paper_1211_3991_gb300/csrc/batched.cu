// Batched FP32 engine: one launch runs many whole sweep + swap + measure
// cycles for a batch of samples.
//
// Work decomposition.  The replicas of a sample are split into groups of Rg
// (a power of two).  Each (sample, group) unit is owned by one thread-block
// cluster of G CTAs.  Inside a unit, every colour class is cut into G
// contiguous chunks; CTA k updates chunk k for all Rg replicas, one thread per
// (site, replica) with the replica index fastest, so the lanes that share a
// site read one contiguous Rg x 8-byte segment of each neighbour's row.
// Spins are interleaved [sample][site][replica] float2 in global memory and
// stay L2-resident for the batch sizes this engine serves; they are read and
// written through L2 (ld/st .cg), and colour phases are separated by cluster
// barriers (release/acquire at cluster scope).  When they fit, the CSR rows
// and random-stream site ids of a CTA's chunks are staged once per launch in
// shared memory, so an update waits on a single L2 round trip (the neighbour
// spins); otherwise they are read through the read-only path.
//
// Sweep (App. B): Metropolis over colours 0..Q-1, then overrelaxation over
// colours 0..Q-1; the last pass also accumulates each replica's energy (links
// to lower colours, counted once at their upper endpoint), magnetisation and,
// on measurement sweeps, the Fourier sums.  Then the groups of a sample meet
// at a bounded global barrier, every CTA reads the sample's energies and takes
// the same PT decisions (FP64, deterministic), and the first CTA of group 0
// adds the measurement.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <mutex>

#include "engines.h"

namespace cg = cooperative_groups;

namespace xyl {
namespace {

constexpr unsigned int kBarrierPolls = 1u << 21;  // about a second of polling
constexpr int kMaxReplicas = 256;

struct BatchedParams {
    const int2 *units;   // (sample, group) per cluster
    int unit_begin;
    int G, Rg, log2Rg;
    int n_sweeps;
    uint32_t ops;
    int measure_every;
    int staged;          // CSR rows / site ids of the CTA's chunks in shared memory
    int owned_max;       // largest number of sites one CTA owns
    int max_deg;
};

__device__ __forceinline__ float2 ld_spin(const float2 *p) { return __ldcg(p); }
__device__ __forceinline__ void st_spin(float2 *p, float2 v) { __stcg(p, v); }

struct SharedState {
    double obs[32][kObsStride];            // per group replica: fused sums of this CTA
    unsigned long long met[32];            // per group replica: accepted Metropolis moves
    double E[kMaxReplicas];                // energies of every replica of the sample
    float beta[kMaxReplicas];              // per slot
    float delta[kMaxReplicas];             // per slot
    int slot_of[kMaxReplicas];
    int rep_at[kMaxReplicas];
    int cls_cb[kMaxColorsBatched + 1];     // colour-sorted start of each class
    int cls_lo[kMaxColorsBatched];         // this CTA's chunk of each class: [lo, hi)
    int cls_hi[kMaxColorsBatched];
    int cls_base[kMaxColorsBatched];       // first staged row of the chunk
    int abort_flag;
};

struct Staged {
    const int *col;      // [owned_max][max_deg] colour-sorted neighbour ids
    const int *deg;      // [owned_max]
    const int *site_id;  // [owned_max] original ids (random-stream keys)
};

// One colour phase of one pass for this CTA's chunk.
template <bool IS_MET, bool FUSE, bool STAGED>
__device__ __forceinline__ void phase(const DevPlan &P, const DevSample &d, SharedState &sh, const BatchedParams &bp,
                                      const Staged &stg, int group, int c, uint32_t t, bool fourier)
{
    const int cb = sh.cls_cb[c];
    const int lo = sh.cls_lo[c], hi = sh.cls_hi[c], base = sh.cls_base[c];
    const int items = hi > lo ? (hi - lo) << bp.log2Rg : 0;
    float2 *sp = reinterpret_cast<float2 *>(P.spins) + d.spin_off;
    const int32_t *rp = P.row_ptr + d.row_off;
    const int32_t *cl = P.col + d.col_off;
    const int R = d.R;
    const int rl = threadIdx.x & (bp.Rg - 1);
    const int r = group * bp.Rg + rl;

    float acc[kObsCount];
#pragma unroll
    for (int f = 0; f < kObsCount; ++f) acc[f] = 0.0f;
    unsigned int n_acc = 0;

    for (int q = threadIdx.x; q < items; q += blockDim.x) {
        const int off = q >> bp.log2Rg;
        const int i = lo + off;
        const int *nb;
        int deg;
        uint32_t site_key;
        if (STAGED) {
            const int l = base + off;
            nb = stg.col + (size_t)l * bp.max_deg;
            deg = stg.deg[l];
            site_key = (uint32_t)stg.site_id[l];
        } else {
            const int rb = __ldg(rp + i);
            nb = cl + rb;
            deg = __ldg(rp + i + 1) - rb;
            site_key = (uint32_t)__ldg(P.perm + d.site_off + i);
        }
        const float2 si = ld_spin(sp + (int64_t)i * R + r);
        float hx = 0.f, hy = 0.f, lx = 0.f, ly = 0.f;
#pragma unroll 6
        for (int k = 0; k < deg; ++k) {
            const int j = STAGED ? nb[k] : __ldg(nb + k);
            const float2 sj = ld_spin(sp + (int64_t)j * R + r);
            hx += sj.x;
            hy += sj.y;
            if (FUSE && j < cb) {
                lx += sj.x;
                ly += sj.y;
            }
        }
        float nx, ny;
        if (IS_MET) {
            const int slot = sh.slot_of[r];
            const Words4 x = philox_draw(site_key, t, kPurposeMet, (uint32_t)r, d.sample_id, P.key);
            const bool ok = metropolis_step(P, si.x, si.y, hx, hy, sh.beta[slot], sh.delta[slot], x, nx, ny);
            if (ok) {
                st_spin(sp + (int64_t)i * R + r, make_float2(nx, ny));
                ++n_acc;
            } else {
                nx = si.x;
                ny = si.y;
            }
        } else {
            overrelax_step(si.x, si.y, hx, hy, nx, ny);
            st_spin(sp + (int64_t)i * R + r, make_float2(nx, ny));
        }
        if (FUSE) {
            acc[kObsE] -= nx * lx + ny * ly;
            acc[kObsMx] += nx;
            acc[kObsMy] += ny;
            if (fourier) {
                const float4 ph = __ldg(reinterpret_cast<const float4 *>(P.phase) + d.site_off + i);
                acc[kObsF1xRe] += nx * ph.x; acc[kObsF1xIm] += nx * ph.y;
                acc[kObsF1yRe] += ny * ph.x; acc[kObsF1yIm] += ny * ph.y;
                acc[kObsF2xRe] += nx * ph.z; acc[kObsF2xIm] += nx * ph.w;
                acc[kObsF2yRe] += ny * ph.z; acc[kObsF2yIm] += ny * ph.w;
            }
        }
    }
    // lanes l and l ^ o (o >= Rg) hold the same replica
    if (IS_MET) {
        for (int o = 16; o >= bp.Rg; o >>= 1) n_acc += __shfl_xor_sync(0xffffffffu, n_acc, o);
        if ((threadIdx.x & 31) < bp.Rg && n_acc) atomicAdd(&sh.met[rl], (unsigned long long)n_acc);
    }
    if (FUSE) {
        const int nf = fourier ? kObsCount : kObsMy + 1;
        for (int f = 0; f < nf; ++f) {
            float v = acc[f];
            for (int o = 16; o >= bp.Rg; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if ((threadIdx.x & 31) < bp.Rg) atomicAdd(&sh.obs[rl][f], (double)v);
        }
    }
}

template <bool STAGED>
__device__ __forceinline__ void run_sweeps(const DevPlan &P, const BatchedParams &bp, SharedState &sh,
                                           const Staged &stg, cg::cluster_group &cluster, int s, int group,
                                           int rank)
{
    const DevSample d = P.samples[s];
    const int R = d.R;
    const int n_groups = R / bp.Rg;
    const bool leader = (group == 0 && rank == 0);
    uint32_t t = P.sweep[s];
    const bool met = bp.ops & XYL_OP_MET, orx = bp.ops & XYL_OP_OR;
    for (int it = 0; it < bp.n_sweeps; ++it) {
        const bool measure = (bp.ops & XYL_OP_MEASURE) && bp.measure_every > 0 &&
                             ((t + 1u) % (uint32_t)bp.measure_every) == 0u;
        if (met) {
            for (int c = 0; c < d.Q; ++c) {
                if (orx) phase<true, false, STAGED>(P, d, sh, bp, stg, group, c, t, false);
                else phase<true, true, STAGED>(P, d, sh, bp, stg, group, c, t, measure);
                cluster.sync();
            }
        }
        if (orx) {
            for (int c = 0; c < d.Q; ++c) {
                phase<false, true, STAGED>(P, d, sh, bp, stg, group, c, t, measure);
                cluster.sync();
            }
        }
        // publish this CTA's partial sums and acceptance counts
        const int buf = (int)(t & 1u);
        double *obs_s = P.obs + ((size_t)buf * P.total_R + d.rep_off) * kObsStride;
        for (int q = threadIdx.x; q < bp.Rg * kObsCount; q += blockDim.x) {
            const int rl = q / kObsCount, f = q % kObsCount;
            const double v = sh.obs[rl][f];
            if (v != 0.0) atomicAdd(obs_s + (size_t)(group * bp.Rg + rl) * kObsStride + f, v);
            sh.obs[rl][f] = 0.0;
        }
        if (met && threadIdx.x < bp.Rg) {
            const int r = group * bp.Rg + threadIdx.x;
            if (sh.met[threadIdx.x]) atomicAdd(&P.met_acc[d.rep_off + sh.slot_of[r]], sh.met[threadIdx.x]);
            sh.met[threadIdx.x] = 0ull;
        }
        cluster.sync();
        if (n_groups > 1) {
            if (rank == 0 && threadIdx.x == 0) {
                __threadfence();
                atomicAdd(&P.barrier[s], 1u);
                if (!wait_counter_at_least(&P.barrier[s], (unsigned int)(n_groups * (it + 1)), kBarrierPolls)) {
                    atomicExch(P.status, XYL_ETIMEOUT);
                    sh.abort_flag = 1;
                }
                __threadfence();
            }
            cluster.sync();
            // the decision comes from rank 0's shared flag so that every CTA of
            // the cluster takes the same branch (a cluster barrier has no timeout)
            const int *flag0 = cluster.map_shared_rank(&sh.abort_flag, 0);
            const int abort_now = *(volatile const int *)flag0;
            cluster.sync();  // rank 0 stays resident until every CTA has read its flag
            if (abort_now) break;
        }
        for (int k = threadIdx.x; k < R; k += blockDim.x) sh.E[k] = __ldcg(obs_s + (size_t)k * kObsStride + kObsE);
        __syncthreads();
        // parallel tempering, identical in every CTA
        if (bp.ops & XYL_OP_PT) {
            for (int p = threadIdx.x; 2 * p + (int)(t & 1u) + 1 < R; p += blockDim.x) {
                const int k = 2 * p + (int)(t & 1u);
                const int a = sh.rep_at[k], b = sh.rep_at[k + 1];
                const double x = (P.beta[d.rep_off + k] - P.beta[d.rep_off + k + 1]) * (sh.E[a] - sh.E[b]);
                const Words4 w = philox_draw((uint32_t)k, t, kPurposePt, 0u, d.sample_id, P.key);
                const bool accept = uniform53(w.w0, w.w1) < exp(x);
                if (leader) P.pt_try[d.rep_off + k] += 1ull;
                if (accept) {
                    sh.rep_at[k] = b;
                    sh.rep_at[k + 1] = a;
                    sh.slot_of[b] = k;
                    sh.slot_of[a] = k + 1;
                    if (leader) P.pt_acc[d.rep_off + k] += 1ull;
                }
            }
            __syncthreads();
        }
        if (leader) {
            const double invN = 1.0 / (double)d.N;
            for (int k = threadIdx.x; k < R; k += blockDim.x) {
                const int r = sh.rep_at[k];
                P.rep_at[d.rep_off + k] = r;
                P.slot_of[d.rep_off + r] = k;
                P.last_E[d.rep_off + k] = sh.E[k];
                if (met) P.met_try[d.rep_off + k] += (unsigned long long)d.N;
                if (measure) {
                    const double *o = obs_s + (size_t)r * kObsStride;
                    double ov[kObsCount];
#pragma unroll
                    for (int f = 0; f < kObsCount; ++f) ov[f] = __ldcg(o + f);
                    const double e = ov[kObsE] * invN;
                    const double mx = ov[kObsMx] * invN, my = ov[kObsMy] * invN;
                    const double m2 = mx * mx + my * my;
                    const double f1 = ov[kObsF1xRe] * ov[kObsF1xRe] + ov[kObsF1xIm] * ov[kObsF1xIm] +
                                      ov[kObsF1yRe] * ov[kObsF1yRe] + ov[kObsF1yIm] * ov[kObsF1yIm];
                    const double f2 = ov[kObsF2xRe] * ov[kObsF2xRe] + ov[kObsF2xIm] * ov[kObsF2xIm] +
                                      ov[kObsF2yRe] * ov[kObsF2yRe] + ov[kObsF2yIm] * ov[kObsF2yIm];
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
                }
            }
        }
        // clear this group's slots of the buffer the next sweep fills: every
        // reader of it finished before the barrier just passed
        if (rank == 0) {
            double *nxt = P.obs + ((size_t)(buf ^ 1) * P.total_R + d.rep_off + group * bp.Rg) * kObsStride;
            for (int q = threadIdx.x; q < bp.Rg * kObsStride; q += blockDim.x) nxt[q] = 0.0;
        }
        ++t;
        cluster.sync();
    }
    if (leader && threadIdx.x == 0) P.sweep[s] = t;
}

__global__ void __launch_bounds__(1024) batched_kernel(DevPlan P, BatchedParams bp)
{
    __shared__ SharedState sh;
    extern __shared__ int dyn[];
    cg::cluster_group cluster = cg::this_cluster();
    const int unit = bp.unit_begin + (int)(blockIdx.x / bp.G);
    const int rank = (int)cluster.block_rank();
    const int2 ug = bp.units[unit];
    const int s = ug.x, group = ug.y;
    const DevSample d = P.samples[s];
    const int R = d.R;

    for (int k = threadIdx.x; k < R; k += blockDim.x) {
        sh.slot_of[k] = P.slot_of[d.rep_off + k];
        sh.rep_at[k] = P.rep_at[d.rep_off + k];
        sh.beta[k] = (float)P.beta[d.rep_off + k];
        sh.delta[k] = (float)P.delta[d.rep_off + k];
    }
    for (int q = threadIdx.x; q < 32 * kObsStride; q += blockDim.x) (&sh.obs[0][0])[q] = 0.0;
    if (threadIdx.x < 32) sh.met[threadIdx.x] = 0ull;
    if (threadIdx.x == 0) {
        sh.abort_flag = 0;
        // this CTA's chunk of every colour class
        int base = 0;
        for (int c = 0; c < d.Q; ++c) {
            const int cb = P.color_ptr[d.color_off + c], ce = P.color_ptr[d.color_off + c + 1];
            const int chunk = (ce - cb + bp.G - 1) / bp.G;
            const int lo = min(ce, cb + rank * chunk), hi = min(ce, lo + chunk);
            sh.cls_cb[c] = cb;
            sh.cls_lo[c] = lo;
            sh.cls_hi[c] = hi;
            sh.cls_base[c] = base;
            base += hi - lo;
        }
        sh.cls_cb[d.Q] = P.color_ptr[d.color_off + d.Q];
    }
    __syncthreads();

    Staged stg{nullptr, nullptr, nullptr};
    if (bp.staged) {
        int *col = dyn;
        int *deg = col + (size_t)bp.owned_max * bp.max_deg;
        int *site = deg + bp.owned_max;
        for (int c = 0; c < d.Q; ++c) {
            const int lo = sh.cls_lo[c], n = sh.cls_hi[c] - lo, base = sh.cls_base[c];
            for (int q = threadIdx.x; q < n; q += blockDim.x) {
                const int i = lo + q, l = base + q;
                const int rb = P.row_ptr[d.row_off + i], re = P.row_ptr[d.row_off + i + 1];
                deg[l] = re - rb;
                site[l] = P.perm[d.site_off + i];
                for (int k = 0; k < re - rb; ++k) col[(size_t)l * bp.max_deg + k] = P.col[d.col_off + rb + k];
            }
        }
        stg = Staged{col, deg, site};
        __syncthreads();
        run_sweeps<true>(P, bp, sh, stg, cluster, s, group, rank);
    } else {
        run_sweeps<false>(P, bp, sh, stg, cluster, s, group, rank);
    }
}

// Function-wide attributes, the same for every plan: clusters up to 16 CTAs and
// dynamic shared memory up to the staging ceiling (a launch asks for less).
cudaError_t set_kernel_attributes(const BatchedShape &)
{
    cudaError_t e = cudaFuncSetAttribute(batched_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(batched_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kStageLimitBytes);
    return e;
}

// Scratch for xyl_sweep_noalloc: a fixed array in every GPU's global memory
// while the library is loaded.  Host code never dereferences this name; it
// asks the runtime for the device address (see batched_noalloc_scratch).
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

}  // namespace

size_t batched_static_smem_bytes() { return sizeof(SharedState); }

// Device address of the static scratch array on the current device.  The first
// call on a device looks it up (with that device current) and caches it.
cudaError_t batched_noalloc_scratch(void **ptr)
{
    static std::mutex mu;
    static void *addr[kMaxDevicesNoAlloc] = {};
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevicesNoAlloc) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(mu);
    if (!addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        addr[dev] = p;
    }
    *ptr = addr[dev];
    return cudaSuccess;
}

// Also sets the kernel attributes the shape needs; call before the first launch.
cudaError_t batched_max_active_clusters(const PlanShape &, const BatchedShape &B, int *clusters)
{
    cudaError_t e = set_kernel_attributes(B);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    cfg.gridDim = dim3(B.G, 1, 1);
    cfg.blockDim = dim3(B.block, 1, 1);
    cfg.dynamicSmemBytes = B.smem_bytes;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = B.G;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaOccupancyMaxActiveClusters(clusters, batched_kernel, &cfg);
}

cudaError_t launch_batched(const DevPlan &P, const PlanShape &, const BatchedShape &B, const int2 *d_units,
                           int unit_begin, int unit_count, int n_sweeps, uint32_t ops, int measure_every,
                           cudaStream_t st)
{
    if (unit_count <= 0) return cudaSuccess;
    BatchedParams bp;
    bp.units = d_units;
    bp.unit_begin = unit_begin;
    bp.G = B.G;
    bp.Rg = B.Rg;
    bp.log2Rg = 0;
    while ((1 << bp.log2Rg) < B.Rg) ++bp.log2Rg;
    bp.n_sweeps = n_sweeps;
    bp.ops = ops;
    bp.measure_every = measure_every;
    bp.staged = B.staged ? 1 : 0;
    bp.owned_max = B.owned_max;
    bp.max_deg = B.max_deg;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    cfg.gridDim = dim3((unsigned)(B.G * unit_count), 1, 1);
    cfg.blockDim = dim3((unsigned)B.block, 1, 1);
    cfg.dynamicSmemBytes = B.smem_bytes;
    cfg.stream = st;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = B.G;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, batched_kernel, P, bp);
}

}  // namespace xyl
