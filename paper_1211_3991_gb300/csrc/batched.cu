// Batched FP32 engine: one launch runs many whole sweep + swap + measure
// cycles for a batch of samples.
//
// Work decomposition.  The replicas of a sample are split into groups of Rg
// (a power of two, or an even divisor of the sample's replica count, up to
// 32).  Each (sample, group)
// unit is owned by one thread-block cluster of G CTAs.  Inside a unit, every
// colour class is cut into G contiguous chunks; CTA k updates chunk k for all
// Rg replicas.  A thread updates RV replicas (2 when Rg is even, else 1) of
// one site per item; the lps = Rg / RV lanes of a site are consecutive
// threads, so they read one contiguous Rg x 8-byte segment of each
// neighbour's row.  Thread t serves lane t % lps of sites t / lps, t / lps +
// spr, ... (spr = block / lps sites per round; with lps not a power of two the
// last block % lps threads idle).
// With span > 1 a unit is G x span CTAs in span clusters, which meet after
// every colour phase at a bounded barrier on a per-unit counter in global
// memory (the whole GPU can then work on one sample while its spins stay in
// L2 for the launch's sweeps).
// Spins are interleaved [sample][site][replica] float2 in global memory; they
// stay L2-resident while the units resident at once fit L2 (a launch wave of
// whole samples, or the clusters that fit when units never wait on one
// another, each running all the launch's sweeps on its unit); they are read and
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
#include "sweep_tail.cuh"

namespace cg = cooperative_groups;

namespace xyl {
namespace {

constexpr unsigned int kBarrierPolls = 1u << 21;  // about a second of polling

struct BatchedParams {
    const int2 *units;   // (sample, group) per unit
    unsigned int *unit_ctr;  // span > 1: per unit of the launch, arrivals at its phase barriers (zeroed before)
    int unit_begin;
    int G, Rg;
    int span;            // clusters per unit (G x span CTAs share a unit's colour chunks)
    int rv;              // replicas one thread updates (1 or 2)
    int lps;             // lanes that share a site (Rg / rv)
    int log2lps;         // log2(lps) when lps is a power of two
    int spr;             // sites per round: block / lps
    int act;             // threads with a lane: spr * lps
    int pow2;            // lps is a power of two: a site's lanes tile every warp (warp-shuffle sums)
    int n_sweeps;
    uint32_t ops;
    int measure_every;
    int staged;          // CSR rows / site ids of the CTA's chunks in shared memory
    int owned_max;       // largest number of sites one CTA owns
    int max_deg;
    int fixed_deg;       // degree of every site of every sample, 0 if degrees differ
};

__device__ __forceinline__ float2 ld_spin(const float2 *p) { return __ldcg(p); }
__device__ __forceinline__ void st_spin(float2 *p, float2 v) { __stcg(p, v); }
__device__ __forceinline__ float4 ld_spin2(const float2 *p) { return __ldcg(reinterpret_cast<const float4 *>(p)); }
__device__ __forceinline__ void st_spin2(float2 *p, float4 v) { __stcg(reinterpret_cast<float4 *>(p), v); }

// Per-CTA sums of one sweep, per replica of the group: the energy of links to
// lower colours (fused into the overrelaxation pass) and, on measurement
// sweeps, magnetisation and Fourier sums (one extra pass over the CTA's sites).
constexpr int kSums = kObsCount;

constexpr int kMaxWarps = 21;      // 672 threads per CTA at most with 96 registers each
constexpr int kMaxWarpsWide = 32;  // 1024 threads with 64 registers each (rows in global memory only)

template <int MW>
struct SharedStateT {
    float part[kSums][MW][32];      // per field, warp, group replica: warp partial sums
    unsigned int part_met[MW][32];  // per warp, group replica: accepted Metropolis moves
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
using SharedState = SharedStateT<kMaxWarps>;

struct Staged {
    const int *col;      // [owned_max][max_deg] colour-sorted neighbour ids
    const int *deg;      // [owned_max]
    const int *site_id;  // [owned_max] original ids (random-stream keys)
};

// What one thread needs about its replicas during a sweep.
// This thread's first site within a chunk (a large value: no lane); it is
// recomputed where needed rather than kept live through the sweep.
__device__ __forceinline__ int first_site(const BatchedParams &bp)
{
    if ((int)threadIdx.x >= bp.act) return 0x3fffffff;
    return bp.pow2 ? (int)threadIdx.x >> bp.log2lps : (int)threadIdx.x / bp.lps;
}

// A thread's items of one colour chunk of n sites.  NP2 = false (lps a power
// of two): item q = site offset x lps + lane, q = thread, thread + block, ...;
// NP2 = true: site offsets first_site, first_site + spr, ...
template <bool NP2>
struct ItemIter;

template <>
struct ItemIter<false> {
    int q, items;
    __device__ __forceinline__ ItemIter(const BatchedParams &bp, int n)
        : q((int)threadIdx.x), items(n > 0 ? n << bp.log2lps : 0) {}
    __device__ __forceinline__ bool ok() const { return q < items; }
    __device__ __forceinline__ int off(const BatchedParams &bp) const { return q >> bp.log2lps; }
    __device__ __forceinline__ bool first() const { return q == (int)threadIdx.x; }
    __device__ __forceinline__ bool next_ok() const { return q + (int)blockDim.x < items; }
    __device__ __forceinline__ int next_off(const BatchedParams &bp) const { return (q + (int)blockDim.x) >> bp.log2lps; }
    __device__ __forceinline__ void step(const BatchedParams &) { q += (int)blockDim.x; }
};

template <>
struct ItemIter<true> {
    int o, n, spr;
    __device__ __forceinline__ ItemIter(const BatchedParams &bp, int n_) : o(first_site(bp)), n(n_), spr(bp.spr) {}
    __device__ __forceinline__ bool ok() const { return o < n; }
    __device__ __forceinline__ int off(const BatchedParams &) const { return o; }
    __device__ __forceinline__ bool first() const { return o < spr; }
    __device__ __forceinline__ bool next_ok() const { return o + spr < n; }
    __device__ __forceinline__ int next_off(const BatchedParams &) const { return o + spr; }
    __device__ __forceinline__ void step(const BatchedParams &) { o += spr; }
};

template <int RV>
struct Lane {
    int r0;              // first replica this thread updates (absolute within the sample)
    float beta[RV], delta[RV];
    float e[RV];         // energy partial sums (fused)
    unsigned int acc[RV];
};

template <int RV>
__device__ __forceinline__ void load_spins(const float2 *row, float2 (&v)[RV])
{
    if constexpr (RV == 2) {
        const float4 q = ld_spin2(row);
        v[0] = make_float2(q.x, q.y);
        v[1] = make_float2(q.z, q.w);
    } else {
        v[0] = ld_spin(row);
    }
}

template <int RV>
__device__ __forceinline__ void store_spins(float2 *row, const float2 (&v)[RV])
{
    if constexpr (RV == 2)
        st_spin2(row, make_float4(v[0].x, v[0].y, v[1].x, v[1].y));
    else
        st_spin(row, v[0]);
}

// One colour phase of one pass for this CTA's chunk: one thread per (site,
// block of RV consecutive replicas).
// Philox block of this thread's first item in colour c (Metropolis pass).
template <bool STAGED, bool NP2, class SS>
__device__ __forceinline__ Words4 first_draw(const DevPlan &P, const DevSample &d, const SS &sh,
                                             const BatchedParams &bp, const Staged &stg, int c, uint32_t t, int r0)
{
    const int lo = sh.cls_lo[c], hi = sh.cls_hi[c];
    const ItemIter<NP2> it(bp, hi - lo);
    Words4 x{0u, 0u, 0u, 0u};
    if (it.ok()) {
        const int o0 = it.off(bp);
        const uint32_t site = STAGED ? (uint32_t)stg.site_id[sh.cls_base[c] + o0]
                                     : (uint32_t)__ldg(P.perm + d.site_off + lo + o0);
        x = met_block_f32(site, t, r0, d.sample_id, P.key);
    }
    return x;
}

// Where the neighbour ids of one item come from, and its random-stream key;
// fetched one item ahead of its use so that an update waits on one memory
// round trip (its neighbours' spins), not three.
template <int DEG>
struct GRow {
    int nb[DEG > 0 ? DEG : 1];  // fixed degree, rows in global memory: the ids themselves
    int rb, deg;                 // otherwise: the row's start (staged rows or global CSR) and length
    uint32_t key;
};

template <bool IS_MET, bool STAGED, int DEG>
__device__ __forceinline__ void fetch_grow(const DevPlan &P, const DevSample &d, const BatchedParams &bp,
                                           const Staged &stg, int i, int l, GRow<DEG> &row)
{
    if (STAGED) {
        row.rb = l * bp.max_deg;
        row.deg = DEG > 0 ? DEG : stg.deg[l];
        if (IS_MET) row.key = (uint32_t)stg.site_id[l];
    } else if (DEG > 0) {
        // every row holds DEG ids and starts at DEG * i: no row_ptr read; the
        // rows of a sample start at an even offset, so ids come in pairs
        const int2 *c = reinterpret_cast<const int2 *>(P.col + d.col_off + (int64_t)DEG * i);
#pragma unroll
        for (int k = 0; k < DEG / 2; ++k) {
            const int2 w = __ldg(c + k);
            row.nb[2 * k] = w.x;
            row.nb[2 * k + 1] = w.y;
        }
        row.deg = DEG;
        if (IS_MET) row.key = (uint32_t)__ldg(P.perm + d.site_off + i);
    } else {
        row.rb = __ldg(P.row_ptr + d.row_off + i);
        row.deg = checked_id(P, __ldg(P.row_ptr + d.row_off + i + 1) - row.rb, bp.max_deg + 1, 0);
        if (IS_MET) row.key = (uint32_t)__ldg(P.perm + d.site_off + i);
    }
}

template <bool IS_MET, bool FUSE_E, bool STAGED, int RV, int DEG, bool DISORDER, bool NP2, class SS>
__device__ __forceinline__ void phase(const DevPlan &P, const DevSample &d, const SS &sh,
                                      const BatchedParams &bp, const Staged &stg, int c, uint32_t t, Lane<RV> &ln,
                                      const Words4 &first)
{
    const int cb = sh.cls_cb[c];
    const int lo = sh.cls_lo[c], hi = sh.cls_hi[c], base = sh.cls_base[c];
    const int n = hi - lo;
    const int R = d.R;
    const float2 *sp = reinterpret_cast<const float2 *>(P.spins) + d.spin_off + ln.r0;
    float2 *spw = reinterpret_cast<float2 *>(P.spins) + d.spin_off + ln.r0;
    const int32_t *cl = P.col + d.col_off;

    ItemIter<NP2> it(bp, n);
    if (!it.ok()) return;
    // rows staged in shared memory are read where they are used; rows in
    // global memory one item ahead
    GRow<DEG> cur;
    if (!STAGED) fetch_grow<IS_MET, STAGED, DEG>(P, d, bp, stg, lo + it.off(bp), 0, cur);
    for (; it.ok(); it.step(bp)) {
        const int o = it.off(bp);
        const int i = lo + o;
        GRow<DEG> nxt;
        if (STAGED)
            fetch_grow<IS_MET, STAGED, DEG>(P, d, bp, stg, i, base + o, cur);
        else if (it.next_ok())
            fetch_grow<IS_MET, STAGED, DEG>(P, d, bp, stg, lo + it.next_off(bp), 0, nxt);
        float2 s[RV];
        load_spins<RV>(sp + i * R, s);
        float hx[RV], hy[RV], lx[RV], ly[RV];
#pragma unroll
        for (int v = 0; v < RV; ++v) hx[v] = hy[v] = lx[v] = ly[v] = 0.f;
        // with DISORDER, a neighbour id with its top bit set is a link with J = -1
        auto gather = [&](int raw) {
            const int j = checked_id(P, DISORDER ? (raw & 0x7fffffff) : raw, d.N, 0);
            float2 sj[RV];
            load_spins<RV>(sp + j * R, sj);
            if (DISORDER && raw < 0) {
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
        };
        if (DEG > 0) {
            // every site has exactly DEG links
#pragma unroll
            for (int k = 0; k < DEG; ++k) gather(STAGED ? stg.col[cur.rb + k] : cur.nb[k]);
        } else if (DEG < 0) {
            // at most -DEG links
#pragma unroll
            for (int k = 0; k < -DEG; ++k)
                if (k < cur.deg) gather(STAGED ? stg.col[cur.rb + k] : __ldg(cl + cur.rb + k));
        } else {
            for (int k = 0; k < cur.deg; ++k) gather(STAGED ? stg.col[cur.rb + k] : __ldg(cl + cur.rb + k));
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
            const Words4 x = it.first() ? first : met_block_f32(cur.key, t, ln.r0, d.sample_id, P.key);
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
            if (any) store_spins<RV>(spw + i * R, n);
        } else {
#pragma unroll
            for (int v = 0; v < RV; ++v) overrelax_step(s[v].x, s[v].y, hx[v], hy[v], n[v].x, n[v].y);
            store_spins<RV>(spw + i * R, n);
        }
        if (FUSE_E) {
#pragma unroll
            for (int v = 0; v < RV; ++v) ln.e[v] -= n[v].x * lx[v] + n[v].y * ly[v];
        }
        if (!STAGED) cur = nxt;
    }
}

// Warp partial of a per-thread value of replica lane_rep+v (lps a power of
// two: lanes l and l ^ o, o >= lps, hold the same replicas), stored per warp
// so that the CTA sum is taken in a fixed order.
template <class SS>
__device__ __forceinline__ void warp_part(SS &sh, const BatchedParams &bp, int lane_rep, int v, int f, float x)
{
    for (int o = 16; o >= (1 << bp.log2lps); o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if ((threadIdx.x & 31) < (1 << bp.log2lps)) sh.part[f][threadIdx.x >> 5][lane_rep + v] = x;
}

template <class SS>
__device__ __forceinline__ void warp_count(SS &sh, const BatchedParams &bp, int lane_rep, int v, unsigned x)
{
    for (int o = 16; o >= (1 << bp.log2lps); o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if ((threadIdx.x & 31) < (1 << bp.log2lps)) sh.part_met[threadIdx.x >> 5][lane_rep + v] = x;
}

// lps not a power of two: the CTA sum of one per-thread value per replica of
// the group, in thread order (so it is the same on every run), added to field
// f of the group's slots.  The warp partial array serves as scratch (it holds
// kSums x 32 floats per warp, at least RV per thread).  Called by every thread.
template <int RV, class SS>
__device__ __forceinline__ void cta_sum_np2(SS &sh, const BatchedParams &bp, const float (&x)[RV], double *obs_g,
                                            int f)
{
    float *tp = &sh.part[0][0][0];
    const int n = (int)blockDim.x;
#pragma unroll
    for (int v = 0; v < RV; ++v) tp[v * n + threadIdx.x] = (int)threadIdx.x < bp.act ? x[v] : 0.f;
    __syncthreads();
    if ((int)threadIdx.x < bp.Rg) {
        const int v = (int)threadIdx.x % RV, lane = (int)threadIdx.x / RV;
        float s = 0.f;
        for (int k = lane; k < bp.act; k += bp.lps) s += tp[v * n + k];
        atomicAdd(obs_g + (size_t)threadIdx.x * kObsStride + f, (double)s);
    }
    __syncthreads();
}

template <int RV, class SS>
__device__ __forceinline__ void cta_count_np2(SS &sh, const BatchedParams &bp, const unsigned (&x)[RV],
                                              unsigned long long *met_acc, int r_base)
{
    unsigned *tp = reinterpret_cast<unsigned *>(&sh.part[0][0][0]);
    const int n = (int)blockDim.x;
#pragma unroll
    for (int v = 0; v < RV; ++v) tp[v * n + threadIdx.x] = (int)threadIdx.x < bp.act ? x[v] : 0u;
    __syncthreads();
    if ((int)threadIdx.x < bp.Rg) {
        const int v = (int)threadIdx.x % RV, lane = (int)threadIdx.x / RV;
        unsigned s = 0;
        for (int k = lane; k < bp.act; k += bp.lps) s += tp[v * n + k];
        if (s) atomicAdd(&met_acc[sh.slot_of[r_base + threadIdx.x]], (unsigned long long)s);
    }
    __syncthreads();
}

// Magnetisation and Fourier sums of the CTA's own sites (final spins), as warp
// partials (lps a power of two) or added to the group's slots of obs_g.
template <int RV, bool NP2, class SS>
__device__ __forceinline__ void measure_own_sites(const DevPlan &P, const DevSample &d, SS &sh,
                                                  const BatchedParams &bp, int r0, int lane_rep, double *obs_g)
{
    float m[RV][kSums - 1];
#pragma unroll
    for (int v = 0; v < RV; ++v)
#pragma unroll
        for (int f = 0; f < kSums - 1; ++f) m[v][f] = 0.f;
    const float2 *sp = reinterpret_cast<const float2 *>(P.spins) + d.spin_off + r0;
    for (int c = 0; c < d.Q; ++c) {
        const int lo = sh.cls_lo[c], hi = sh.cls_hi[c];
        for (ItemIter<NP2> it(bp, hi - lo); it.ok(); it.step(bp)) {
            const int i = lo + it.off(bp);
            float2 s[RV];
            load_spins<RV>(sp + i * d.R, s);
            const float4 ph = __ldg(reinterpret_cast<const float4 *>(P.phase) + d.site_off + i);
#pragma unroll
            for (int v = 0; v < RV; ++v) {
                m[v][kObsMx - 1] += s[v].x;
                m[v][kObsMy - 1] += s[v].y;
                m[v][kObsF1xRe - 1] += s[v].x * ph.x; m[v][kObsF1xIm - 1] += s[v].x * ph.y;
                m[v][kObsF1yRe - 1] += s[v].y * ph.x; m[v][kObsF1yIm - 1] += s[v].y * ph.y;
                m[v][kObsF2xRe - 1] += s[v].x * ph.z; m[v][kObsF2xIm - 1] += s[v].x * ph.w;
                m[v][kObsF2yRe - 1] += s[v].y * ph.z; m[v][kObsF2yIm - 1] += s[v].y * ph.w;
            }
        }
    }
    if constexpr (!NP2) {
#pragma unroll
        for (int v = 0; v < RV; ++v)
#pragma unroll
            for (int f = 1; f < kSums; ++f) warp_part(sh, bp, lane_rep, v, f, m[v][f - 1]);
    } else {
#pragma unroll
        for (int f = 1; f < kSums; ++f) {
            float x[RV];
#pragma unroll
            for (int v = 0; v < RV; ++v) x[v] = m[v][f - 1];
            cta_sum_np2<RV>(sh, bp, x, obs_g, f);
        }
    }
}

// span > 1: the clusters of a unit meet.  Every thread makes its spin writes
// visible GPU-wide, the cluster synchronises, its first thread adds the
// cluster's arrival to the unit's counter and waits (bounded) until all span
// clusters have arrived at this barrier, then tells its cluster the outcome
// before the cluster synchronises again.  False after a timeout (the status
// word then holds XYL_ETIMEOUT).
template <class SS>
__device__ __forceinline__ bool unit_barrier(const DevPlan &P, SS &sh, cg::cluster_group &cluster,
                                             const BatchedParams &bp, unsigned int *ctr, unsigned int &arrivals,
                                             int rank)
{
    __threadfence();
    cluster.sync();
    arrivals += (unsigned int)bp.span;
    if (rank == 0 && threadIdx.x == 0) {
        atomicAdd(ctr, 1u);
        int failed = 0;
        if (!wait_counter_at_least(ctr, arrivals, kBarrierPolls)) {
            atomicExch(P.status, XYL_ETIMEOUT);
            failed = 1;
        }
        __threadfence();
        for (int k = 0; k < bp.G; ++k) *cluster.map_shared_rank(&sh.abort_flag, k) = failed;
    }
    cluster.sync();
    return *(volatile int *)&sh.abort_flag == 0;
}

template <bool STAGED, int RV, int DEG, bool DISORDER, bool NP2, bool SPAN, class SS>
__device__ __forceinline__ void run_sweeps(const DevPlan &P, const BatchedParams &bp, SS &sh,
                                           const Staged &stg, cg::cluster_group &cluster, int s, int group,
                                           int rank, int cta, unsigned int *unit_ctr)
{
    const DevSample d = P.samples[s];
    const int R = d.R;
    const int n_groups = R / bp.Rg;
    const int ctas = SPAN ? bp.G * bp.span : bp.G;  // CTAs of one unit
    const bool leader = (group == 0 && cta == 0);
    const bool sample_barrier = n_groups > 1 || SPAN;
    unsigned int arrivals = 0;
    // replica offset within the group of this thread's lane (threads past
    // spr * lps have no lane and update nothing)
    const int lane_rep = NP2 ? ((int)threadIdx.x < bp.act ? ((int)threadIdx.x % bp.lps) * RV : 0)
                             : (int)(threadIdx.x & ((1 << bp.log2lps) - 1)) * RV;
    Lane<RV> ln;
    ln.r0 = group * bp.Rg + lane_rep;
    uint32_t t = P.sweep[s];
    const bool met = bp.ops & XYL_OP_MET, orx = bp.ops & XYL_OP_OR;
    Words4 first = first_draw<STAGED, NP2>(P, d, sh, bp, stg, 0, t, ln.r0);
    for (int it = 0; it < bp.n_sweeps; ++it) {
        const bool measure = (bp.ops & XYL_OP_MEASURE) && bp.measure_every > 0 &&
                             ((t + 1u) % (uint32_t)bp.measure_every) == 0u;
#pragma unroll
        for (int v = 0; v < RV; ++v) {
            const int slot = sh.slot_of[ln.r0 + v];
            ln.beta[v] = sh.beta[slot];
            ln.delta[v] = sh.delta[slot];
            ln.e[v] = 0.f;
            ln.acc[v] = 0u;
        }
        if (met) {
            // the next phase's first Philox block is drawn while the cluster
            // barrier of the previous phase completes
            for (int c = 0; c < d.Q; ++c) {
                if (orx) phase<true, false, STAGED, RV, DEG, DISORDER, NP2>(P, d, sh, bp, stg, c, t, ln, first);
                else phase<true, true, STAGED, RV, DEG, DISORDER, NP2>(P, d, sh, bp, stg, c, t, ln, first);
                if (orx || c + 1 < d.Q) {
                    if constexpr (!SPAN) {
                        cluster_arrive();
                        if (c + 1 < d.Q) first = first_draw<STAGED, NP2>(P, d, sh, bp, stg, c + 1, t, ln.r0);
                        cluster_wait();
                    } else {
                        if (c + 1 < d.Q) first = first_draw<STAGED, NP2>(P, d, sh, bp, stg, c + 1, t, ln.r0);
                        if (!unit_barrier(P, sh, cluster, bp, unit_ctr, arrivals, rank)) return;
                    }
                }
            }
        }
        if (orx) {
            const Words4 none{0u, 0u, 0u, 0u};
            for (int c = 0; c < d.Q; ++c) {
                phase<false, true, STAGED, RV, DEG, DISORDER, NP2>(P, d, sh, bp, stg, c, t, ln, none);
                if (c + 1 < d.Q) {
                    if constexpr (!SPAN) cluster.sync();
                    else if (!unit_barrier(P, sh, cluster, bp, unit_ctr, arrivals, rank)) return;
                }
            }
        }
        // this CTA's sums: fused energies, Metropolis counts, and on measurement
        // sweeps the magnetisation and Fourier sums of its own (final) sites;
        // CTA sums in a fixed order (FP32 over at most a few thousand sites),
        // then FP64 across the CTAs of the sample
        const int buf = (int)(t & 1u);
        double *obs_s = P.obs + ((size_t)buf * P.total_R + d.rep_off) * kObsStride;
        double *obs_g = obs_s + (size_t)group * bp.Rg * kObsStride;
        if constexpr (!NP2) {
#pragma unroll
            for (int v = 0; v < RV; ++v) {
                warp_part(sh, bp, lane_rep, v, kObsE, ln.e[v]);
                if (met) warp_count(sh, bp, lane_rep, v, ln.acc[v]);
            }
            if (measure) {
                __syncthreads();  // own sites written by other threads of this CTA
                measure_own_sites<RV, NP2>(P, d, sh, bp, ln.r0, lane_rep, obs_g);
            }
            __syncthreads();
            // per replica: the warp partials in warp order
            const int nf = measure ? kSums : 1;
            const int n_warps = (int)(blockDim.x >> 5);
            for (int q = threadIdx.x; q < bp.Rg * nf; q += blockDim.x) {
                const int rl = q / nf, f = q % nf;
                float v = 0.f;
                for (int w = 0; w < n_warps; ++w) v += sh.part[f][w][rl];
                atomicAdd(obs_g + (size_t)rl * kObsStride + f, (double)v);
            }
            if (met && threadIdx.x < bp.Rg) {
                const int r = group * bp.Rg + threadIdx.x;
                unsigned int n = 0;
                for (int w = 0; w < n_warps; ++w) n += sh.part_met[w][threadIdx.x];
                if (n) atomicAdd(&P.met_acc[d.rep_off + sh.slot_of[r]], (unsigned long long)n);
            }
        } else {
            // per replica: the thread values in thread order
            __syncthreads();  // every thread is past its last phase before the scratch is written
            cta_sum_np2<RV>(sh, bp, ln.e, obs_g, kObsE);
            if (met) cta_count_np2<RV>(sh, bp, ln.acc, P.met_acc + d.rep_off, group * bp.Rg);
            if (measure) measure_own_sites<RV, NP2>(P, d, sh, bp, ln.r0, lane_rep, obs_g);
        }
        if (sample_barrier) {
            // every CTA of the sample signs in once its sums are out; the first
            // CTA of each cluster waits for all of them (bounded) and tells the
            // other CTAs of its cluster the outcome through their shared memory
            __threadfence();
            __syncthreads();
            if (threadIdx.x == 0) atomicAdd(&P.barrier[s], 1u);
            if (rank == 0 && threadIdx.x == 0) {
                int failed = 0;
                if (!wait_counter_at_least(&P.barrier[s], (unsigned int)(ctas * n_groups * (it + 1)), kBarrierPolls)) {
                    atomicExch(P.status, XYL_ETIMEOUT);
                    failed = 1;
                }
                __threadfence();
                for (int k = 0; k < bp.G; ++k) *cluster.map_shared_rank(&sh.abort_flag, k) = failed;
            }
        }
        cluster_arrive();
        if (met) first = first_draw<STAGED, NP2>(P, d, sh, bp, stg, 0, t + 1u, ln.r0);  // next sweep's first draw
        cluster_wait();
        if (sample_barrier && *(volatile int *)&sh.abort_flag) break;
        for (int k = threadIdx.x; k < R; k += blockDim.x) sh.E[k] = __ldcg(obs_s + (size_t)k * kObsStride + kObsE);
        __syncthreads();
        pt_and_record(P, d, sh.E, sh.rep_at, sh.slot_of, t, bp.ops, leader, met, measure, obs_s);
        // clear this group's slots of the buffer the next sweep fills: every
        // reader of it finished before the barrier just passed
        if (cta == 0) {
            double *nxt = P.obs + ((size_t)(buf ^ 1) * P.total_R + d.rep_off + group * bp.Rg) * kObsStride;
            for (int q = threadIdx.x; q < bp.Rg * kObsStride; q += blockDim.x) nxt[q] = 0.0;
        }
        ++t;
        __syncthreads();
    }
    if (leader && threadIdx.x == 0) P.sweep[s] = t;
}

template <bool STAGED, int RV, int DEG, bool DISORDER, bool NP2, bool SPAN, int MW>
__device__ __forceinline__ void batched_body(const DevPlan &P, const BatchedParams &bp)
{
    __shared__ SharedStateT<MW> sh;
    extern __shared__ int dyn[];
    cg::cluster_group cluster = cg::this_cluster();
    const int ctas = SPAN ? bp.G * bp.span : bp.G;    // CTAs of one unit, span clusters
    const int unit = bp.unit_begin + (int)(blockIdx.x / ctas);
    const int cta = (int)(blockIdx.x % ctas);         // which chunk of the unit's classes
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
    if (threadIdx.x == 0) {
        sh.abort_flag = 0;
        // this CTA's chunk of every colour class
        int base = 0;
        for (int c = 0; c < d.Q; ++c) {
            int cb = P.color_ptr[d.color_off + c], ce = P.color_ptr[d.color_off + c + 1];
            checked_class(P, cb, ce, d.N);
            const int chunk = (ce - cb + ctas - 1) / ctas;
            const int lo = min(ce, cb + cta * chunk), hi = min(ce, lo + chunk);
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
    if (STAGED) {
        int *col = dyn;
        int *deg = col + (size_t)bp.owned_max * bp.max_deg;
        int *site = deg + bp.owned_max;
        for (int c = 0; c < d.Q; ++c) {
            const int lo = sh.cls_lo[c], n = sh.cls_hi[c] - lo, base = sh.cls_base[c];
            for (int q = threadIdx.x; q < n; q += blockDim.x) {
                const int i = lo + q, l = base + q;
                const int rb = P.row_ptr[d.row_off + i];
                const int n_k = checked_id(P, P.row_ptr[d.row_off + i + 1] - rb, bp.max_deg + 1, 0);
                deg[l] = n_k;
                site[l] = P.perm[d.site_off + i];
                for (int k = 0; k < n_k; ++k) col[(size_t)l * bp.max_deg + k] = P.col[d.col_off + rb + k];
            }
        }
        stg = Staged{col, deg, site};
        __syncthreads();
    }
    run_sweeps<STAGED, RV, DEG, DISORDER, NP2, SPAN>(P, bp, sh, stg, cluster, s, group, rank, cta,
                                               bp.unit_ctr + (unit - bp.unit_begin));
}

// Up to 672 threads with 96 registers each, or, rows in global memory only,
// up to 1024 threads with 64 registers each (more warps to cover the latency
// of the neighbour gathers).
// NP2: lanes per site not a power of two (even groups of 6, 10, 12, ... replicas).
// SPAN: a unit spans several clusters (phase barriers through global memory).
template <bool STAGED, int RV, int DEG, bool DISORDER, bool NP2, bool SPAN>
__global__ void __maxnreg__(96) batched_kernel(DevPlan P, BatchedParams bp)
{
    batched_body<STAGED, RV, DEG, DISORDER, NP2, SPAN, kMaxWarps>(P, bp);
}

template <int RV, int DEG, bool DISORDER, bool NP2, bool SPAN>
__global__ void __launch_bounds__(1024, 1) batched_kernel_wide(DevPlan P, BatchedParams bp)
{
    batched_body<false, RV, DEG, DISORDER, NP2, SPAN, kMaxWarpsWide>(P, bp);
}

using KernelFn = void (*)(DevPlan, BatchedParams);

// The specialisation for a launch shape: CSR staged or not, one or two
// replicas per thread, fixed degree 6 / at most 8 / any degree, random bonds or
// fields, lanes per site a power of two or not, one cluster per unit or several.
template <bool STAGED, int RV, bool DISORDER, bool NP2, bool SPAN>
KernelFn pick_deg(const BatchedShape &B)
{
    if (!STAGED && B.block > kMaxWarps * 32) {
        if (B.fixed_deg == 6) return batched_kernel_wide<RV, 6, DISORDER, NP2, SPAN>;
        if (B.max_deg <= 8) return batched_kernel_wide<RV, -8, DISORDER, NP2, SPAN>;
        return batched_kernel_wide<RV, 0, DISORDER, NP2, SPAN>;
    }
    if (B.fixed_deg == 6) return batched_kernel<STAGED, RV, 6, DISORDER, NP2, SPAN>;
    if (B.max_deg <= 8) return batched_kernel<STAGED, RV, -8, DISORDER, NP2, SPAN>;
    return batched_kernel<STAGED, RV, 0, DISORDER, NP2, SPAN>;
}

template <bool DISORDER>
KernelFn pick_kernel_d(const BatchedShape &B)
{
    // groups are a power of two (one or two replicas a thread) or even (two);
    // a unit over several clusters takes a power of two of at least two
    const bool rv2 = B.Rg % 2 == 0;
    const int lps = rv2 ? B.Rg / 2 : B.Rg;
    if (B.span > 1)
        return B.staged ? pick_deg<true, 2, DISORDER, false, true>(B) : pick_deg<false, 2, DISORDER, false, true>(B);
    if (lps & (lps - 1))
        return B.staged ? pick_deg<true, 2, DISORDER, true, false>(B) : pick_deg<false, 2, DISORDER, true, false>(B);
    if (B.staged)
        return rv2 ? pick_deg<true, 2, DISORDER, false, false>(B) : pick_deg<true, 1, DISORDER, false, false>(B);
    return rv2 ? pick_deg<false, 2, DISORDER, false, false>(B) : pick_deg<false, 1, DISORDER, false, false>(B);
}

KernelFn pick_kernel(const BatchedShape &B) { return B.disorder ? pick_kernel_d<true>(B) : pick_kernel_d<false>(B); }

// Function-wide attributes, the same for every plan: clusters up to 16 CTAs and
// dynamic shared memory up to the staging ceiling (a launch asks for less).
cudaError_t set_kernel_attributes(KernelFn k)
{
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kStageLimitBytes);
    return e;
}

// Scratch for xyl_sweep_noalloc: a fixed array in every GPU's global memory
// while the library is loaded.  Host code never dereferences this name; it
// asks the runtime for the device address (see batched_noalloc_scratch).
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

}  // namespace

size_t batched_static_smem_bytes() { return sizeof(SharedStateT<kMaxWarpsWide>); }

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
    const KernelFn kernel = pick_kernel(B);
    cudaError_t e = set_kernel_attributes(kernel);
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
    return cudaOccupancyMaxActiveClusters(clusters, kernel, &cfg);
}

cudaError_t launch_batched(const DevPlan &P, const PlanShape &, const BatchedShape &B, const int2 *d_units,
                           unsigned int *unit_ctr, int unit_begin, int unit_count, int n_sweeps, uint32_t ops,
                           int measure_every, cudaStream_t st)
{
    if (unit_count <= 0) return cudaSuccess;
    if (B.span > 1) {
        // the phase barriers count arrivals from zero in every launch
        const cudaError_t e = cudaMemsetAsync(unit_ctr, 0, (size_t)unit_count * sizeof(unsigned int), st);
        if (e != cudaSuccess) return e;
    }
    BatchedParams bp;
    bp.units = d_units;
    bp.unit_ctr = unit_ctr;
    bp.unit_begin = unit_begin;
    bp.span = B.span;
    bp.G = B.G;
    bp.Rg = B.Rg;
    bp.rv = (B.Rg % 2 == 0) ? 2 : 1;
    bp.lps = B.Rg / bp.rv;
    bp.spr = B.block / bp.lps;
    bp.act = bp.spr * bp.lps;
    bp.pow2 = (bp.lps & (bp.lps - 1)) == 0 ? 1 : 0;
    bp.log2lps = 0;
    while ((1 << bp.log2lps) < bp.lps) ++bp.log2lps;
    bp.n_sweeps = n_sweeps;
    bp.ops = ops;
    bp.measure_every = measure_every;
    bp.staged = B.staged ? 1 : 0;
    bp.owned_max = B.owned_max;
    bp.max_deg = B.max_deg;
    bp.fixed_deg = B.fixed_deg;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    cfg.gridDim = dim3((unsigned)(B.G * B.span * unit_count), 1, 1);
    cfg.blockDim = dim3((unsigned)B.block, 1, 1);
    cfg.dynamicSmemBytes = B.smem_bytes;
    cfg.stream = st;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = B.G;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, pick_kernel(B), P, bp);
}

}  // namespace xyl
