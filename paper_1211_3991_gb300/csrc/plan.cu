// C ABI of libxyl: plans, workspace layout, bind, sweeps (captured into CUDA
// graphs), standalone PT / measurement / recompute, read-back and checkpoint.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <tuple>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "engines.h"
#include "internal.h"

// A named NVTX range over one library call: profilers that read NVTX (ncu
// --nvtx) see each call's launches under its name; without a tool attached
// the push and pop cost next to nothing.
struct CallRange {
    explicit CallRange(const char *name) { nvtxRangePushA(name); }
    ~CallRange() { nvtxRangePop(); }
    CallRange(const CallRange &) = delete;
    CallRange &operator=(const CallRange &) = delete;
};

using namespace xyl;

namespace {

struct HostSample {
    int32_t N = 0, Q = 0, R = 0, L = 0, max_deg = 0;
    uint32_t sample_id = 0;
    std::vector<double> beta, delta;
    std::vector<int32_t> perm, row_ptr, col, color_ptr, xy;
    std::vector<int8_t> jcsr;  // couplings of the CSR entries, empty = all +1
    std::vector<double> field; // field_dim x N field components per original id, empty = no field
    int32_t field_dim = 0;
};

struct Region {
    size_t off = 0, bytes = 0;
};

constexpr size_t kAlign = 256;

size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

const int kGraphChunk = 32;  // sweeps per captured graph of the plain engine

}  // namespace

// A part of a batched plan: the samples of one size run with one launch
// shape (a plan whose samples all have the same size has one part).
struct Part {
    std::vector<int> samples;   // plan samples it runs (indices), in plan order
    BatchedShape B;
    int stage_mode = 0;
    std::vector<int2> units;    // (sample, group) per unit, sample by sample
    int u0 = 0;                 // its first unit in the plan's unit table
    int wave_units = 0;         // units one launch runs together
    int live_units = 0;         // units resident on the GPU at once (their spins: the live set)
    int max_clusters = 0;       // clusters of its shape that can be resident at once
    bool barrier_free = false;  // no cluster waits on another: may run beside other parts
};

struct xyl_plan {
    int engine = 0;
    uint64_t seed = 0;
    std::vector<HostSample> hs;
    PlanShape shape;
    std::vector<Part> parts;
    int recompute_every = 0;
    int resident_req = 0;   // the caller's resident setting: 1 only, -1 never, 0 either
    int waves_req = 0;      // the caller's waves setting: 1 L2-sized, -1 never, 0 either (autotuner)
    int64_t sweeps_since_recompute = 0;
    int total_R = 0;
    int64_t total_N = 0, total_nnz = 0, total_spins = 0;
    int total_Q1 = 0;
    std::vector<int2> units;  // every part's units, part by part
    size_t ws_bytes = 0;
    char *ws = nullptr;
    bool bound = false;
    DevPlan dev{};
    Region r_samples, r_row_ptr, r_col, r_perm, r_color_ptr, r_phase, r_spins, r_beta, r_delta, r_slot_of, r_rep_at,
        r_obs, r_last_E, r_acc, r_met_acc, r_met_try, r_pt_acc, r_pt_try, r_sweep, r_status, r_barrier, r_drift,
        r_units, r_push, r_field, r_check, r_unit_ctr;
    cudaStream_t capture_stream = nullptr;
    // parts that run side by side: one stream and one event each, and the fork event
    std::vector<cudaStream_t> part_streams;
    std::vector<cudaEvent_t> part_events;
    cudaEvent_t fork_event = nullptr;
    std::map<std::tuple<int, uint32_t, int>, cudaGraphExec_t> graphs;
    int64_t last_launches = 0;
    int64_t launches_per_graph_plain = 0;

    size_t spin_elem() const
    {
        if (shape.dim == 3) return shape.fp64 ? sizeof(double4_32a) : sizeof(float4);
        return shape.fp64 ? sizeof(double2) : sizeof(float2);
    }

    void drop_graphs()
    {
        for (auto &kv : graphs) cudaGraphExecDestroy(kv.second);
        graphs.clear();
    }
    ~xyl_plan()
    {
        drop_graphs();
        if (capture_stream) cudaStreamDestroy(capture_stream);
        for (cudaStream_t q : part_streams) cudaStreamDestroy(q);
        for (cudaEvent_t e : part_events) cudaEventDestroy(e);
        if (fork_event) cudaEventDestroy(fork_event);
    }
};

namespace {

int cuda_fail(cudaError_t e, const char *what)
{
    return fail(XYL_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define XYL_CUDA(call, what)                          \
    do {                                              \
        cudaError_t e_ = (call);                      \
        if (e_ != cudaSuccess) return cuda_fail(e_, what); \
    } while (0)

cudaStream_t as_stream(void *s) { return reinterpret_cast<cudaStream_t>(s); }

void layout(xyl_plan *p)
{
    size_t off = 0;
    auto take = [&](Region &r, size_t bytes) {
        r.off = off;
        r.bytes = bytes;
        off = align_up(off + std::max<size_t>(bytes, 1));
    };
    const size_t S = p->hs.size();
    take(p->r_samples, S * sizeof(DevSample));
    take(p->r_row_ptr, (p->total_N + S) * sizeof(int32_t));
    take(p->r_col, p->total_nnz * sizeof(int32_t));
    take(p->r_perm, p->total_N * sizeof(int32_t));
    take(p->r_color_ptr, p->total_Q1 * sizeof(int32_t));
    take(p->r_phase, p->total_N * (p->shape.fp64 ? sizeof(double4_32a) : sizeof(float4)));
    take(p->r_spins, p->total_spins * p->spin_elem());
    take(p->r_beta, p->total_R * sizeof(double));
    take(p->r_delta, p->total_R * sizeof(double));
    take(p->r_slot_of, p->total_R * sizeof(int32_t));
    take(p->r_rep_at, p->total_R * sizeof(int32_t));
    take(p->r_obs, 2 * (size_t)p->total_R * kObsStride * sizeof(double));
    take(p->r_last_E, p->total_R * sizeof(double));
    take(p->r_acc, (size_t)p->total_R * kAccCount * sizeof(double));
    take(p->r_met_acc, p->total_R * sizeof(unsigned long long));
    take(p->r_met_try, p->total_R * sizeof(unsigned long long));
    take(p->r_pt_acc, p->total_R * sizeof(unsigned long long));
    take(p->r_pt_try, p->total_R * sizeof(unsigned long long));
    take(p->r_sweep, S * sizeof(uint32_t));
    take(p->r_status, sizeof(int32_t));
    take(p->r_barrier, S * sizeof(unsigned int));
    take(p->r_drift, 2 * sizeof(double));  // the recorded drift, and a save slot for xyl_write_spins
    take(p->r_check, sizeof(unsigned long long));  // violation count of xyl_check_plan
    take(p->r_units, std::max<size_t>(p->total_R, 1) * sizeof(int2));  // the most units any shape makes
    take(p->r_unit_ctr, std::max<size_t>(p->total_R, 1) * sizeof(unsigned int));  // phase-barrier arrivals per unit
    take(p->r_push, p->total_N * sizeof(uint16_t));
    // random fields: one vector per site, only when some sample has them
    // (O(3): padded 4-vectors, like the spins)
    const size_t field_elem = p->shape.dim == 3 ? (p->shape.fp64 ? sizeof(double4_32a) : sizeof(float4))
                                                : (p->shape.fp64 ? sizeof(double2) : sizeof(float2));
    take(p->r_field, p->shape.fields ? p->total_N * field_elem : 0);
    p->ws_bytes = off;
}

template <typename T>
T *at(xyl_plan *p, const Region &r)
{
    return reinterpret_cast<T *>(p->ws + r.off);
}

int check_bound(xyl_plan *p, const char *who)
{
    if (!p) return fail(XYL_EINVAL, "%s: NULL plan", who);
    if (!p->bound) return fail(XYL_ESTATE, "%s: plan is not bound to a workspace", who);
    return XYL_OK;
}

// Shared-memory layout of the resident shape for groups of g replicas shared
// by G CTAs with `block` threads each: spins of every site (with one zero
// row) | warp partial sums | accepted counts | 16-bit site ids | 16-bit CSR
// rows of the CTA's own sites, the last two when they fit.  A cluster holds
// every group of a sample when G x groups <= 16, else one group.  Returns
// false when the shape does not apply to this batch.
bool resident_fit(const xyl_plan *p, const std::vector<int> &samples, int g, int G, int block, int stage,
                  BatchedShape &B)
{
    const int R0 = p->hs[samples[0]].R;
    int max_N = 0, max_deg = 0, owned = 0;
    for (int si : samples) {
        const HostSample &h = p->hs[si];
        if (h.R != R0) return false;
        max_N = std::max(max_N, h.N);
        max_deg = std::max(max_deg, h.max_deg);
        int o = 0;
        for (int c = 0; c < h.Q; ++c) o += (h.color_ptr[c + 1] - h.color_ptr[c] + G - 1) / G;
        owned = std::max(owned, o);
    }
    if (R0 % g) return false;
    const int n_groups = R0 / g;
    auto a16 = [](size_t v) { return (v + 15) / 16 * 16; };
    const size_t n_warps = (size_t)block / 32;
    const size_t spins = a16((size_t)(max_N + 1) * g * sizeof(float2));
    const size_t part = a16((size_t)kObsCount * n_warps * g * sizeof(float));
    const size_t met = a16(n_warps * g * sizeof(unsigned));
    const size_t beta = a16((size_t)R0 * sizeof(double));
    size_t off = spins + part + met + beta;
    if (off > kResidentDynLimitBytes) return false;
    B.rs_off_part = spins;
    B.rs_off_met = spins + part;
    B.rs_off_beta = spins + part + met;
    B.rs_ids = false;
    B.rs_csr_w = 0;
    B.rs_off_ids = B.rs_off_col = B.rs_off_peers = 0;
    if (G > 1) {
        const size_t peers = a16((size_t)owned * sizeof(uint16_t));
        if (off + peers <= kResidentDynLimitBytes) {
            B.rs_off_peers = off;
            off += peers;
        }
    }
    if (max_N <= 65535) {  // ids and the padding id N fit 16 bits
        const size_t ids = a16((size_t)owned * sizeof(uint16_t));
        if (off + ids <= kResidentDynLimitBytes) {
            B.rs_ids = true;
            B.rs_off_ids = off;
            off += ids;
        }
        const int W = B.fixed_deg == 6 ? 6 : 8;
        const size_t col = a16((size_t)owned * W * sizeof(uint16_t));
        // with couplings bit 15 of a staged id holds J, so ids (and the padding id N) stay below 2^15;
        // rows longer than eight are read from the global CSR
        if (stage >= 0 && max_deg <= 8 && off + col <= kResidentDynLimitBytes &&
            (!p->shape.coupled || max_N <= 32767)) {
            B.rs_csr_w = W;
            B.rs_off_col = off;
            off += col;
        }
    }
    B.resident = true;
    B.G = G;
    B.gpc = n_groups * G <= 16 ? n_groups : 1;
    B.cpc = G * B.gpc;
    B.owned_max = owned;
    B.staged = B.rs_csr_w != 0;
    B.smem_bytes = off;
    return true;
}

// Shared-memory layout of the O(3) resident shape: one CTA per group of g
// replicas keeps three single-precision component arrays of every site (one
// zero row) | warp partial sums (16 fields) | accepted counts | FP64 slot
// inverse temperatures | 16-bit site ids | 16-bit CSR rows, the last two when
// they fit.  The groups of a sample share a cluster when they are at most 16.
bool resident_fit_o3(const xyl_plan *p, const std::vector<int> &samples, int g, int block, int stage,
                     BatchedShape &B)
{
    const int R0 = p->hs[samples[0]].R;
    int max_N = 0, max_deg = 0;
    for (int si : samples) {
        const HostSample &h = p->hs[si];
        if (h.R != R0) return false;
        max_N = std::max(max_N, h.N);
        max_deg = std::max(max_deg, h.max_deg);
    }
    if (R0 % g || block % g) return false;
    const int n_groups = R0 / g;
    auto a16 = [](size_t v) { return (v + 15) / 16 * 16; };
    const size_t n_warps = (size_t)block / 32;
    const size_t comp = ((size_t)(max_N + 1) * g + 3) / 4 * 4;
    const size_t spins = 3 * comp * sizeof(float);
    const size_t part = a16((size_t)kObsCount3 * n_warps * g * sizeof(float));
    const size_t met = a16(n_warps * g * sizeof(unsigned));
    const size_t beta = a16((size_t)R0 * sizeof(double));
    size_t off = spins + part + met + beta;
    if (off > kResidentDynLimitBytes) return false;
    B.rs_off_part = spins;
    B.rs_off_met = spins + part;
    B.rs_off_beta = spins + part + met;
    B.rs_ids = false;
    B.rs_csr_w = 0;
    B.rs_off_ids = B.rs_off_col = B.rs_off_peers = 0;
    if (max_N <= 65535) {
        const size_t ids = a16((size_t)max_N * sizeof(uint16_t));
        if (off + ids <= kResidentDynLimitBytes) {
            B.rs_ids = true;
            B.rs_off_ids = off;
            off += ids;
        }
        const int W = B.fixed_deg == 6 ? 6 : 8;
        const size_t col = a16((size_t)max_N * W * sizeof(uint16_t));
        if (stage >= 0 && max_deg <= 8 && off + col <= kResidentDynLimitBytes && (!p->shape.coupled || max_N <= 32767)) {
            B.rs_csr_w = W;
            B.rs_off_col = off;
            off += col;
        }
    }
    B.resident = true;
    B.dim = 3;
    B.o3_comp = (int)comp;
    B.G = 1;
    B.gpc = n_groups <= 16 ? n_groups : 1;
    B.cpc = B.gpc;
    B.owned_max = max_N;
    B.staged = B.rs_csr_w != 0;
    B.smem_bytes = off;
    return true;
}

// Launch shape of the batched engine: R_g replicas per group, G CTAs per
// cluster, `block` threads per CTA; stage < 0 disables shared-memory staging;
// resident != 0 asks for the resident shape (G is then ignored).  O(3) spins
// run in the resident shape with one CTA per group.
int apply_shape(xyl_plan *p, Part &part, int g, int G, int block, int stage, int resident, int waves = 0,
                int span = 1)
{
    if (span < 1 || (span > 1 && (resident || p->shape.dim == 3)))
        return fail(XYL_EINVAL, "span=%d: clusters per group above 1 run in the global-memory shape only", span);
    if (span > 1 && (g < 2 || (g & (g - 1))))
        return fail(XYL_EINVAL, "span=%d: a group over several clusters takes a power of two >= 2 (group=%d)", span, g);
    if (g < 1 || g > 32) return fail(XYL_EINVAL, "group=%d must be in [1, 32]", g);
    if ((g & (g - 1)) && (resident || p->shape.dim == 3 || g % 2))
        return fail(XYL_EINVAL, "group=%d: a group that is not a power of two must be even and runs in the "
                    "global-memory shape", g);
    for (int si : part.samples)
        if (p->hs[si].R % g) return fail(XYL_EINVAL, "group=%d does not divide n_temps=%d", g, p->hs[si].R);
    if (G < 1 || G > 16) return fail(XYL_EINVAL, "cluster=%d must be in [1, 16]", G);
    if (block < 32 || block % 32 || block > 1024)
        return fail(XYL_EINVAL, "block=%d must be a multiple of 32 <= 1024", block);
    BatchedShape &B = part.B;
    B = BatchedShape{};
    B.G = G;
    B.span = span;
    B.Rg = g;
    B.block = block;
    B.disorder = p->shape.disorder;
    int max_deg = 1;
    for (int si : part.samples) max_deg = std::max(max_deg, p->hs[si].max_deg);
    B.max_deg = max_deg;
    int fixed = -1;
    for (int si : part.samples) {
        const HostSample &h = p->hs[si];
        for (int i = 0; i < h.N && fixed != 0; ++i) {
            const int dg = h.row_ptr[i + 1] - h.row_ptr[i];
            fixed = (fixed < 0 || fixed == dg) ? dg : 0;
        }
    }
    B.fixed_deg = fixed < 0 ? 0 : fixed;
    part.stage_mode = stage;
    part.units.clear();
    for (int si : part.samples)
        for (int k = 0; k < p->hs[si].R / g; ++k) part.units.push_back(make_int2(si, k));
    if (p->shape.dim == 3) {
        if (!resident || G != 1)
            return fail(XYL_EINVAL, "O(3) spins on the batched engine run in the resident shape, one CTA per group");
        if (!resident_fit_o3(p, part.samples, g, block, stage, B))
            return fail(XYL_EINVAL, "O(3) resident shape with group=%d does not fit this batch (equal n_temps, a "
                        "group's spins, 12 B a site, within %zu B of shared memory)", g, kResidentDynLimitBytes);
        return XYL_OK;
    }
    if (resident) {
        if (!resident_fit(p, part.samples, g, G, block, stage, B))
            return fail(XYL_EINVAL, "resident shape with group=%d does not fit this batch (equal n_temps, "
                        "a group's spins within %zu B of shared memory)", g, kResidentDynLimitBytes);
        return XYL_OK;
    }
    int owned = 0;
    for (int si : part.samples) {
        const HostSample &h = p->hs[si];
        int o = 0;
        for (int c = 0; c < h.Q; ++c) o += (h.color_ptr[c + 1] - h.color_ptr[c] + G * span - 1) / (G * span);
        owned = std::max(owned, o);
    }
    B.owned_max = owned;
    const size_t bytes = (size_t)owned * (size_t)(max_deg + 2) * sizeof(int32_t);
    // CTAs above 672 threads (64 registers each) read their rows from global memory
    B.staged = stage >= 0 && bytes <= kStageLimitBytes && block <= 672;
    B.smem_bytes = B.staged ? bytes : 0;
    B.l2_waves = waves > 0;
    return XYL_OK;
}

// Device bytes one sample keeps live during a sweep of the global-memory
// shape: its spins, CSR, site ids and Fourier phases.
size_t sample_live_bytes(const HostSample &h)
{
    return (size_t)h.N * h.R * sizeof(float2) + h.col.size() * sizeof(int32_t) +
           (size_t)(2 * h.N + 1) * sizeof(int32_t) + (size_t)h.N * sizeof(float4);
}

// Samples a launch wave of the global-memory shape may hold so that their
// working set stays in L2 (three quarters of it, the rest for the sums and
// the other traffic); at least one.
int l2_wave_samples(const xyl_plan *p, const Part &part)
{
    int dev = 0, l2 = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev) != cudaSuccess)
        return 1;
    size_t per = 1;
    for (int si : part.samples) per = std::max(per, sample_live_bytes(p->hs[si]));
    return (int)std::max<size_t>(1, (size_t)l2 * 3 / 4 / per);
}

int pick_part_shape(xyl_plan *p, Part &part, const xyl_tuning *tune)
{
    const int mode = tune ? tune->resident : 0;
    const int stage = tune ? tune->stage : 0;
    const int span = (tune && tune->span > 0) ? tune->span : 1;
    if (tune && tune->span < 0) return fail(XYL_EINVAL, "span=%d must be >= 0", tune->span);
    if (span > 1 && (mode > 0 || p->shape.dim == 3))
        return fail(XYL_EINVAL, "span=%d: clusters per group above 1 run in the global-memory shape only", span);
    int block = 512;
    if (tune && tune->block > 0) block = tune->block;
    if (p->shape.dim == 3) {
        // O(3): resident only, the largest group that fits, all groups of a sample in one cluster first
        if (mode < 0) return fail(XYL_EINVAL, "O(3) spins on the batched engine run in the resident shape");
        for (int pass = 0; pass < 2; ++pass)
            for (int g = 32; g >= 1; g >>= 1) {
                if (tune && tune->group > 0 && g != tune->group) continue;
                bool divides = true;
                for (int si : part.samples) divides &= (p->hs[si].R % g == 0);
                if (!divides || apply_shape(p, part, g, 1, block, stage, 1) != XYL_OK) continue;
                if (pass == 1 || part.B.gpc * g == p->hs[part.samples[0]].R) return XYL_OK;
            }
        return fail(XYL_EINVAL, "O(3) resident shape does not fit this batch (equal n_temps, a group's spins, 12 B "
                    "a site, within %zu B of shared memory)", kResidentDynLimitBytes);
    }
    if (mode >= 0 && span == 1) {
        // resident: the largest group that fits with all groups of a sample in
        // one cluster (pairs of replicas share a Philox block); a caller's
        // group or cluster width is taken as given
        const int G = (tune && tune->cluster > 0) ? tune->cluster : 1;
        const bool given = mode == 1 || (tune && (tune->group > 0 || tune->cluster > 0));
        for (int pass = 0; pass < (given ? 2 : 1); ++pass) {
            for (int g = 32; g >= 1; g >>= 1) {
                if (tune && tune->group > 0 && g != tune->group) continue;
                bool divides = true;
                for (int si : part.samples) divides &= (p->hs[si].R % g == 0);
                if (!divides || apply_shape(p, part, g, G, block, stage, 1) != XYL_OK) continue;
                // first choice: every group of a sample in one cluster
                if (pass == 1 || part.B.gpc * g == p->hs[part.samples[0]].R) return XYL_OK;
            }
        }
        if (mode == 1)
            return fail(XYL_EINVAL, "resident shape does not fit this batch (equal n_temps, a group's "
                        "spins within %zu B of shared memory)", kResidentDynLimitBytes);
        clear_error();
    }
    // replicas per cluster: largest power of two <= 16 dividing every sample's R
    int g = 16;
    for (int si : part.samples)
        while (g > 1 && p->hs[si].R % g) g >>= 1;
    if (tune && tune->group > 0) g = tune->group;
    int max_N = 0;
    for (int si : part.samples) max_N = std::max(max_N, p->hs[si].N);
    // default cluster width: enough CTAs that a phase has a few thousand items per CTA
    int G = 1;
    const double items_per_phase = (double)max_N * g / std::max(1, p->shape.max_Q);
    while (G < 16 && items_per_phase / (G * 2) >= 1024.0) G *= 2;
    if (tune && tune->cluster > 0) G = tune->cluster;
    return apply_shape(p, part, g, G, block, stage, 0, tune ? tune->waves : 0, span);
}

void gather_units(xyl_plan *p);

// Split a batched plan into parts: one per sample size (largest first) when
// the library chooses the shapes and the sizes differ, else one part.
int pick_batched_shape(xyl_plan *p, const xyl_tuning *tune)
{
    const bool caller_shape = tune && (tune->resident != 0 || tune->group > 0 || tune->cluster > 0 || tune->block > 0 ||
                                       tune->span > 0);
    std::vector<int> sizes;
    for (auto &h : p->hs) sizes.push_back(h.N);
    std::sort(sizes.begin(), sizes.end(), std::greater<int>());
    sizes.erase(std::unique(sizes.begin(), sizes.end()), sizes.end());
    p->parts.clear();
    if (caller_shape || sizes.size() == 1) {
        Part part;
        for (int s = 0; s < (int)p->hs.size(); ++s) part.samples.push_back(s);
        p->parts.push_back(part);
    } else {
        for (int n : sizes) {
            Part part;
            for (int s = 0; s < (int)p->hs.size(); ++s)
                if (p->hs[s].N == n) part.samples.push_back(s);
            p->parts.push_back(part);
        }
    }
    for (Part &part : p->parts) {
        const int rc = pick_part_shape(p, part, tune);
        if (rc) return rc;
    }
    gather_units(p);
    return XYL_OK;
}

// The plan's unit table: every part's units, part by part.
void gather_units(xyl_plan *p)
{
    p->units.clear();
    for (Part &part : p->parts) {
        part.u0 = (int)p->units.size();
        p->units.insert(p->units.end(), part.units.begin(), part.units.end());
    }
}

// Set the kernel attributes of a part's shape, size its launch waves (all
// groups of a sample resident together when they meet at a global barrier)
// and, for a site split, upload the peer masks of its samples.
int configure_part(xyl_plan *p, Part &part, cudaStream_t st)
{
    int clusters = 0;
    const BatchedShape &B = part.B;
    const HostSample &h0 = p->hs[part.samples[0]];
    const int n_units = (int)part.units.size();
    if (B.resident) {
        if (B.dim == 3)
            XYL_CUDA(resident_o3_max_active_clusters(B, &clusters), "batched: occupancy");
        else
            XYL_CUDA(resident_max_active_clusters(B, &clusters), "batched: occupancy");
        if (clusters < 1)
            return fail(XYL_EINVAL, "batched: a resident cluster of %d CTAs x %d threads (%zu B shared) cannot be resident",
                        B.cpc, B.block, B.smem_bytes);
        const int n_groups = h0.R / B.Rg;
        if (B.gpc == n_groups) {
            // a cluster is a whole sample and never waits on another: one
            // launch, the hardware queues the clusters that do not fit yet
            part.wave_units = n_units;
            part.live_units = std::min(n_units, clusters * B.gpc);
            part.barrier_free = true;
        } else {
            // the clusters of a sample meet at a global barrier: a wave holds
            // whole samples that are resident together
            const int per_sample = n_groups / B.gpc;
            const int samples_per_wave = clusters / per_sample;
            if (samples_per_wave < 1)
                return fail(XYL_EINVAL, "batched: %d resident clusters of %d CTAs cannot be co-resident (max %d)",
                            per_sample, B.cpc, clusters);
            part.wave_units = samples_per_wave * n_groups;
            part.live_units = part.wave_units;
            part.barrier_free = false;
        }
        if (B.G > 1) {
            // per site: the other CTAs of its group whose chunks link to it
            std::vector<int64_t> site_off(p->hs.size(), 0);
            for (size_t s = 1; s < p->hs.size(); ++s) site_off[s] = site_off[s - 1] + p->hs[s - 1].N;
            for (int si : part.samples) {
                const HostSample &h = p->hs[si];
                std::vector<int> owner(h.N);
                std::vector<uint16_t> mask(h.N, 0);
                for (int c = 0; c < h.Q; ++c) {
                    const int cb = h.color_ptr[c], ce = h.color_ptr[c + 1];
                    const int chunk = (ce - cb + B.G - 1) / B.G;
                    for (int i = cb; i < ce; ++i) owner[i] = (i - cb) / chunk;
                }
                for (int i = 0; i < h.N; ++i) {
                    uint32_t m = 0;
                    for (int k = h.row_ptr[i]; k < h.row_ptr[i + 1]; ++k) m |= 1u << owner[h.col[k]];
                    mask[i] = (uint16_t)(m & ~(1u << owner[i]));
                }
                XYL_CUDA(cudaMemcpyAsync(p->ws + p->r_push.off + site_off[si] * sizeof(uint16_t), mask.data(),
                                         mask.size() * sizeof(uint16_t), cudaMemcpyHostToDevice, st), "batched: peer masks");
                XYL_CUDA(cudaStreamSynchronize(st), "batched: sync");
            }
        }
        return XYL_OK;
    }
    XYL_CUDA(batched_max_active_clusters(p->shape, B, &clusters), "batched: occupancy");
    if (clusters < 1)
        return fail(XYL_EINVAL, "batched: a cluster of %d CTAs x %d threads (%zu B shared) cannot be resident",
                    B.G, B.block, B.smem_bytes);
    part.max_clusters = clusters;
    const int n_groups = h0.R / B.Rg;
    bool uniform_groups = true;
    int groups_max = 1;
    for (int si : part.samples) {
        uniform_groups &= (p->hs[si].R / B.Rg == n_groups);
        groups_max = std::max(groups_max, p->hs[si].R / B.Rg);
    }
    if (groups_max > 1 || B.span > 1) {
        if (!uniform_groups) return fail(XYL_EINVAL, "batched: several groups per sample need equal n_temps");
        // every cluster of a sample (its groups x span) must be resident at once
        int samples_per_wave = clusters / (n_groups * B.span);
        if (samples_per_wave < 1)
            return fail(XYL_EINVAL, "batched: %d clusters of %d CTAs cannot be co-resident (max %d)",
                        n_groups * B.span, B.G, clusters);
        if (B.l2_waves) samples_per_wave = std::min(samples_per_wave, l2_wave_samples(p, part));
        part.wave_units = samples_per_wave * n_groups;
        part.live_units = part.wave_units;
        part.barrier_free = false;
    } else {
        // one group per sample: clusters never wait on one another, so a launch
        // may hold more than fit at once (the hardware queues them), unless
        // its waves are sized to L2
        part.wave_units = B.l2_waves ? std::min(n_units, l2_wave_samples(p, part)) : n_units;
        part.live_units = std::min(part.wave_units, clusters);
        part.barrier_free = true;
    }
    return XYL_OK;
}

// Upload the unit table; streams and events for parts that run side by side;
// the global-memory shape expects the sum buffer of its next sweep cleared.
int finish_configure(xyl_plan *p, cudaStream_t st)
{
    gather_units(p);
    XYL_CUDA(cudaMemcpyAsync(p->ws + p->r_units.off, p->units.data(), p->units.size() * sizeof(int2),
                             cudaMemcpyHostToDevice, st), "batched: unit table");
    XYL_CUDA(cudaMemsetAsync(p->ws + p->r_obs.off, 0, p->r_obs.bytes, st), "batched: obs");
    XYL_CUDA(cudaStreamSynchronize(st), "batched: sync");
    int side = 0;
    for (const Part &part : p->parts) side += part.barrier_free ? 1 : 0;
    while ((int)p->part_streams.size() < side) {
        cudaStream_t q = nullptr;
        cudaEvent_t e = nullptr;
        XYL_CUDA(cudaStreamCreateWithFlags(&q, cudaStreamNonBlocking), "batched: stream");
        p->part_streams.push_back(q);
        XYL_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "batched: event");
        p->part_events.push_back(e);
    }
    if (!p->fork_event && side > 1)
        XYL_CUDA(cudaEventCreateWithFlags(&p->fork_event, cudaEventDisableTiming), "batched: event");
    p->drop_graphs();
    return XYL_OK;
}

int configure_batched(xyl_plan *p, cudaStream_t st)
{
    for (Part &part : p->parts) {
        const int rc = configure_part(p, part, st);
        if (rc) return rc;
    }
    return finish_configure(p, st);
}

}  // namespace

extern "C" {

int xyl_plan_create(const xyl_sample *samples, int32_t n_samples, int32_t engine, uint64_t seed,
                    const xyl_tuning *tune, xyl_plan **out, size_t *workspace_bytes)
{
    clear_error();
    if (!out) return fail(XYL_EINVAL, "xyl_plan_create: out is NULL");
    *out = nullptr;
    if (!samples || n_samples < 1) return fail(XYL_EINVAL, "xyl_plan_create: empty batch");
    if (engine != XYL_FP64_PLAIN && engine != XYL_FP32_BATCHED && engine != XYL_FP32_PLAIN)
        return fail(XYL_EINVAL, "xyl_plan_create: unknown engine %d", engine);
    auto *p = new xyl_plan();
    p->engine = engine;
    p->seed = seed;
    p->shape.fp64 = (engine == XYL_FP64_PLAIN);
    p->shape.layout = (engine == XYL_FP32_BATCHED) ? kInterleaved : kReplicaMajor;
    p->recompute_every = tune ? std::max(0, tune->recompute_every) : 0;
    p->resident_req = tune ? tune->resident : 0;
    p->waves_req = tune ? tune->waves : 0;
    const int dim = (tune && tune->spin_dim) ? tune->spin_dim : 2;
    if (dim != 2 && dim != 3) {
        delete p;
        return fail(XYL_EINVAL, "xyl_plan_create: spin_dim %d (2 = XY, 3 = O(3))", dim);
    }
    p->shape.dim = dim;
    // O(3) spins are padded 4-vectors, replica-major in global memory on every engine
    if (dim == 3) p->shape.layout = kReplicaMajor;
    for (int s = 0; s < n_samples; ++s) {
        const xyl_sample &in = samples[s];
        const xyl_graph *g = in.graph;
        if (!g || in.n_temps < 1 || !in.beta || !in.delta) {
            delete p;
            return fail(XYL_EINVAL, "xyl_plan_create: sample %d has no graph, slots or temperatures", s);
        }
        if (engine == XYL_FP32_BATCHED && in.n_temps > 256) {
            delete p;
            return fail(XYL_EINVAL, "xyl_plan_create: batched engine supports at most 256 slots per sample");
        }
        if (engine == XYL_FP32_BATCHED && g->n_colors > kMaxColorsBatched) {
            delete p;
            return fail(XYL_EINVAL, "xyl_plan_create: batched engine supports at most %d colour classes",
                        kMaxColorsBatched);
        }
        HostSample h;
        h.N = g->n; h.Q = g->n_colors; h.R = in.n_temps; h.L = g->L; h.max_deg = g->max_deg;
        h.sample_id = in.sample_id;
        h.beta.assign(in.beta, in.beta + in.n_temps);
        h.delta.assign(in.delta, in.delta + in.n_temps);
        for (int k = 0; k < in.n_temps; ++k) {
            if (!std::isfinite(h.beta[k]) || h.beta[k] < 0 || !std::isfinite(h.delta[k]) || h.delta[k] < 0) {
                delete p;
                return fail(XYL_EINVAL, "xyl_plan_create: sample %d slot %d has a bad beta/delta", s, k);
            }
        }
        h.perm = g->perm; h.row_ptr = g->row_ptr; h.col = g->col; h.color_ptr = g->color_ptr; h.xy = g->xy;
        h.jcsr = g->jcsr;
        for (int8_t j : h.jcsr) p->shape.coupled |= (j < 0);
        h.field = g->field;
        h.field_dim = g->field_dim;
        if (!h.field.empty() && h.field_dim != dim) {
            delete p;
            return fail(XYL_EINVAL, "xyl_plan_create: sample %d has %d-component fields for %d-component spins "
                        "(xyl_graph_set_fields for XY, xyl_graph_set_fields3 for O(3))", s, h.field_dim, dim);
        }
        p->shape.fields |= !h.field.empty();
        p->total_R += h.R;
        p->total_N += h.N;
        p->total_nnz += (int64_t)h.col.size();
        p->total_spins += (int64_t)h.N * h.R;
        p->total_Q1 += h.Q + 1;
        p->shape.max_R = std::max(p->shape.max_R, h.R);
        p->shape.max_Q = std::max(p->shape.max_Q, h.Q);
        p->shape.max_N = std::max(p->shape.max_N, h.N);
        if ((int)p->shape.class_max.size() < h.Q) p->shape.class_max.resize(h.Q, 0);
        for (int c = 0; c < h.Q; ++c) {
            p->shape.max_class = std::max(p->shape.max_class, h.color_ptr[c + 1] - h.color_ptr[c]);
            p->shape.class_max[c] = std::max(p->shape.class_max[c], h.color_ptr[c + 1] - h.color_ptr[c]);
        }
        p->hs.push_back(std::move(h));
    }
    p->shape.n_samples = n_samples;
    p->shape.disorder = p->shape.coupled || p->shape.fields;
    if (engine == XYL_FP32_BATCHED) {
        const int rc = pick_batched_shape(p, tune);
        if (rc) { delete p; return rc; }
    }
    layout(p);
    if (workspace_bytes) *workspace_bytes = p->ws_bytes;
    *out = p;
    return XYL_OK;
}

int xyl_bind(xyl_plan *p, void *d_workspace, size_t bytes, void *stream)
{
    CallRange range_("xyl_bind");
    clear_error();
    if (!p || !d_workspace) return fail(XYL_EINVAL, "xyl_bind: NULL plan or workspace");
    if (bytes < p->ws_bytes) return fail(XYL_ENOSPC, "xyl_bind: workspace %zu B < required %zu B", bytes, p->ws_bytes);
    if (reinterpret_cast<uintptr_t>(d_workspace) % kAlign) return fail(XYL_EINVAL, "xyl_bind: workspace not 256-byte aligned");
    cudaStream_t st = as_stream(stream);
    p->drop_graphs();
    p->ws = static_cast<char *>(d_workspace);
    // host images of the constant tables
    const size_t S = p->hs.size();
    std::vector<DevSample> ds(S);
    std::vector<int32_t> row_ptr, col, perm, color_ptr;
    row_ptr.reserve(p->total_N + S); col.reserve(p->total_nnz); perm.reserve(p->total_N); color_ptr.reserve(p->total_Q1);
    std::vector<float4> ph32;
    std::vector<double4_32a> ph64;
    std::vector<double> beta, delta;
    int64_t site_off = 0, row_off = 0, col_off = 0, spin_off = 0;
    int color_off = 0, rep_off = 0;
    for (size_t s = 0; s < S; ++s) {
        const HostSample &h = p->hs[s];
        DevSample &d = ds[s];
        d.N = h.N; d.Q = h.Q; d.R = h.R; d.L = h.L; d.sample_id = h.sample_id; d.max_deg = h.max_deg;
        d.color_off = color_off; d.rep_off = rep_off; d.site_off = site_off; d.row_off = row_off;
        d.col_off = col_off; d.spin_off = spin_off;
        row_ptr.insert(row_ptr.end(), h.row_ptr.begin(), h.row_ptr.end());
        col.insert(col.end(), h.col.begin(), h.col.end());
        // random bonds: J = -1 in the top bit of the neighbour id
        if (!h.jcsr.empty())
            for (size_t k = 0; k < h.col.size(); ++k)
                if (h.jcsr[k] < 0) col[col.size() - h.col.size() + k] |= (int32_t)0x80000000u;
        perm.insert(perm.end(), h.perm.begin(), h.perm.end());
        color_ptr.insert(color_ptr.end(), h.color_ptr.begin(), h.color_ptr.end());
        for (int i = 0; i < h.N; ++i) {
            const int v = h.perm[i];
            const double ax = 2.0 * M_PI * (double)h.xy[2 * v] / (double)h.L;
            const double ay = 2.0 * M_PI * (double)h.xy[2 * v + 1] / (double)h.L;
            if (p->shape.fp64)
                ph64.push_back(make_double4_32a(std::cos(ax), std::sin(ax), std::cos(ay), std::sin(ay)));
            else
                ph32.push_back(make_float4((float)std::cos(ax), (float)std::sin(ax), (float)std::cos(ay), (float)std::sin(ay)));
        }
        beta.insert(beta.end(), h.beta.begin(), h.beta.end());
        delta.insert(delta.end(), h.delta.begin(), h.delta.end());
        site_off += h.N; row_off += h.N + 1; col_off += (int64_t)h.col.size(); spin_off += (int64_t)h.N * h.R;
        color_off += h.Q + 1; rep_off += h.R;
    }
    auto up = [&](const Region &r, const void *src, size_t n) -> cudaError_t {
        if (!n) return cudaSuccess;
        return cudaMemcpyAsync(p->ws + r.off, src, n, cudaMemcpyHostToDevice, st);
    };
    XYL_CUDA(up(p->r_samples, ds.data(), ds.size() * sizeof(DevSample)), "xyl_bind: upload");
    XYL_CUDA(up(p->r_row_ptr, row_ptr.data(), row_ptr.size() * 4), "xyl_bind: upload");
    XYL_CUDA(up(p->r_col, col.data(), col.size() * 4), "xyl_bind: upload");
    XYL_CUDA(up(p->r_perm, perm.data(), perm.size() * 4), "xyl_bind: upload");
    XYL_CUDA(up(p->r_color_ptr, color_ptr.data(), color_ptr.size() * 4), "xyl_bind: upload");
    if (p->shape.fp64)
        XYL_CUDA(up(p->r_phase, ph64.data(), ph64.size() * sizeof(double4_32a)), "xyl_bind: upload");
    else
        XYL_CUDA(up(p->r_phase, ph32.data(), ph32.size() * sizeof(float4)), "xyl_bind: upload");
    XYL_CUDA(up(p->r_beta, beta.data(), beta.size() * 8), "xyl_bind: upload");
    if (p->shape.fields) {
        // field of each site in colour-sorted order (zero for samples without fields)
        std::vector<double> f64;
        std::vector<float> f32;
        // (O(3): (h_x, h_y, h_z, 0) per site)
        const int dim = p->shape.dim, slots = dim == 3 ? 4 : 2;
        for (const HostSample &h : p->hs)
            for (int i = 0; i < h.N; ++i) {
                const int v = h.perm[i];
                for (int a = 0; a < slots; ++a) {
                    const double f = (h.field.empty() || a >= dim) ? 0.0 : h.field[dim * (size_t)v + a];
                    if (p->shape.fp64) f64.push_back(f);
                    else f32.push_back((float)f);
                }
            }
        if (p->shape.fp64) XYL_CUDA(up(p->r_field, f64.data(), f64.size() * 8), "xyl_bind: upload");
        else XYL_CUDA(up(p->r_field, f32.data(), f32.size() * 4), "xyl_bind: upload");
    }
    XYL_CUDA(up(p->r_delta, delta.data(), delta.size() * 8), "xyl_bind: upload");
    // everything mutable starts zeroed
    const Region *zero[] = {&p->r_spins, &p->r_slot_of, &p->r_rep_at, &p->r_obs, &p->r_last_E, &p->r_acc,
                            &p->r_met_acc, &p->r_met_try, &p->r_pt_acc, &p->r_pt_try, &p->r_sweep, &p->r_status,
                            &p->r_barrier, &p->r_drift};
    for (const Region *r : zero) XYL_CUDA(cudaMemsetAsync(p->ws + r->off, 0, r->bytes, st), "xyl_bind: memset");
    DevPlan &P = p->dev;
    P.samples = at<DevSample>(p, p->r_samples);
    P.n_samples = (int32_t)S;
    P.total_R = p->total_R;
    P.row_ptr = at<int32_t>(p, p->r_row_ptr);
    P.col = at<int32_t>(p, p->r_col);
    P.perm = at<int32_t>(p, p->r_perm);
    P.color_ptr = at<int32_t>(p, p->r_color_ptr);
    P.phase = p->ws + p->r_phase.off;
    P.field = p->shape.fields ? p->ws + p->r_field.off : nullptr;
    P.spins = p->ws + p->r_spins.off;
    P.beta = at<double>(p, p->r_beta);
    P.delta = at<double>(p, p->r_delta);
    P.slot_of = at<int32_t>(p, p->r_slot_of);
    P.rep_at = at<int32_t>(p, p->r_rep_at);
    P.obs = at<double>(p, p->r_obs);
    P.last_E = at<double>(p, p->r_last_E);
    P.acc = at<double>(p, p->r_acc);
    P.met_acc = at<unsigned long long>(p, p->r_met_acc);
    P.met_try = at<unsigned long long>(p, p->r_met_try);
    P.pt_acc = at<unsigned long long>(p, p->r_pt_acc);
    P.pt_try = at<unsigned long long>(p, p->r_pt_try);
    P.sweep = at<uint32_t>(p, p->r_sweep);
    P.status = at<int32_t>(p, p->r_status);
    P.barrier = at<unsigned int>(p, p->r_barrier);
    P.drift = at<double>(p, p->r_drift);
    P.push = at<uint16_t>(p, p->r_push);
    P.key = p->seed;
    // Maclaurin coefficients by the factorial recurrence a_k = a_{k-1} / (n (n+1))
    {
        double a = 1.0;
        P.sin_coef[0] = 1.0;
        for (int k = 1; k < kSinTerms; ++k) {
            a = a / (double)((2 * k) * (2 * k + 1));
            P.sin_coef[k] = (k & 1) ? -a : a;
        }
        a = 1.0;
        P.cos_coef[0] = 1.0;
        for (int k = 1; k < kCosTerms; ++k) {
            a = a / (double)((2 * k - 1) * (2 * k));
            P.cos_coef[k] = (k & 1) ? -a : a;
        }
    }
    if (!p->capture_stream) XYL_CUDA(cudaStreamCreateWithFlags(&p->capture_stream, cudaStreamNonBlocking), "xyl_bind: stream");
    if (p->engine == XYL_FP32_BATCHED) {
        const int rc = configure_batched(p, st);
        if (rc) return rc;
    }
    XYL_CUDA(cudaStreamSynchronize(st), "xyl_bind: sync");
    p->bound = true;
    return XYL_OK;
}

}  // extern "C"

namespace {

int buffer_mode(const xyl_plan *p) { return p->engine == XYL_FP32_BATCHED ? 1 : 0; }

int zero_region(xyl_plan *p, const Region &r, cudaStream_t st)
{
    XYL_CUDA(cudaMemsetAsync(p->ws + r.off, 0, r.bytes, st), "memset");
    return XYL_OK;
}

// Launch units [u, u + cnt) of a part, in its waves.
int launch_units(xyl_plan *p, const DevPlan &P, const Part &part, int u_begin, int cnt, int n, uint32_t ops,
                 int measure_every, cudaStream_t st, int64_t *launches)
{
    for (int u = u_begin; u < u_begin + cnt; u += part.wave_units) {
        const int c = std::min(part.wave_units, u_begin + cnt - u);
        if (part.B.resident && part.B.dim == 3)
            XYL_CUDA(launch_resident_o3(P, part.B, at<int2>(p, p->r_units), u, c, n, ops, measure_every, st),
                     "sweep: resident launch");
        else if (part.B.resident)
            XYL_CUDA(launch_resident(P, part.B, at<int2>(p, p->r_units), u, c, n, ops, measure_every, st),
                     "sweep: resident launch");
        else
            XYL_CUDA(launch_batched(P, p->shape, part.B, at<int2>(p, p->r_units), at<unsigned int>(p, p->r_unit_ctr),
                                    u, c, n, ops, measure_every, st),
                     "sweep: batched launch");
        ++*launches;
    }
    return XYL_OK;
}

// The batched engine's launches for n sweeps: parts whose clusters wait on
// other clusters of their sample run first, one after another, each with the
// whole GPU (nothing else may hold the SMs their waves count on); then the
// parts that never wait run side by side on forked streams.
int issue_batched(xyl_plan *p, const DevPlan &P, int n, uint32_t ops, int measure_every, cudaStream_t st,
                  int64_t *launches, bool side_by_side)
{
    int rc;
    XYL_CUDA(cudaMemsetAsync(reinterpret_cast<char *>(P.barrier), 0, p->hs.size() * sizeof(unsigned int), st),
             "sweep: barrier reset");
    std::vector<const Part *> free_parts;
    for (const Part &part : p->parts) {
        if (part.barrier_free) {
            free_parts.push_back(&part);
            continue;
        }
        if ((rc = launch_units(p, P, part, part.u0, (int)part.units.size(), n, ops, measure_every, st, launches)))
            return rc;
    }
    if (free_parts.size() <= 1 || !side_by_side || !p->fork_event) {
        for (const Part *part : free_parts)
            if ((rc = launch_units(p, P, *part, part->u0, (int)part->units.size(), n, ops, measure_every, st, launches)))
                return rc;
        return XYL_OK;
    }
    XYL_CUDA(cudaEventRecord(p->fork_event, st), "sweep: fork");
    for (size_t k = 0; k < free_parts.size(); ++k) {
        cudaStream_t q = p->part_streams[k];
        XYL_CUDA(cudaStreamWaitEvent(q, p->fork_event, 0), "sweep: fork");
        if ((rc = launch_units(p, P, *free_parts[k], free_parts[k]->u0, (int)free_parts[k]->units.size(), n, ops,
                               measure_every, q, launches)))
            return rc;
        XYL_CUDA(cudaEventRecord(p->part_events[k], q), "sweep: join");
        XYL_CUDA(cudaStreamWaitEvent(st, p->part_events[k], 0), "sweep: join");
    }
    return XYL_OK;
}

// Enqueue the work of `n` sweeps (no graph).
int issue_sweeps(xyl_plan *p, int n, uint32_t ops, int measure_every, cudaStream_t st, int64_t *launches)
{
    if (p->engine == XYL_FP32_BATCHED) return issue_batched(p, p->dev, n, ops, measure_every, st, launches, true);
    for (int k = 0; k < n; ++k)
        XYL_CUDA(launch_plain_sweep(p->dev, p->shape, ops, measure_every, st, launches), "sweep: plain launch");
    return XYL_OK;
}

int run_captured(xyl_plan *p, int n, uint32_t ops, int measure_every, cudaStream_t st)
{
    const auto key = std::make_tuple(n, ops, measure_every);
    auto it = p->graphs.find(key);
    int64_t launches = 0;
    if (it == p->graphs.end()) {
        XYL_CUDA(cudaStreamBeginCapture(p->capture_stream, cudaStreamCaptureModeThreadLocal), "sweep: begin capture");
        const int rc = issue_sweeps(p, n, ops, measure_every, p->capture_stream, &launches);
        cudaGraph_t graph = nullptr;
        const cudaError_t ec = cudaStreamEndCapture(p->capture_stream, &graph);
        if (rc) {
            if (graph) cudaGraphDestroy(graph);
            return rc;
        }
        if (ec != cudaSuccess) return cuda_fail(ec, "sweep: end capture");
        cudaGraphExec_t exec = nullptr;
        const cudaError_t ei = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (ei != cudaSuccess) return cuda_fail(ei, "sweep: instantiate");
        it = p->graphs.emplace(key, exec).first;
        p->launches_per_graph_plain = launches;
    }
    XYL_CUDA(cudaGraphLaunch(it->second, st), "sweep: graph launch");
    return XYL_OK;
}

int64_t launches_of(xyl_plan *p, int n, uint32_t ops)
{
    if (p->engine == XYL_FP32_BATCHED) {
        int64_t n_launch = 0;
        for (const Part &part : p->parts)
            n_launch += ((int64_t)part.units.size() + part.wave_units - 1) / part.wave_units;
        return n_launch;
    }
    const int64_t per_sweep = (int64_t)(((ops & XYL_OP_MET) ? p->shape.max_Q : 0) +
                                        ((ops & XYL_OP_OR) ? p->shape.max_Q : 0) + 1);
    return per_sweep * n;
}

int do_recompute(xyl_plan *p, int renormalise, cudaStream_t st)
{
    XYL_CUDA(launch_recompute(p->dev, p->shape, renormalise, buffer_mode(p), st), "recompute");
    return zero_region(p, p->r_obs, st);
}

}  // namespace

extern "C" {

int xyl_init_spins(xyl_plan *p, int32_t aligned, void *stream)
{
    CallRange range_("xyl_init_spins");
    clear_error();
    int rc = check_bound(p, "xyl_init_spins");
    if (rc) return rc;
    cudaStream_t st = as_stream(stream);
    const Region *zero[] = {&p->r_obs, &p->r_last_E, &p->r_acc, &p->r_met_acc, &p->r_met_try, &p->r_pt_acc,
                            &p->r_pt_try, &p->r_status, &p->r_barrier};
    for (const Region *r : zero)
        if ((rc = zero_region(p, *r, st))) return rc;
    XYL_CUDA(launch_init(p->dev, p->shape, aligned, st), "xyl_init_spins: launch");
    if ((rc = do_recompute(p, 0, st))) return rc;
    if ((rc = zero_region(p, p->r_drift, st))) return rc;
    p->sweeps_since_recompute = 0;
    return XYL_OK;
}

int xyl_sweep(xyl_plan *p, int32_t n_sweeps, uint32_t ops, int32_t measure_every, void *stream)
{
    CallRange range_("xyl_sweep");
    clear_error();
    int rc = check_bound(p, "xyl_sweep");
    if (rc) return rc;
    if (n_sweeps < 0) return fail(XYL_EINVAL, "xyl_sweep: n_sweeps < 0");
    if (!(ops & (XYL_OP_MET | XYL_OP_OR))) return fail(XYL_EINVAL, "xyl_sweep: ops must include MET or OR");
    if (ops & ~(XYL_OP_MET | XYL_OP_OR | XYL_OP_PT | XYL_OP_MEASURE)) return fail(XYL_EINVAL, "xyl_sweep: unknown op bits");
    if ((ops & XYL_OP_MEASURE) && measure_every < 1) return fail(XYL_EINVAL, "xyl_sweep: measure_every must be >= 1");
    if (!(ops & XYL_OP_MEASURE)) measure_every = 1;
    cudaStream_t st = as_stream(stream);
    p->last_launches = 0;
    int left = n_sweeps;
    while (left > 0) {
        int n = left;
        if (p->recompute_every > 0) n = (int)std::min<int64_t>(n, p->recompute_every - p->sweeps_since_recompute);
        int chunk = n;
        if (p->engine != XYL_FP32_BATCHED) chunk = std::min(n, kGraphChunk);
        if ((rc = run_captured(p, chunk, ops, measure_every, st))) return rc;
        p->last_launches += launches_of(p, chunk, ops);
        left -= chunk;
        p->sweeps_since_recompute += chunk;
        if (p->recompute_every > 0 && p->sweeps_since_recompute >= p->recompute_every) {
            if ((rc = do_recompute(p, 1, st))) return rc;
            p->last_launches += 1;
            p->sweeps_since_recompute = 0;
        }
    }
    return XYL_OK;
}

int xyl_sweep_units(xyl_plan *p, int32_t first_unit, int32_t n_units, int32_t n_sweeps, uint32_t ops,
                    int32_t measure_every, void *stream)
{
    CallRange range_("xyl_sweep_units");
    clear_error();
    int rc = check_bound(p, "xyl_sweep_units");
    if (rc) return rc;
    if (p->engine != XYL_FP32_BATCHED) return fail(XYL_EINVAL, "xyl_sweep_units: batched engine only");
    const int total = (int)p->units.size();
    if (first_unit < 0 || n_units < 1 || first_unit + n_units > total || n_sweeps < 0)
        return fail(XYL_EINVAL, "xyl_sweep_units: bad unit range [%d, %d) of %d", first_unit, first_unit + n_units, total);
    if (!(ops & (XYL_OP_MET | XYL_OP_OR))) return fail(XYL_EINVAL, "xyl_sweep_units: ops must include MET or OR");
    if ((ops & XYL_OP_MEASURE) && measure_every < 1) return fail(XYL_EINVAL, "xyl_sweep_units: measure_every must be >= 1");
    if (!(ops & XYL_OP_MEASURE)) measure_every = 1;
    cudaStream_t st = as_stream(stream);
    p->last_launches = 0;
    // the range may span parts: each part runs its own units of it
    for (const Part &part : p->parts) {
        const int lo = std::max(first_unit, part.u0);
        const int hi = std::min(first_unit + n_units, part.u0 + (int)part.units.size());
        if (lo >= hi) continue;
        if (part.B.resident && ((lo - part.u0) % part.B.gpc || (hi - lo) % part.B.gpc))
            return fail(XYL_EINVAL, "xyl_sweep_units: a resident cluster runs %d units together", part.B.gpc);
    }
    XYL_CUDA(cudaMemsetAsync(p->ws + p->r_barrier.off, 0, p->r_barrier.bytes, st), "xyl_sweep_units: barrier reset");
    for (const Part &part : p->parts) {
        const int lo = std::max(first_unit, part.u0);
        const int hi = std::min(first_unit + n_units, part.u0 + (int)part.units.size());
        if (lo >= hi) continue;
        if ((rc = launch_units(p, p->dev, part, lo, hi - lo, n_sweeps, ops, measure_every, st, &p->last_launches)))
            return rc;
    }
    return XYL_OK;
}

int xyl_sweep_noalloc(xyl_plan *p, int32_t n_sweeps, uint32_t ops, int32_t measure_every, void *stream)
{
    clear_error();
    int rc = check_bound(p, "xyl_sweep_noalloc");
    if (rc) return rc;
    if (p->engine != XYL_FP32_BATCHED) return fail(XYL_EINVAL, "xyl_sweep_noalloc: batched engine only");
    if (n_sweeps < 0) return fail(XYL_EINVAL, "xyl_sweep_noalloc: n_sweeps < 0");
    if (!(ops & (XYL_OP_MET | XYL_OP_OR))) return fail(XYL_EINVAL, "xyl_sweep_noalloc: ops must include MET or OR");
    if (ops & ~(XYL_OP_MET | XYL_OP_OR | XYL_OP_PT | XYL_OP_MEASURE))
        return fail(XYL_EINVAL, "xyl_sweep_noalloc: unknown op bits");
    if ((ops & XYL_OP_MEASURE) && measure_every < 1)
        return fail(XYL_EINVAL, "xyl_sweep_noalloc: measure_every must be >= 1");
    if (!(ops & XYL_OP_MEASURE)) measure_every = 1;
    // scratch: the two per-replica sum buffers, then the per-sample barrier counters
    const size_t obs_bytes = 2 * (size_t)p->total_R * kObsStride * sizeof(double);
    const size_t bar_off = align_up(obs_bytes);
    const size_t need = bar_off + p->hs.size() * sizeof(unsigned int);
    if (need > kNoAllocScratchBytes)
        return fail(XYL_EINVAL, "xyl_sweep_noalloc: batch needs %zu B of scratch, the fixed array holds %zu B "
                    "(%d slots and %zu samples; use xyl_sweep)", need, kNoAllocScratchBytes, p->total_R, p->hs.size());
    p->last_launches = 0;
    if (n_sweeps == 0) return XYL_OK;  // like xyl_sweep: nothing runs, the shared array is not touched
    void *scratch = nullptr;
    XYL_CUDA(batched_noalloc_scratch(&scratch), "xyl_sweep_noalloc: scratch address");
    cudaStream_t st = as_stream(stream);
    char *base = static_cast<char *>(scratch);
    DevPlan P = p->dev;
    P.obs = reinterpret_cast<double *>(base);
    P.barrier = reinterpret_cast<unsigned int *>(base + bar_off);
    // the sweeps are cut at the FP64 recompute points exactly as xyl_sweep cuts them
    int left = n_sweeps;
    while (left > 0) {
        int n = left;
        if (p->recompute_every > 0) n = (int)std::min<int64_t>(n, p->recompute_every - p->sweeps_since_recompute);
        // every launch finds the sum buffer of its first sweep and the barrier counters at zero
        XYL_CUDA(cudaMemsetAsync(base, 0, need, st), "xyl_sweep_noalloc: clear scratch");
        if ((rc = issue_batched(p, P, n, ops, measure_every, st, &p->last_launches, false))) return rc;
        left -= n;
        p->sweeps_since_recompute += n;
        if (p->recompute_every > 0 && p->sweeps_since_recompute >= p->recompute_every) {
            if ((rc = do_recompute(p, 1, st))) return rc;
            p->last_launches += 1;
            p->sweeps_since_recompute = 0;
        }
    }
    // xyl_sweep's kernels add into the plan's own sum buffer of their first
    // sweep and expect it cleared; these sweeps moved the sweep parity without
    // touching that buffer, so clear it here (a memset of the caller's
    // workspace: nothing is allocated)
    return zero_region(p, p->r_obs, st);
}

int32_t xyl_unit_count(const xyl_plan *p)
{
    return (p && p->engine == XYL_FP32_BATCHED) ? (int32_t)p->units.size() : 0;
}

int32_t xyl_wave_units(const xyl_plan *p)
{
    return (p && p->engine == XYL_FP32_BATCHED && p->bound) ? (int32_t)p->parts[0].wave_units : 0;
}

int32_t xyl_live_units(const xyl_plan *p)
{
    return (p && p->engine == XYL_FP32_BATCHED && p->bound) ? (int32_t)p->parts[0].live_units : 0;
}

int32_t xyl_part_count(const xyl_plan *p)
{
    return (p && p->engine == XYL_FP32_BATCHED) ? (int32_t)p->parts.size() : 0;
}

int xyl_pt_swap(xyl_plan *p, void *stream)
{
    CallRange range_("xyl_pt_swap");
    clear_error();
    int rc = check_bound(p, "xyl_pt_swap");
    if (rc) return rc;
    cudaStream_t st = as_stream(stream);
    XYL_CUDA(launch_recompute(p->dev, p->shape, 0, buffer_mode(p), st), "xyl_pt_swap: recompute");
    XYL_CUDA(launch_finalize(p->dev, p->shape, XYL_OP_PT, 1, 0, buffer_mode(p), st), "xyl_pt_swap: finalize");
    // the batched kernels add the next sweep's sums into a cleared buffer
    return buffer_mode(p) ? zero_region(p, p->r_obs, st) : XYL_OK;
}

int xyl_measure(xyl_plan *p, void *stream)
{
    CallRange range_("xyl_measure");
    clear_error();
    int rc = check_bound(p, "xyl_measure");
    if (rc) return rc;
    cudaStream_t st = as_stream(stream);
    XYL_CUDA(launch_recompute(p->dev, p->shape, 0, buffer_mode(p), st), "xyl_measure: recompute");
    XYL_CUDA(launch_finalize(p->dev, p->shape, XYL_OP_MEASURE, 1, 0, buffer_mode(p), st), "xyl_measure: finalize");
    return buffer_mode(p) ? zero_region(p, p->r_obs, st) : XYL_OK;
}

int xyl_recompute(xyl_plan *p, void *stream)
{
    CallRange range_("xyl_recompute");
    clear_error();
    int rc = check_bound(p, "xyl_recompute");
    if (rc) return rc;
    return do_recompute(p, 1, as_stream(stream));
}

int xyl_set_delta(xyl_plan *p, int32_t sample, const double *delta, void *stream)
{
    clear_error();
    int rc = check_bound(p, "xyl_set_delta");
    if (rc) return rc;
    if (sample < 0 || sample >= (int)p->hs.size() || !delta) return fail(XYL_EINVAL, "xyl_set_delta: bad sample");
    HostSample &h = p->hs[sample];
    int rep_off = 0;
    for (int s = 0; s < sample; ++s) rep_off += p->hs[s].R;
    for (int k = 0; k < h.R; ++k) {
        if (!std::isfinite(delta[k]) || delta[k] < 0) return fail(XYL_EINVAL, "xyl_set_delta: bad delta");
        h.delta[k] = delta[k];
    }
    cudaStream_t st = as_stream(stream);
    XYL_CUDA(cudaMemcpyAsync(p->ws + p->r_delta.off + rep_off * sizeof(double), h.delta.data(), h.R * sizeof(double),
                             cudaMemcpyHostToDevice, st), "xyl_set_delta: copy");
    XYL_CUDA(cudaStreamSynchronize(st), "xyl_set_delta: sync");
    // graphs hold kernel arguments only (pointers), so they stay valid
    return XYL_OK;
}

int xyl_get_delta(const xyl_plan *p, int32_t sample, double *delta)
{
    clear_error();
    if (!p || !delta) return fail(XYL_EINVAL, "xyl_get_delta: NULL argument");
    if (sample < 0 || sample >= (int)p->hs.size()) return fail(XYL_EINVAL, "xyl_get_delta: bad sample");
    const HostSample &h = p->hs[sample];
    std::copy(h.delta.begin(), h.delta.end(), delta);
    return XYL_OK;
}

int xyl_tune_delta(xyl_plan *p, int32_t rounds, int32_t n_sweeps, uint32_t ops, double target, double *rate,
                   void *stream)
{
    CallRange range_("xyl_tune_delta");
    clear_error();
    int rc = check_bound(p, "xyl_tune_delta");
    if (rc) return rc;
    if (rounds < 0 || n_sweeps < 1 || !(ops & XYL_OP_MET) || !(target > 0.0 && target < 1.0))
        return fail(XYL_EINVAL, "xyl_tune_delta: need rounds >= 0, n_sweeps >= 1, XYL_OP_MET and 0 < target < 1");
    ops &= (XYL_OP_MET | XYL_OP_OR | XYL_OP_PT);
    cudaStream_t st = as_stream(stream);
    const size_t slots = (size_t)p->total_R;
    std::vector<uint64_t> acc(slots), tries(slots);
    std::vector<double> last(slots, 0.0);
    for (int round = 0; round <= rounds; ++round) {
        if ((rc = xyl_reset_observables(p, stream))) return rc;
        if ((rc = xyl_sweep(p, n_sweeps, ops, 1, stream))) return rc;
        if ((rc = xyl_read_observables(p, nullptr, acc.data(), tries.data(), nullptr, nullptr, stream))) return rc;
        size_t k = 0;
        for (size_t s = 0; s < p->hs.size(); ++s) {
            HostSample &h = p->hs[s];
            std::vector<double> d(h.delta);
            for (int j = 0; j < h.R; ++j, ++k) {
                last[k] = tries[k] ? (double)acc[k] / (double)tries[k] : 0.0;
                // acceptance falls as the step grows: scale the step by the ratio
                // of the measured to the wanted acceptance, at most x2 or /2 per
                // round, within [1e-3, pi]
                const double f = std::min(2.0, std::max(0.5, last[k] / target));
                d[j] = std::min(M_PI, std::max(1e-3, d[j] * f));
            }
            // the last round only measures the frozen widths
            if (round < rounds && (rc = xyl_set_delta(p, (int32_t)s, d.data(), stream))) return rc;
        }
    }
    if (rate) std::copy(last.begin(), last.end(), rate);
    return xyl_reset_observables(p, stream);
}

static int read_region(xyl_plan *p, const Region &r, void *dst, cudaStream_t st)
{
    if (!dst) return XYL_OK;
    XYL_CUDA(cudaMemcpyAsync(dst, p->ws + r.off, r.bytes, cudaMemcpyDeviceToHost, st), "read");
    return XYL_OK;
}

static int finish_read(xyl_plan *p, cudaStream_t st)
{
    XYL_CUDA(cudaStreamSynchronize(st), "read: sync");
    int32_t status = 0;
    XYL_CUDA(cudaMemcpy(&status, p->ws + p->r_status.off, sizeof(status), cudaMemcpyDeviceToHost), "read: status");
    if (status) return fail(status, "device status word is %d", status);
    return XYL_OK;
}

int xyl_read_observables(xyl_plan *p, double *acc, uint64_t *met_acc, uint64_t *met_try, uint64_t *pt_acc,
                         uint64_t *pt_try, void *stream)
{
    clear_error();
    int rc = check_bound(p, "xyl_read_observables");
    if (rc) return rc;
    cudaStream_t st = as_stream(stream);
    if ((rc = read_region(p, p->r_acc, acc, st))) return rc;
    if ((rc = read_region(p, p->r_met_acc, met_acc, st))) return rc;
    if ((rc = read_region(p, p->r_met_try, met_try, st))) return rc;
    if ((rc = read_region(p, p->r_pt_acc, pt_acc, st))) return rc;
    if ((rc = read_region(p, p->r_pt_try, pt_try, st))) return rc;
    return finish_read(p, st);
}

int xyl_reset_observables(xyl_plan *p, void *stream)
{
    clear_error();
    int rc = check_bound(p, "xyl_reset_observables");
    if (rc) return rc;
    cudaStream_t st = as_stream(stream);
    const Region *zero[] = {&p->r_acc, &p->r_met_acc, &p->r_met_try, &p->r_pt_acc, &p->r_pt_try};
    for (const Region *r : zero)
        if ((rc = zero_region(p, *r, st))) return rc;
    return XYL_OK;
}

int xyl_read_energies(xyl_plan *p, double *E, void *stream)
{
    clear_error();
    int rc = check_bound(p, "xyl_read_energies");
    if (rc) return rc;
    cudaStream_t st = as_stream(stream);
    if ((rc = read_region(p, p->r_last_E, E, st))) return rc;
    return finish_read(p, st);
}

int xyl_read_labels(xyl_plan *p, int32_t *replica_at_slot, void *stream)
{
    clear_error();
    int rc = check_bound(p, "xyl_read_labels");
    if (rc) return rc;
    cudaStream_t st = as_stream(stream);
    if ((rc = read_region(p, p->r_rep_at, replica_at_slot, st))) return rc;
    return finish_read(p, st);
}

static int spin_copy(xyl_plan *p, int32_t sample, int32_t replica, double *out, const double *in, cudaStream_t st)
{
    if (sample < 0 || sample >= (int)p->hs.size()) return fail(XYL_EINVAL, "spins: bad sample %d", sample);
    const HostSample &h = p->hs[sample];
    if (replica < 0 || replica >= h.R) return fail(XYL_EINVAL, "spins: bad replica %d", replica);
    int64_t spin_off = 0;
    for (int s = 0; s < sample; ++s) spin_off += (int64_t)p->hs[s].N * p->hs[s].R;
    const size_t elem = p->spin_elem();
    char *base = p->ws + p->r_spins.off + spin_off * elem;
    std::vector<char> buf((size_t)h.N * elem);
    const bool inter = p->shape.layout == kInterleaved;
    char *dev = inter ? base + (size_t)replica * elem : base + (size_t)replica * h.N * elem;
    const size_t pitch = inter ? (size_t)h.R * elem : elem;
    const int dim = p->shape.dim;
    if (out) {
        XYL_CUDA(cudaMemcpy2DAsync(buf.data(), elem, dev, pitch, elem, h.N, cudaMemcpyDeviceToHost, st), "spins: copy");
        XYL_CUDA(cudaStreamSynchronize(st), "spins: sync");
        for (int i = 0; i < h.N; ++i) {
            const int v = h.perm[i];
            if (dim == 3 && p->shape.fp64) {
                const double4_32a s = reinterpret_cast<const double4_32a *>(buf.data())[i];
                out[3 * v] = s.x; out[3 * v + 1] = s.y; out[3 * v + 2] = s.z;
            } else if (dim == 3) {
                const float4 s = reinterpret_cast<const float4 *>(buf.data())[i];
                out[3 * v] = s.x; out[3 * v + 1] = s.y; out[3 * v + 2] = s.z;
            } else if (p->shape.fp64) {
                const double2 s = reinterpret_cast<const double2 *>(buf.data())[i];
                out[2 * v] = s.x; out[2 * v + 1] = s.y;
            } else {
                const float2 s = reinterpret_cast<const float2 *>(buf.data())[i];
                out[2 * v] = s.x; out[2 * v + 1] = s.y;
            }
        }
        return finish_read(p, st);
    }
    for (int i = 0; i < h.N; ++i) {
        const int v = h.perm[i];
        if (dim == 3 && p->shape.fp64) {
            double4_32a s;
            s.x = in[3 * v]; s.y = in[3 * v + 1]; s.z = in[3 * v + 2]; s.w = 0.0;
            reinterpret_cast<double4_32a *>(buf.data())[i] = s;
        } else if (dim == 3) {
            reinterpret_cast<float4 *>(buf.data())[i] =
                make_float4((float)in[3 * v], (float)in[3 * v + 1], (float)in[3 * v + 2], 0.0f);
        } else if (p->shape.fp64)
            reinterpret_cast<double2 *>(buf.data())[i] = make_double2(in[2 * v], in[2 * v + 1]);
        else
            reinterpret_cast<float2 *>(buf.data())[i] = make_float2((float)in[2 * v], (float)in[2 * v + 1]);
    }
    XYL_CUDA(cudaMemcpy2DAsync(dev, pitch, buf.data(), elem, elem, h.N, cudaMemcpyHostToDevice, st), "spins: copy");
    XYL_CUDA(cudaStreamSynchronize(st), "spins: sync");
    return XYL_OK;
}

int xyl_read_spins(xyl_plan *p, int32_t sample, int32_t replica, double *sxy, void *stream)
{
    clear_error();
    int rc = check_bound(p, "xyl_read_spins");
    if (rc) return rc;
    if (!sxy) return fail(XYL_EINVAL, "xyl_read_spins: NULL output");
    return spin_copy(p, sample, replica, sxy, nullptr, as_stream(stream));
}

int xyl_write_spins(xyl_plan *p, int32_t sample, int32_t replica, const double *sxy, void *stream)
{
    clear_error();
    int rc = check_bound(p, "xyl_write_spins");
    if (rc) return rc;
    if (!sxy) return fail(XYL_EINVAL, "xyl_write_spins: NULL input");
    cudaStream_t st = as_stream(stream);
    if ((rc = spin_copy(p, sample, replica, nullptr, sxy, st))) return rc;
    // the energies of the new spins are not a drift of the FP32 update: keep
    // the recorded maximum as it was
    char *drift = p->ws + p->r_drift.off;
    XYL_CUDA(cudaMemcpyAsync(drift + sizeof(double), drift, sizeof(double), cudaMemcpyDeviceToDevice, st),
             "xyl_write_spins: save drift");
    if ((rc = do_recompute(p, 0, st))) return rc;
    XYL_CUDA(cudaMemcpyAsync(drift, drift + sizeof(double), sizeof(double), cudaMemcpyDeviceToDevice, st),
             "xyl_write_spins: restore drift");
    return XYL_OK;
}

int xyl_check_plan(xyl_plan *p, int64_t *violations, void *stream)
{
    CallRange range_("xyl_check_plan");
    clear_error();
    int rc = check_bound(p, "xyl_check_plan");
    if (rc) return rc;
    if (!violations) return fail(XYL_EINVAL, "xyl_check_plan: NULL output");
    cudaStream_t st = as_stream(stream);
    unsigned long long *d = at<unsigned long long>(p, p->r_check);
    XYL_CUDA(cudaMemsetAsync(d, 0, sizeof(unsigned long long), st), "xyl_check_plan: clear");
    XYL_CUDA(launch_check(p->dev, p->shape, d, st), "xyl_check_plan: launch");
    unsigned long long n = 0;
    XYL_CUDA(cudaMemcpyAsync(&n, d, sizeof(n), cudaMemcpyDeviceToHost, st), "xyl_check_plan: copy");
    XYL_CUDA(cudaStreamSynchronize(st), "xyl_check_plan: sync");
    *violations = (int64_t)n;
    return XYL_OK;
}

int xyl_read_drift(xyl_plan *p, double *max_drift, int32_t reset, void *stream)
{
    clear_error();
    int rc = check_bound(p, "xyl_read_drift");
    if (rc) return rc;
    if (!max_drift) return fail(XYL_EINVAL, "xyl_read_drift: NULL output");
    cudaStream_t st = as_stream(stream);
    XYL_CUDA(cudaMemcpyAsync(max_drift, p->ws + p->r_drift.off, sizeof(double), cudaMemcpyDeviceToHost, st),
             "xyl_read_drift: copy");
    if (reset) XYL_CUDA(cudaMemsetAsync(p->ws + p->r_drift.off, 0, sizeof(double), st), "xyl_read_drift: reset");
    return finish_read(p, st);
}

int xyl_read_status(xyl_plan *p, int32_t *status, uint64_t *sweep_index, void *stream)
{
    clear_error();
    int rc = check_bound(p, "xyl_read_status");
    if (rc) return rc;
    cudaStream_t st = as_stream(stream);
    XYL_CUDA(cudaStreamSynchronize(st), "xyl_read_status: sync");
    int32_t s = 0;
    uint32_t t = 0;
    XYL_CUDA(cudaMemcpy(&s, p->ws + p->r_status.off, sizeof(s), cudaMemcpyDeviceToHost), "xyl_read_status");
    XYL_CUDA(cudaMemcpy(&t, p->ws + p->r_sweep.off, sizeof(t), cudaMemcpyDeviceToHost), "xyl_read_status");
    if (status) *status = s;
    if (sweep_index) *sweep_index = t;
    return XYL_OK;
}

}  // extern "C"

namespace {

std::vector<const Region *> state_regions(xyl_plan *p)
{
    return {&p->r_spins, &p->r_slot_of, &p->r_rep_at, &p->r_sweep, &p->r_last_E, &p->r_acc,
            &p->r_met_acc, &p->r_met_try, &p->r_pt_acc, &p->r_pt_try, &p->r_drift};
}

}  // namespace

extern "C" {

size_t xyl_state_bytes(const xyl_plan *p)
{
    if (!p) return 0;
    size_t n = 16;
    for (const Region *r : state_regions(const_cast<xyl_plan *>(p))) n += r->bytes;
    return n;
}

int xyl_export_state(xyl_plan *p, void *host, size_t bytes, void *stream)
{
    clear_error();
    int rc = check_bound(p, "xyl_export_state");
    if (rc) return rc;
    if (!host || bytes < xyl_state_bytes(p)) return fail(XYL_ENOSPC, "xyl_export_state: buffer too small");
    cudaStream_t st = as_stream(stream);
    char *dst = static_cast<char *>(host);
    const uint64_t magic = 0x584C5953544154ull, size = xyl_state_bytes(p);
    std::memcpy(dst, &magic, 8);
    std::memcpy(dst + 8, &size, 8);
    size_t off = 16;
    for (const Region *r : state_regions(p)) {
        XYL_CUDA(cudaMemcpyAsync(dst + off, p->ws + r->off, r->bytes, cudaMemcpyDeviceToHost, st), "xyl_export_state");
        off += r->bytes;
    }
    return finish_read(p, st);
}

int xyl_import_state(xyl_plan *p, const void *host, size_t bytes, void *stream)
{
    clear_error();
    int rc = check_bound(p, "xyl_import_state");
    if (rc) return rc;
    if (!host || bytes < xyl_state_bytes(p)) return fail(XYL_EINVAL, "xyl_import_state: buffer too small");
    const char *src = static_cast<const char *>(host);
    uint64_t magic = 0, size = 0;
    std::memcpy(&magic, src, 8);
    std::memcpy(&size, src + 8, 8);
    if (magic != 0x584C5953544154ull || size != xyl_state_bytes(p))
        return fail(XYL_EINVAL, "xyl_import_state: not a checkpoint of this plan");
    cudaStream_t st = as_stream(stream);
    size_t off = 16;
    for (const Region *r : state_regions(p)) {
        XYL_CUDA(cudaMemcpyAsync(p->ws + r->off, src + off, r->bytes, cudaMemcpyHostToDevice, st), "xyl_import_state");
        off += r->bytes;
    }
    XYL_CUDA(cudaMemsetAsync(p->ws + p->r_obs.off, 0, p->r_obs.bytes, st), "xyl_import_state");
    XYL_CUDA(cudaMemsetAsync(p->ws + p->r_status.off, 0, p->r_status.bytes, st), "xyl_import_state");
    XYL_CUDA(cudaStreamSynchronize(st), "xyl_import_state: sync");
    return XYL_OK;
}

int64_t xyl_last_launch_count(const xyl_plan *p) { return p ? p->last_launches : 0; }

int xyl_get_part_tuning(const xyl_plan *p, int32_t part, xyl_tuning *out, int32_t *n_samples)
{
    if (!p || !out) return fail(XYL_EINVAL, "xyl_get_part_tuning: NULL argument");
    std::memset(out, 0, sizeof(*out));
    out->recompute_every = p->recompute_every;
    out->spin_dim = p->shape.dim;
    if (n_samples) *n_samples = 0;
    if (p->engine != XYL_FP32_BATCHED) return part == 0 ? XYL_OK : fail(XYL_EINVAL, "xyl_get_part_tuning: bad part");
    if (part < 0 || part >= (int)p->parts.size()) return fail(XYL_EINVAL, "xyl_get_part_tuning: bad part %d", part);
    const BatchedShape &B = p->parts[part].B;
    out->block = B.block;
    out->cluster = B.G;
    out->group = B.Rg;
    out->stage = B.staged ? 1 : -1;
    out->resident = B.resident ? 1 : -1;
    out->waves = B.l2_waves ? 1 : -1;
    out->span = B.span;
    if (n_samples) *n_samples = (int32_t)p->parts[part].samples.size();
    return XYL_OK;
}

int xyl_set_part_tuning(xyl_plan *p, int32_t part, const xyl_tuning *t, void *stream)
{
    clear_error();
    if (!p || !t) return fail(XYL_EINVAL, "xyl_set_part_tuning: NULL argument");
    if (p->engine != XYL_FP32_BATCHED) return fail(XYL_EINVAL, "xyl_set_part_tuning: batched engine only");
    if (part < 0 || part >= (int)p->parts.size()) return fail(XYL_EINVAL, "xyl_set_part_tuning: bad part %d", part);
    if (t->resident == 0 || t->group < 1 || t->cluster < 1 || t->block < 1)
        return fail(XYL_EINVAL, "xyl_set_part_tuning: resident (+-1), group, cluster and block must be given");
    Part &pt = p->parts[part];
    const Part keep = pt;
    int rc = apply_shape(p, pt, t->group, t->cluster, t->block, t->stage, t->resident > 0 ? 1 : 0,
                         t->waves > 0 ? 1 : 0, t->span > 0 ? t->span : 1);
    if (!rc && p->bound) {
        cudaStream_t st = as_stream(stream);
        rc = configure_part(p, pt, st);
        if (!rc) rc = finish_configure(p, st);
    }
    if (rc) {
        pt = keep;  // the part keeps its shape
        gather_units(p);
        return rc;
    }
    if (!p->bound) gather_units(p);
    return XYL_OK;
}

int xyl_get_tuning(const xyl_plan *p, xyl_tuning *out)
{
    if (!p || !out) return fail(XYL_EINVAL, "xyl_get_tuning: NULL argument");
    return xyl_get_part_tuning(p, 0, out, nullptr);
}

int xyl_autotune(xyl_plan *p, int32_t n_sweeps, uint32_t ops, int32_t measure_every, xyl_tuning *best,
                 void *stream)
{
    CallRange range_("xyl_autotune");
    clear_error();
    int rc = check_bound(p, "xyl_autotune");
    if (rc) return rc;
    if (p->engine != XYL_FP32_BATCHED) return fail(XYL_EINVAL, "xyl_autotune: batched engine only");
    if (n_sweeps < 1 || !(ops & (XYL_OP_MET | XYL_OP_OR))) return fail(XYL_EINVAL, "xyl_autotune: bad sweep request");
    if ((ops & XYL_OP_MEASURE) && measure_every < 1) return fail(XYL_EINVAL, "xyl_autotune: measure_every must be >= 1");
    if (!(ops & XYL_OP_MEASURE)) measure_every = 1;
    cudaStream_t st = as_stream(stream);
    // the state is saved once and restored once: the timed tries advance the
    // chain, which does not change how long a sweep takes
    std::vector<char> snap(xyl_state_bytes(p));
    if ((rc = xyl_export_state(p, snap.data(), snap.size(), stream))) return rc;
    cudaEvent_t e0, e1;
    XYL_CUDA(cudaEventCreate(&e0), "xyl_autotune: event");
    XYL_CUDA(cudaEventCreate(&e1), "xyl_autotune: event");
    int dev = 0, n_sm = 0, l2 = 0;
    XYL_CUDA(cudaGetDevice(&dev), "xyl_autotune: device");
    XYL_CUDA(cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev), "xyl_autotune: SM count");
    XYL_CUDA(cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev), "xyl_autotune: L2 size");
    bool any = false;
    // each part on its own: its launches alone are timed for every shape
    for (Part &part : p->parts) {
        const BatchedShape keep = part.B;
        const int keep_stage = part.stage_mode;
        float best_ms = -1.f;
        int best_g = keep.Rg, best_G = keep.G, best_block = keep.block, best_res = keep.resident ? 1 : 0;
        int best_waves = keep.l2_waves ? 1 : 0, best_span = keep.span;
        size_t live = 0;
        int64_t spins = 0;
        for (int si : part.samples) {
            live += sample_live_bytes(p->hs[si]);
            spins += (int64_t)p->hs[si].N * p->hs[si].R;
        }
        // L2-sized waves change nothing when the whole part fits in L2
        const bool try_waves = live > (size_t)l2 * 3 / 4 && p->waves_req >= 0;
        const bool large = spins >= ((int64_t)1 << 26);
        for (int res = 0; res <= 1; ++res) {
            if ((p->resident_req < 0 && res) || (p->resident_req > 0 && !res)) continue;
            for (int waves = 0; waves <= (res ? 0 : 1); ++waves) {
                if (waves ? !try_waves : p->waves_req > 0) continue;
                for (int g = 1; g <= 32; ++g) {
                    // resident: powers of two; global memory: also even groups from 6
                    // (one group per sample where n_temps is not a power of two)
                    if ((g & (g - 1)) && (res || g % 2 || g < 6)) continue;
                    bool divides = true;
                    for (int si : part.samples) divides &= (p->hs[si].R % g == 0);
                    if (!divides) continue;
                    int64_t units = 0;
                    for (int si : part.samples) units += p->hs[si].R / g;
                    for (int G : {1, 2, 3, 4, 5, 6, 7, 8, 12, 16}) {
                        if (p->shape.dim == 3 && (G > 1 || !res)) continue;  // O(3): resident, one CTA per group
                        // global-memory shape: powers of two and 6, 12 (a GPC holds two
                        // clusters of 6 or 8 but one of 12 or 16); split a resident
                        // group across CTAs only while the batch leaves SMs idle
                        if (!res && (G & (G - 1)) && G != 6 && G != 12) continue;
                        if (res && G > 1 && units * G > 2 * (int64_t)n_sm) continue;
                        for (int block : {128, 256, 384, 512, 640, 768, 1024}) {
                            if (res ? block == 128 : block == 384) continue;
                            if (!res && large && block < 512) continue;  // large samples: many items per CTA
                            // one unit per span of clusters: span 1, and (one group per sample,
                            // large samples) a sample spread over every cluster that fits, or half
                            int spans[3] = {1, 0, 0};
                            for (int k = 0; k < 3; ++k) {
                                const int span = spans[k];
                                if (span < 1) continue;
                                if (apply_shape(p, part, g, G, block, keep_stage, res, waves, span) ||
                                    configure_part(p, part, st) || finish_configure(p, st))
                                    continue;
                                if (k == 0 && !res && !waves && large && G <= 8 && units == (int64_t)part.samples.size()) {
                                    spans[1] = part.max_clusters;
                                    spans[2] = part.max_clusters / 2;
                                }
                                float ms = 0.f, rep_ms = 0.f;
                                bool ok = true;
                                for (int rep = 0; rep < 2 && ok; ++rep) {
                                    // a shape already 1.5x slower than the best on its first timing cannot win
                                    if (rep == 1 && best_ms > 0.f && ms > 1.5f * best_ms) break;
                                    int64_t launches = 0;
                                    XYL_CUDA(cudaMemsetAsync(p->ws + p->r_barrier.off, 0, p->r_barrier.bytes, st),
                                             "xyl_autotune");
                                    XYL_CUDA(cudaEventRecord(e0, st), "xyl_autotune: record");
                                    if (launch_units(p, p->dev, part, part.u0, (int)part.units.size(), n_sweeps, ops,
                                                     measure_every, st, &launches)) {
                                        ok = false;
                                        break;
                                    }
                                    XYL_CUDA(cudaEventRecord(e1, st), "xyl_autotune: record");
                                    XYL_CUDA(cudaEventSynchronize(e1), "xyl_autotune: sync");
                                    XYL_CUDA(cudaEventElapsedTime(&rep_ms, e0, e1), "xyl_autotune: time");
                                    ms = rep == 0 ? rep_ms : std::min(ms, rep_ms);  // the faster of the two timings
                                    int32_t status = 0;
                                    XYL_CUDA(cudaMemcpy(&status, p->ws + p->r_status.off, sizeof(status),
                                                        cudaMemcpyDeviceToHost), "xyl_autotune: status");
                                    if (status) {
                                        ok = false;
                                        XYL_CUDA(cudaMemset(p->ws + p->r_status.off, 0, sizeof(int32_t)),
                                                 "xyl_autotune: status");
                                    }
                                }
                                clear_error();
                                if (ok && (best_ms < 0.f || ms < best_ms)) {
                                    best_ms = ms;
                                    best_g = g;
                                    best_G = G;
                                    best_block = block;
                                    best_res = res;
                                    best_waves = waves;
                                    best_span = span;
                                }
                            }
                        }
                    }
                }
            }
        }
        any |= best_ms >= 0.f;
        if ((rc = apply_shape(p, part, best_g, best_G, best_block, keep_stage, best_res, best_waves, best_span)))
            return rc;
        if ((rc = configure_part(p, part, st))) return rc;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if ((rc = finish_configure(p, st))) return rc;
    if ((rc = xyl_import_state(p, snap.data(), snap.size(), stream))) return rc;
    if (best) xyl_get_tuning(p, best);
    return any ? XYL_OK : fail(XYL_EINVAL, "xyl_autotune: no launch shape ran");
}

void xyl_plan_free(xyl_plan *p) { delete p; }

}  // extern "C"
