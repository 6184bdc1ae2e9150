// Launchers of the device engines (host side), shared by the API layer.
#pragma once

#include <cuda_runtime.h>

#include <vector>

#include "device.cuh"

namespace xyl {

enum Layout : int { kReplicaMajor = 0, kInterleaved = 1 };

struct PlanShape {
    int n_samples = 0;
    int max_R = 0;
    int max_Q = 0;
    int max_class = 0;
    std::vector<int> class_max;  // per colour index: largest class of that colour over the samples
    int max_N = 0;
    int layout = kReplicaMajor;
    bool fp64 = false;
    bool coupled = false;   // some link has J = -1: neighbour ids carry J in bit 31
    bool fields = false;    // sites carry a field vector (DevPlan::field)
    bool disorder = false;  // coupled || fields: the kernels' DISORDER variants run
    int dim = 2;            // spin components: 2 (XY) or 3 (O(3), plain engines)
};

// Batched-engine launch shape chosen by the tuner.
struct BatchedShape {
    int G = 1;              // CTAs per cluster (one team per replica group)
    int span = 1;           // global-memory shape: clusters per replica group (above 1 they meet at a
                            // bounded global barrier after every colour phase)
    int Rg = 1;             // replicas per group (divides every R, <= 32; a power of two, or even in the global shape)
    int block = 512;        // threads per CTA
    bool staged = false;    // CSR rows of each CTA's chunks held in shared memory
    int owned_max = 0;      // largest number of sites one CTA owns
    int max_deg = 0;
    int fixed_deg = 0;      // degree shared by every site of every sample, 0 if degrees differ
    bool disorder = false;  // random bonds or fields (see PlanShape)
    size_t smem_bytes = 0;  // dynamic shared memory per CTA
    // resident shape: one CTA per replica group holds the group's spins of
    // every site in shared memory; the groups of a sample form one cluster
    bool resident = false;
    bool l2_waves = false;  // global-memory shape: launch waves hold as many samples as fit in L2
    int dim = 2;            // spin components: 3 runs the O(3) resident kernel
    int o3_comp = 0;        // O(3) resident: floats in each spin component array
    int gpc = 1;            // replica groups per cluster (resident shape)
    int cpc = 1;            // CTAs per cluster of the resident shape, G x gpc
    int rs_csr_w = 0;       // staged CSR row width (16-bit ids), 0 = rows from global memory
    bool rs_ids = false;    // random-stream site ids staged (16-bit)
    size_t rs_off_ids = 0, rs_off_col = 0, rs_off_part = 0, rs_off_met = 0, rs_off_peers = 0;
    size_t rs_off_beta = 0; // FP64 slot inverse temperatures of the sample
};

// Shared memory a CTA may use for staged CSR rows.
constexpr size_t kStageLimitBytes = 160 * 1024;
// Dynamic shared memory of a resident-shape CTA (spins, staged tables, partial sums).
constexpr size_t kResidentDynLimitBytes = 220 * 1024;
// Resident CTAs above this many threads use the 64-register kernel (up to 1024 threads).
constexpr int kResidentNarrowMaxThreads = 672;

// Fixed scratch of xyl_sweep_noalloc (per GPU, for the life of the library).
constexpr size_t kNoAllocScratchBytes = 1u << 20;
constexpr int kMaxDevicesNoAlloc = 64;
cudaError_t batched_noalloc_scratch(void **ptr);

cudaError_t launch_init(const DevPlan &P, const PlanShape &S, int aligned, cudaStream_t st);
cudaError_t launch_check(const DevPlan &P, const PlanShape &S, unsigned long long *violations, cudaStream_t st);
cudaError_t launch_finalize(const DevPlan &P, const PlanShape &S, uint32_t ops, int measure_every, int advance,
                            int obs_buf_from_sweep, cudaStream_t st);
cudaError_t launch_recompute(const DevPlan &P, const PlanShape &S, int renormalise, int obs_buf_from_sweep,
                             cudaStream_t st);
cudaError_t launch_plain_sweep(const DevPlan &P, const PlanShape &S, uint32_t ops, int measure_every,
                               cudaStream_t st, int64_t *launches);

// O(3) spins (plain engines): initialisation, one sweep, FP64 recompute.
cudaError_t launch_o3_init(const DevPlan &P, const PlanShape &S, int aligned, cudaStream_t st);
cudaError_t launch_o3_sweep(const DevPlan &P, const PlanShape &S, uint32_t ops, int measure_every,
                            cudaStream_t st, int64_t *launches);
cudaError_t launch_o3_recompute(const DevPlan &P, const PlanShape &S, int renormalise, int buffer_mode,
                                cudaStream_t st);

// Batched engine: one launch per wave of samples; `units` lists (sample, group) per cluster.
cudaError_t launch_batched(const DevPlan &P, const PlanShape &S, const BatchedShape &B, const int2 *d_units,
                           unsigned int *unit_ctr, int unit_begin, int unit_count, int n_sweeps, uint32_t ops,
                           int measure_every, cudaStream_t st);
cudaError_t batched_max_active_clusters(const PlanShape &S, const BatchedShape &B, int *clusters);
size_t batched_static_smem_bytes();

// Resident shape: one launch over units [unit_begin, unit_begin + unit_count), a multiple of gpc.
cudaError_t launch_resident(const DevPlan &P, const BatchedShape &B, const int2 *d_units, int unit_begin,
                            int unit_count, int n_sweeps, uint32_t ops, int measure_every, cudaStream_t st);
cudaError_t resident_max_active_clusters(const BatchedShape &B, int *clusters);
size_t resident_static_smem_bytes();

// Resident shape for O(3) spins (one CTA per replica group, G = 1).
cudaError_t launch_resident_o3(const DevPlan &P, const BatchedShape &B, const int2 *d_units, int unit_begin,
                               int unit_count, int n_sweeps, uint32_t ops, int measure_every, cudaStream_t st);
cudaError_t resident_o3_max_active_clusters(const BatchedShape &B, int *clusters);

}  // namespace xyl
