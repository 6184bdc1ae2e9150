/*
 * xyl.h -- C ABI of the GB300 (sm_103a) Monte Carlo library for the XY model on
 * dilute Levy graphs (Ibanez Berganza & Leuzzi, "Critical behavior of the XY
 * model in complex topologies").
 *
 * Model, Eq. (HXY): H = -sum_{i<j} J_ij S_i . S_j with S_i a unit 2-vector and
 * J_ij in {0,1} the adjacency of the graph.  Variants the method carries over
 * to (App. B): random couplings J = +-1 per link, random fields -sum h_i . S_i,
 * and O(3) spins (unit 3-vectors; xyl_tuning.spin_dim = 3).
 * Graph, Eq. (Levyi): sites of an L x L square lattice; a link lands at
 * distance r with probability proportional to r^-rho.  Two ensembles: every site carrying exactly z links
 * on the periodic lattice (xyl_build_graph_csr), or a fixed total of links with
 * free degrees on the periodic or free lattice, the paper's own (Sec. II,
 * xyl_build_levy_bonds).
 *
 * Conventions for every entry point:
 *   * The return value is a status: XYL_OK (0) or a negative XYL_E* code; the
 *     thread-local message of the last failure is xyl_last_error().  Nothing
 *     aborts, nothing prints.
 *   * Graph handles live in host memory and are owned by the library
 *     (xyl_graph_free).  Plans are host objects owned by the library
 *     (xyl_plan_free).
 *   * ALL device memory is owned by the caller: xyl_plan_create reports the
 *     workspace size, the caller allocates it (any allocator) and passes the
 *     device pointer to xyl_bind.  The library never allocates or frees device
 *     memory after that.
 *   * `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Device calls are asynchronous on that stream, except the
 *     xyl_read_* / xyl_export_state calls, which synchronise it before
 *     returning host data.
 *   * Sites have two numberings: the ORIGINAL id (x + L*y on the lattice, or the
 *     caller's id for xyl_graph_from_edges) and the colour-sorted id of the CSR.
 *     Random streams and every host-visible per-site array use original ids.
 *   * Threads: a plan (and the CUDA graphs it caches) serves one caller at a
 *     time; different plans may be used from different threads.  A graph is
 *     only read by xyl_plan_create (which copies what it needs), so it may be
 *     freed or changed afterwards.
 */
#ifndef XYL_H
#define XYL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define XYL_OK 0
#define XYL_EINVAL (-1)   /* bad argument */
#define XYL_ENOSPC (-2)   /* workspace too small */
#define XYL_EGRAPH (-3)   /* no valid graph within the restart limit */
#define XYL_ECUDA (-4)    /* a CUDA runtime call failed */
#define XYL_ETIMEOUT (-5) /* a bounded device-side wait gave up */
#define XYL_ESTATE (-6)   /* wrong call order (e.g. sweep before bind) */
#define XYL_EBOUNDS (-7)  /* debug builds (XYL_DEBUG) only: a kernel met an id outside its array and skipped it */

/* ---- sweep operations (bit mask) --------------------------------------- */
#define XYL_OP_MET 1u     /* Metropolis pass over the colour classes (App. B) */
#define XYL_OP_OR 2u      /* overrelaxation pass (App. B, Creutz reflection) */
#define XYL_OP_PT 4u      /* parallel-tempering swap attempt after the sweep */
#define XYL_OP_MEASURE 8u /* accumulate the Sec. III observables */

/* ---- engines ------------------------------------------------------------ */
#define XYL_FP64_PLAIN 0   /* FP64 unit vectors, one launch per colour phase */
#define XYL_FP32_BATCHED 1 /* FP32 unit vectors, persistent resident engine */
#define XYL_FP32_PLAIN 2   /* FP32 arithmetic on the per-phase launch structure */

/* ---- accumulator layout: per (sample, temperature slot), FP64 ----------- */
#define XYL_ACC_N 0     /* number of measurements */
#define XYL_ACC_E 1     /* sum of e = E/N */
#define XYL_ACC_E2 2    /* sum of e^2 */
#define XYL_ACC_ABSM 3  /* sum of |m| */
#define XYL_ACC_MX 4    /* sum of m_x */
#define XYL_ACC_MY 5    /* sum of m_y */
#define XYL_ACC_M2 6    /* sum of m^2 */
#define XYL_ACC_M4 7    /* sum of m^4 */
#define XYL_ACC_CHIK 8  /* sum of (|F(k1)|^2 + |F(k2)|^2) / (2N), k = 2 pi / L */
#define XYL_ACC_MZ 9    /* sum of m_z (O(3) spins; 0 for XY) */
#define XYL_ACC_COUNT 10

typedef struct xyl_graph xyl_graph;
typedef struct xyl_plan xyl_plan;

/* Thread-local description of the last failure ("" if none). */
const char *xyl_last_error(void);

/* ABI version of this header (major * 100 + minor). */
int xyl_version(void);

/* ========================================================================= */
/* Graphs (host)                                                             */
/* ========================================================================= */

/*
 * xyl_build_graph_csr -- one dilute Levy graph, Eq. (Levyi), and its
 * colour-sorted CSR (App. B "Graph coloring", "Memory management").
 *   L         even lattice side >= 4; N = L*L sites, periodic boundaries.
 *   z         links per site (every site exactly z); N*z must be even.
 *   rho       decay exponent of the link-length law r^-rho (minimum-image
 *             Euclidean r, displacements dx,dy in {-L/2+1..L/2}).
 *   seed      64-bit key of the graph random stream; sample_id selects an
 *             independent stream (disorder realisation).
 *   out       receives a new handle (free with xyl_graph_free).
 * Construction: sequential pairing; a uniformly chosen unsaturated site links
 * to an eligible partner (unsaturated, not yet linked, not itself) drawn with
 * the link law restricted to eligible partners; a dead end restarts the whole
 * graph (at most 100 restarts, then XYL_EGRAPH).  Colouring: smallest-last
 * ordering, ties by smallest id, greedy colours in reverse removal order.
 * Errors: XYL_EINVAL for bad sizes, XYL_EGRAPH as above.
 */
int xyl_build_graph_csr(int32_t L, int32_t z, double rho, uint64_t seed, uint32_t sample_id, xyl_graph **out);

/* ---- boundary conditions of xyl_build_levy_bonds ---------------------- */
#define XYL_PBC 0 /* periodic: minimum-image distances, r_max = (L/2) sqrt(2) */
#define XYL_FBC 1 /* free: distances inside the L x L square, r_max = L sqrt(2) */

/*
 * xyl_build_levy_bonds -- one graph of the paper's own ensemble (Sec. II,
 * Eq. (Levyi)): exactly n_bonds links (2N gives the mean degree 4 the paper
 * uses), each a pair of sites drawn with probability proportional to
 * |r_i - r_j|^-rho among all pairs of the lattice; degrees vary (Poisson with
 * mean 4 at rho = 0, the Erdos-Renyi limit).  Coloured and packed like
 * xyl_build_graph_csr.
 *   L         lattice side; XYL_PBC needs an even L in [4, 4096], XYL_FBC any
 *             L in [2, 4096]; N = L*L sites.
 *   rho       decay exponent of the link law (finite).
 *   n_bonds   number of links, 0 <= n_bonds <= N(N-1)/2.
 *   boundary  XYL_PBC or XYL_FBC.
 *   seed      64-bit key of the graph random stream; sample_id selects an
 *             independent stream (disorder realisation).
 *   out       receives a new handle (free with xyl_graph_free).
 * Draws: attempt a takes Philox block a of the graph stream (its own stream
 * id, apart from xyl_build_graph_csr's); the first site i from the first 64
 * bits (uniform over the N sites), the displacement from the second 64 bits
 * (the link-law table of the boundary condition); a partner outside the
 * square (XYL_FBC) or an existing link rejects the attempt.
 * Errors: XYL_EINVAL for bad arguments, XYL_EGRAPH when 64 n_bonds + 10^6
 * attempts do not give n_bonds distinct links.
 */
int xyl_build_levy_bonds(int32_t L, double rho, int64_t n_bonds, int32_t boundary, uint64_t seed, uint32_t sample_id,
                         xyl_graph **out);

/*
 * xyl_graph_from_edges -- a graph from an explicit simple edge list (for the
 * chain, ring and small-graph checks).  edges: 2*n_edges ids in [0,n), no
 * self-loops or repeated pairs (XYL_EINVAL otherwise).  xy: 2n lattice
 * coordinates used by the Fourier sums at k = 2 pi / L, or NULL (then x = id,
 * y = 0 and the period is n).  Coloured and packed like xyl_build_graph_csr.
 */
int xyl_graph_from_edges(int32_t n, int64_t n_edges, const int32_t *edges, const int32_t *xy, int32_t L,
                         xyl_graph **out);

/*
 * xyl_graph_set_couplings -- random bonds: H = -sum_(ij) J_ij S_i . S_j with
 * J_ij = +1 or -1 per link (the paper's method applied to "random bonds", App.
 * B; J = -1 everywhere on a bipartite graph is the antiferromagnet, random
 * signs the XY spin glass).  j: one value per link in creation order (the
 * order of xyl_graph_export_edges), each +1 or -1 (XYL_EINVAL otherwise), or
 * NULL to restore J = 1.  Plans made from the graph afterwards use the
 * couplings (a plan copies the graph when it is created).  Engines: every
 * engine; the resident shape of the batched engine keeps J in bit 15 of its
 * 16-bit staged rows, so with couplings it stages rows only when N <= 32767.
 */
int xyl_graph_set_couplings(xyl_graph *g, const int8_t *j);

/* Couplings of the CSR entries (2*n_edges values aligned with xyl_graph_export_csr's col). */
int xyl_graph_export_couplings(const xyl_graph *g, int8_t *j_csr);

/*
 * xyl_graph_set_fields -- random fields: H gains -sum_i h_i . S_i with one
 * field vector per site (the paper's method applied to "random fields", App.
 * B).  hxy: 2n values, (h_x, h_y) of each ORIGINAL site id, finite
 * (XYL_EINVAL otherwise), or NULL to remove the fields.  The local field of a
 * site becomes sum_j J_ij S_j + h_i (the neighbours summed first) and the
 * energies include the field term.  Plans made afterwards use the fields; a
 * plan with fields keeps one FP32 (FP64 for XYL_FP64_PLAIN) vector per site in
 * its workspace.  These are XY fields: a plan with O(3) spins refuses them
 * (XYL_EINVAL at xyl_plan_create).  Errors: XYL_EINVAL.
 */
int xyl_graph_set_fields(xyl_graph *g, const double *hxy);

/*
 * xyl_graph_set_fields3 -- random fields for O(3) spins: hxyz holds 3n values,
 * (h_x, h_y, h_z) of each ORIGINAL site id, finite (XYL_EINVAL otherwise), or
 * NULL to remove the fields.  As xyl_graph_set_fields otherwise: H gains
 * -sum_i h_i . S_i, the local field is sum_j J_ij S_j + h_i (the neighbours
 * summed first), the energies include the field term; a plan keeps one padded
 * 4-vector per site.  Only plans with spin_dim = 3 take them (XYL_EINVAL at
 * xyl_plan_create otherwise).  Errors: XYL_EINVAL.
 */
int xyl_graph_set_fields3(xyl_graph *g, const double *hxyz);

/* Sizes of a graph; any output pointer may be NULL.  restarts: pairing restarts used. */
int xyl_graph_info(const xyl_graph *g, int32_t *n, int64_t *n_edges, int32_t *n_colors, int32_t *max_deg,
                   int32_t *restarts);

/*
 * xyl_graph_export_csr -- copy out the colour-sorted CSR (host buffers owned by
 * the caller): perm[n] (colour-sorted id -> original id), row_ptr[n+1],
 * col[2*n_edges] (colour-sorted neighbour ids, ascending within a row),
 * color_ptr[n_colors+1] (first colour-sorted id of each colour).
 */
int xyl_graph_export_csr(const xyl_graph *g, int32_t *perm, int32_t *row_ptr, int32_t *col, int32_t *color_ptr);

/* Links in creation order (ei chose ej), original ids; n_edges entries each. */
int xyl_graph_export_edges(const xyl_graph *g, int32_t *ei, int32_t *ej);

void xyl_graph_free(xyl_graph *g);

/* ========================================================================= */
/* Plans: a batch of samples x temperature slots bound to one workspace       */
/* ========================================================================= */

typedef struct {
    const xyl_graph *graph; /* borrowed for the duration of xyl_plan_create */
    uint32_t sample_id;     /* keys the spin random streams of this sample */
    int32_t n_temps;        /* temperature slots = replicas of this sample */
    const double *beta;     /* n_temps inverse temperatures (slot order) */
    const double *delta;    /* n_temps Metropolis half-widths (slot order) */
} xyl_sample;

typedef struct {
    int32_t block;           /* threads per CTA of the batched engine, <= 1024 (0 = 512); above 672 the
                                global-memory shape reads its CSR rows from global memory */
    int32_t cluster;         /* CTAs per cluster of the batched engine (0 = tuned default) */
    int32_t group;           /* replicas per cluster, dividing every n_temps, <= 32: a power of two, or
                                even in the global-memory shape (0 = default) */
    int32_t recompute_every; /* FP64 energy recompute + renormalise every this many sweeps (0 = never) */
    int32_t stage;           /* batched engine: 0 = stage CSR rows in shared memory when they fit, -1 = never */
    int32_t resident;        /* batched engine: 1 = resident shape, -1 = never, 0 = library's choice (below) */
    int32_t spin_dim;        /* spin components: 0 or 2 = XY; 3 = O(3) (see below) */
    int32_t waves;           /* batched engine, global-memory shape: 1 = cap each launch wave to the samples whose
                                spins and tables fit in L2, -1 = never, 0 = library's choice (never) */
    int32_t span;            /* batched engine, global-memory shape: clusters per replica group (0 or 1 = one); above
                                one (group a power of two >= 2), the group's cluster x span CTAs share its colour
                                chunks and meet at a bounded
                                global barrier after every colour phase, so few samples can hold the whole GPU while
                                their spins stay in L2 for a launch's sweeps; all must be resident at once */
} xyl_tuning;

/*
 * O(3) spins (spin_dim = 3; App. B names O(3) among the continuous models the
 * method carries over to).  Same Hamiltonian with three-component unit
 * vectors, same sweep, parallel tempering and measurements; m^2, m^4 and
 * chi(k) take all three components and XYL_ACC_MZ sums m_z.  Initial spins
 * are uniform on the sphere: z = 2u - 1, phi = 2 pi u' - pi from the INIT
 * block of (site, replica) (u53(w0,w1), u53(w2,w3) in FP64; u24(w0), u24(w1)
 * in FP32), aligned = (1, 0, 0).  Metropolis proposes a point uniform on the
 * spherical cap of angular radius Delta around S: 1 - cos theta =
 * u * 2 sin^2(Delta/2), azimuth phi = 2 pi u'' - pi in the orthonormal frame
 * e1 = (g + x^2 a, b, -x), e2 = (b, g + y^2 a, -y), g = sign(z) (+1 at z = 0),
 * a = -1/(g + z), b = x y a (Duff et al., JCGT 2017, first vector times g),
 * S' = cos theta S + sin theta (cos phi e1 + sin phi e2); accept as for XY.
 * FP64 draws: block (site, t, MET<<24 | r): u = u53(w0,w1), test u53(w2,w3);
 * block (site, t, MET<<24 | 0x800000 | r): u'' = u53(w0,w1).  FP32: one block
 * (site, t, MET<<24 | r) per replica, u24(w0), u24(w1), u24(w2), and the
 * proposal renormalised.  Overrelaxation: S' = 2 (S.h) h / |h|^2 - S.  Spins
 * are stored as padded 4-vectors (16 B FP32, 32 B FP64), replica-major.  On
 * XYL_FP32_BATCHED, O(3) spins run in the resident shape only: one CTA per
 * group of replicas keeps three single-precision component arrays of every
 * site in shared memory (12 B a site and replica, within 220 KB), with the
 * plain engine's per-spin arithmetic, so both engines give bit-identical
 * spins from the same state.  Random fields on O(3) spins are 3-vectors
 * (xyl_graph_set_fields3), on every engine.
 */

/*
 * Resident shape of the batched engine.  One CTA owns a group of `group`
 * replicas of one sample and keeps their spins of every site in shared memory
 * for the whole launch ((n + 1) x group x 8 bytes, with the per-warp partial
 * sums, within 220 KB); the n_temps / group CTAs of a sample form one cluster
 * (at most 16), so every sample must have the same n_temps.  Colour phases
 * then touch no global memory but the CSR: rows of up to eight neighbours
 * (16-bit ids) and the site ids are staged beside the spins when they fit
 * (stage >= 0), else read from global memory, and longer rows (the 2N-bond
 * graphs) are read from the global CSR entry by entry.  Spins are bit-equal to the global-memory shape's
 * from the same state.  On input `cluster` is ignored for this shape; on output
 * (xyl_get_tuning, xyl_autotune) it holds the cluster size.  The library's
 * choice (resident = 0) is the resident shape when it fits with group >= 1,
 * else the global-memory shape.
 */

/*
 * xyl_plan_create -- lay out a batch of n_samples samples (each with its own
 * graph and temperature slots) for one engine.  Replica r of a sample starts at
 * slot r.  seed keys every spin/Metropolis/PT random stream.  tune may be NULL.
 * *workspace_bytes receives the device bytes xyl_bind needs.
 * Errors: XYL_EINVAL (empty batch, bad slot count, unknown engine, spin_dim
 * other than 0, 2 or 3, fields whose component count differs from the spins'
 * or, for O(3) spins on the batched engine, outside the resident shape).
 */
int xyl_plan_create(const xyl_sample *samples, int32_t n_samples, int32_t engine, uint64_t seed,
                    const xyl_tuning *tune, xyl_plan **out, size_t *workspace_bytes);

/*
 * xyl_bind -- attach a caller-owned device workspace (>= workspace_bytes,
 * 256-byte aligned) and upload graphs, tables and temperatures into it.  The
 * workspace must outlive the plan's use.  Synchronises `stream`.
 * Errors: XYL_ENOSPC, XYL_EINVAL (misaligned), XYL_ECUDA.
 */
int xyl_bind(xyl_plan *p, void *d_workspace, size_t bytes, void *stream);

/*
 * xyl_init_spins -- theta = 2 pi u - pi from the INIT stream of each (site,
 * replica, sample), stored as unit vectors; aligned != 0 sets every spin to
 * (1, 0) instead (O(3) spins: uniform on the sphere, see above).  Resets the sweep counter, the slot labels, the per-slot
 * accumulators and the status word.
 */
int xyl_init_spins(xyl_plan *p, int32_t aligned, void *stream);

/*
 * xyl_sweep -- n_sweeps Monte Carlo sweeps (App. B).  One sweep: the Metropolis
 * pass (XYL_OP_MET) runs the colour classes in turn, each site proposing
 * theta + Delta (2u - 1) and accepting iff dE <= 0 or u' < exp(-beta dE); the
 * overrelaxation pass (XYL_OP_OR) then reflects each spin about its local
 * field, s' = 2 (s.h) h / |h|^2 - s (unchanged when h = 0); the energy and the
 * Fourier/magnetisation sums of each replica are fused into the last pass.
 * XYL_OP_PT: swap attempts between slots (k, k+1), k = t mod 2, 4, ...,
 * accepted iff u < exp((beta_k - beta_k+1)(E_k - E_k+1)) in FP64.
 * XYL_OP_MEASURE: when (t+1) is a multiple of measure_every, add the Sec. III
 * observables of the replica at each slot to that slot's FP64 accumulators.
 * Must include XYL_OP_MET or XYL_OP_OR.  Errors: XYL_EINVAL, XYL_ESTATE,
 * XYL_ECUDA; a device wait that gives up sets the status word (see
 * xyl_read_status) and later calls return XYL_ETIMEOUT.
 */
int xyl_sweep(xyl_plan *p, int32_t n_sweeps, uint32_t ops, int32_t measure_every, void *stream);

/*
 * xyl_sweep_units -- XYL_FP32_BATCHED only: run xyl_sweep on the work units
 * [first_unit, first_unit + n_units) of the batch (a unit is one group of
 * replicas of one sample; units are numbered part by part, see
 * xyl_part_count, and sample by sample within a part).  All units of
 * a sample must be included for parallel tempering to proceed: a sample whose
 * groups are split across calls makes the in-kernel wait for the missing
 * groups give up after about a second, set the status word to XYL_ETIMEOUT
 * and return (the GPU context stays usable; xyl_init_spins clears it).  In
 * the resident shape a cluster is a whole sample, so the range must cover
 * whole samples (XYL_EINVAL otherwise).
 * Errors: XYL_EINVAL (wrong engine or range), XYL_ESTATE, XYL_ECUDA.
 */
int xyl_sweep_units(xyl_plan *p, int32_t first_unit, int32_t n_units, int32_t n_sweeps, uint32_t ops,
                    int32_t measure_every, void *stream);

/*
 * xyl_sweep_noalloc -- XYL_FP32_BATCHED only: the same sweeps as xyl_sweep
 * (same kernel, same results), for callers that cannot obtain device memory
 * while they run: code embedded in a host application that owns every
 * allocation, or that must not allocate once its memory budget is fixed.
 * It allocates nothing and needs no scratch from the caller: the kernel's
 * scratch (per-replica sums of the sweep and the per-sample barrier counters)
 * lives in one fixed array of 1 MiB that every GPU using the library holds
 * until the process exits.  Inputs and outputs stay in the plan's workspace.
 * The batch must fit that array: 256 B per temperature slot (rounded up to
 * a multiple of 256 B) plus 4 B per sample, i.e. 256 * slots + 4 * samples
 * <= 1048576 (at most 4095 slots; 31 samples x 128 slots fit, 32 x 128 do
 * not); larger batches get XYL_EINVAL.  The first call on a device looks up
 * the array's device address (with that device current), so make it before
 * any stream capture.  All calls share the one array, which keeps the last
 * call's contents; every launch clears what it needs first, so calls that
 * overlap on the GPU (different streams, plans or threads) race and must be
 * serialised by the caller.  Like xyl_sweep, the sweeps are cut into launches
 * at the FP64 recompute points (xyl_tuning.recompute_every), n_sweeps = 0
 * does nothing, and xyl_sweep and xyl_sweep_noalloc may be mixed freely on one
 * plan.  No graph is used.  Errors: XYL_EINVAL, XYL_ESTATE, XYL_ECUDA.  The
 * paper has no counterpart of this entry point.
 */
int xyl_sweep_noalloc(xyl_plan *p, int32_t n_sweeps, uint32_t ops, int32_t measure_every, void *stream);

/* Number of work units of a batched plan (0 for other engines). */
int32_t xyl_unit_count(const xyl_plan *p);

/* Work units one launch of a bound batched plan runs together (part 0's wave; 0 for other engines or before bind). */
int32_t xyl_wave_units(const xyl_plan *p);

/*
 * Work units of part 0 of a bound batched plan that are resident on the GPU at
 * once: the whole wave when its clusters wait on one another, else as many
 * clusters as fit (the hardware starts the others as those finish, each unit
 * running all of a launch's sweeps while resident).  Their spins are what a
 * launch keeps live at a time.  0 for other engines or before bind.
 */
int32_t xyl_live_units(const xyl_plan *p);

/*
 * Mixed sizes in one batch (App. B "Computational speed": the cost of a sweep
 * follows the graph's size and colour count, so each size wants its own
 * launch shape).  When the library chooses the shape (xyl_tuning resident,
 * group, cluster and block all 0) and the samples of a batched plan differ in
 * size, the plan runs one part per size, largest first, each with its own
 * launch shape (spins in shared memory where a replica group fits, else in
 * global memory); a caller-given shape applies to the whole batch as one part.
 * In one xyl_sweep the parts whose clusters wait on other clusters of their
 * sample (a cross-cluster barrier) run first, one at a time; the others run
 * side by side on forked streams (also inside the captured CUDA graph).
 * Results are those of any single shape: every shape performs the same
 * per-site arithmetic.  xyl_get_tuning reports part 0; xyl_autotune tunes
 * every part.
 */
int32_t xyl_part_count(const xyl_plan *p);

/* Launch shape of one part (0 <= part < xyl_part_count) and its number of samples (may be NULL). */
int xyl_get_part_tuning(const xyl_plan *p, int32_t part, xyl_tuning *out, int32_t *n_samples);

/*
 * xyl_set_part_tuning -- give one part of a batched plan a launch shape, e.g.
 * one an earlier xyl_autotune chose for a batch of the same sizes: resident
 * (1 or -1), group, cluster and block must be set, stage and waves as in
 * xyl_tuning.  On a bound plan the shape takes effect at once (synchronises
 * `stream`); the sampler state is untouched.  A shape that does not fit
 * leaves the part as it was.  Errors: XYL_EINVAL, XYL_ECUDA.
 */
int xyl_set_part_tuning(xyl_plan *p, int32_t part, const xyl_tuning *t, void *stream);

/*
 * xyl_autotune -- XYL_FP32_BATCHED only: time n_sweeps sweeps (ops,
 * measure_every as in xyl_sweep) for every launch shape (replicas per cluster
 * R_g, CTAs per cluster G, threads per CTA) that can be resident, keep the
 * fastest, and restore the sampler state (spins, labels, counters) exactly as
 * it was.  *best (may be NULL) receives the chosen shape.  Synchronises
 * `stream`.  Errors: XYL_EINVAL, XYL_ESTATE, XYL_ECUDA.
 */
int xyl_autotune(xyl_plan *p, int32_t n_sweeps, uint32_t ops, int32_t measure_every, xyl_tuning *best,
                 void *stream);

/* Current launch shape of a batched plan (block, cluster, group, stage filled in; part 0 of a mixed-size plan). */
int xyl_get_tuning(const xyl_plan *p, xyl_tuning *out);

/*
 * xyl_pt_swap -- one parallel-tempering step (App. B "Improved equilibrium
 * dynamics") at the current sweep index, from freshly recomputed FP64
 * energies; does not advance the sweep counter.
 */
int xyl_pt_swap(xyl_plan *p, void *stream);

/*
 * xyl_measure -- recompute every replica's energy, magnetisation and Fourier
 * sums in FP64 from the stored spins and add one measurement (Sec. III
 * observables) to each slot's accumulators.
 */
int xyl_measure(xyl_plan *p, void *stream);

/*
 * xyl_recompute -- FP64 recomputation of every replica's energy from its spins
 * and renormalisation |s| = 1; records the largest |E_fused - E_fp64| seen.
 */
int xyl_recompute(xyl_plan *p, void *stream);

/* Replace the Metropolis half-widths of one sample's slots (n_temps values). */
int xyl_set_delta(xyl_plan *p, int32_t sample, const double *delta, void *stream);

/* The current Metropolis half-widths of one sample's slots (n_temps values; host call). */
int xyl_get_delta(const xyl_plan *p, int32_t sample, double *delta);

/*
 * xyl_tune_delta -- warm-up that sets each slot's Metropolis half-width
 * Delta so that about `target` of its proposals are accepted, then freezes it
 * (the paper fixes no proposal, App. B; the half-width is tuned before any
 * measurement and stays fixed while measuring).  Runs rounds + 1 blocks of
 * n_sweeps sweeps with `ops` (XYL_OP_MET required; XYL_OP_MEASURE ignored).
 * After each of the first `rounds` blocks, Delta_k becomes Delta_k * f with
 * f = a_k / target clamped to [1/2, 2], a_k the block's acceptance at slot k,
 * and Delta_k kept in [1e-3, pi]; the last block only measures.  A slot
 * whose acceptance stays above target at Delta = pi (hot slots) keeps pi.
 * rate (may be NULL) receives each slot's acceptance in the last block,
 * slot-major over the batch.  The sweep counter advances; the accumulators
 * and counters are zeroed at the end.  Synchronises `stream`.
 * Errors: XYL_EINVAL, XYL_ESTATE, XYL_ECUDA.
 */
int xyl_tune_delta(xyl_plan *p, int32_t rounds, int32_t n_sweeps, uint32_t ops, double target, double *rate,
                   void *stream);

/*
 * xyl_read_observables -- per-slot accumulators, slot-major over the batch
 * (sample 0 slots, sample 1 slots, ...).  acc: [slots][XYL_ACC_COUNT];
 * met_acc/met_try: accepted / attempted Metropolis updates per slot; pt_acc /
 * pt_try: accepted / attempted swaps of pair (k, k+1) stored at slot k.  Any
 * pointer may be NULL.  Synchronises `stream`.
 */
int xyl_read_observables(xyl_plan *p, double *acc, uint64_t *met_acc, uint64_t *met_try, uint64_t *pt_acc,
                         uint64_t *pt_try, void *stream);

/* Zero the per-slot accumulators and counters (e.g. between bins). */
int xyl_reset_observables(xyl_plan *p, void *stream);

/* Energy of every replica after the last sweep / recompute (FP64), replica-major over the batch. */
int xyl_read_energies(xyl_plan *p, double *E, void *stream);

/* replica_at_slot[k] for every slot of the batch (slot-major). */
int xyl_read_labels(xyl_plan *p, int32_t *replica_at_slot, void *stream);

/* Spin vectors of one replica, original site order: sxy[d*i + k], k < d, d = 2 (XY) or 3 (O(3)), FP64. */
int xyl_read_spins(xyl_plan *p, int32_t sample, int32_t replica, double *sxy, void *stream);

/* Overwrite the spin vectors of one replica (original site order). */
int xyl_write_spins(xyl_plan *p, int32_t sample, int32_t replica, const double *sxy, void *stream);

/*
 * xyl_read_drift -- the largest |E_fused - E_fp64| over every replica seen
 * since xyl_init_spins (or the last reset): E_fused is the energy a sweep
 * summed in FP32 alongside its last pass, E_fp64 the energy recomputed in FP64
 * from the stored spins by the next FP64 recompute (xyl_recompute, the
 * periodic recompute of xyl_tuning.recompute_every, xyl_pt_swap,
 * xyl_measure).  It is the health signal of the FP32-update / FP64-observable
 * split (App. B "Memory management": single-precision spins, double-precision
 * observables); the paper reports no such figure.  xyl_write_spins does not
 * change it.  reset != 0 clears it after the read.  Synchronises `stream`.
 * Errors: XYL_EINVAL (NULL output), XYL_ESTATE, XYL_ECUDA.
 */
int xyl_read_drift(xyl_plan *p, double *max_drift, int32_t reset, void *stream);

/*
 * xyl_check_plan -- check, on the device, the colour-sorted CSR the sweeps
 * read, for every sample of the plan: each colour class is an independent
 * set (App. B "Graph coloring": the sites of one colour update at once only
 * because no link joins two of them), neighbour ids lie in [0, N) and differ
 * from the site, rows are ascending (no repeated link), and every link is in
 * both of its rows.  *violations receives the number of failed checks (0 for
 * a sound plan).  A debugging aid in place of memory checkers; it reads the
 * workspace only.  Synchronises `stream`.  Errors: XYL_EINVAL, XYL_ESTATE,
 * XYL_ECUDA.
 */
int xyl_check_plan(xyl_plan *p, int64_t *violations, void *stream);

/* Status word (0 = fine, else the first XYL_E* code recorded on the device: XYL_ETIMEOUT from a bounded
 * wait; in a debug build, XYL_EBOUNDS from a neighbour id, row length or colour-class bound out of range,
 * which the kernel skipped) and the sweep index of sample 0. */
int xyl_read_status(xyl_plan *p, int32_t *status, uint64_t *sweep_index, void *stream);

/* Bytes of a checkpoint: spins, labels, sweep counters, accumulators, counters. */
size_t xyl_state_bytes(const xyl_plan *p);

/* Copy the whole sampler state to / from a host buffer of xyl_state_bytes(). */
int xyl_export_state(xyl_plan *p, void *host, size_t bytes, void *stream);
int xyl_import_state(xyl_plan *p, const void *host, size_t bytes, void *stream);

/* ========================================================================= */
/* Random walks: spectral dimension of a graph                               */
/* ========================================================================= */

/*
 * xyl_walk_returns -- n_walkers independent simple random walks on a graph
 * given as a CSR in device memory, counting the walkers back on their
 * starting node after each step: P(tau) = returns[tau] / returns[0] decays as
 * tau^(-dbar/2), dbar the spectral dimension (Sec. "Spectral dimension",
 * Eq. (eqbard); App. A).  All pointers are device pointers owned by the
 * caller; nothing is allocated.
 *   row_ptr, col  CSR of n nodes and nnz neighbour entries (row_ptr[n] == nnz),
 *                 e.g. xyl_graph_export_csr copied to the device; node ids are
 *                 those of this CSR.
 *   start         n_walkers starting nodes.
 *   first_walker  id of walker 0: walker w draws from the stream of id
 *                 first_walker + w, so a large ensemble can be run in pieces.
 *   n_steps       steps per walker.
 *   seed          64-bit key of the walk streams.
 *   returns       n_steps + 1 counters, overwritten: returns[0] = walkers that
 *                 ran, returns[tau] = walkers on their start after tau steps.
 * Step tau of walker w takes word tau mod 4 of Philox block floor(tau/4) at
 * counter (w, floor(tau/4), 4<<24, 0): a node of degree k > 0 sends the walker
 * to neighbour floor(word * k / 2^32) of its CSR row; a node without
 * neighbours keeps it.  A start outside [0, n) leaves that walker out; a row
 * or neighbour outside the CSR stops that walker (no fault).  Asynchronous on
 * `stream`.  Errors: XYL_EINVAL (sizes, NULL pointers, walker ids beyond
 * 2^32), XYL_ECUDA.
 */
int xyl_walk_returns(const int32_t *row_ptr, const int32_t *col, int32_t n, int64_t nnz, const int32_t *start,
                     int64_t n_walkers, uint32_t first_walker, int32_t n_steps, uint64_t seed, uint64_t *returns,
                     void *stream);

/*
 * xyl_philox -- the library's random generator, Philox4x32-10 (Salmon, Moraes,
 * Dror & Shaw, SC'11: ten rounds, multipliers 0xD2511F53 / 0xCD9E8D57, key
 * increments 0x9E3779B9 / 0xBB67AE85), one block per (counter, key) pair, so
 * that the generator every stream draws from can be checked against other
 * implementations.  Device pointers owned by the caller: ctr 4n words
 * (16-byte aligned), key 2n words (8-byte aligned), out 4n words (16-byte
 * aligned).  Asynchronous on `stream`.  Errors: XYL_EINVAL (n < 0, NULL or
 * misaligned pointers), XYL_ECUDA.
 */
int xyl_philox(const uint32_t *ctr, const uint32_t *key, int64_t n, uint32_t *out, void *stream);

/* Number of kernel launches the last xyl_sweep call issued (graph nodes count). */
int64_t xyl_last_launch_count(const xyl_plan *p);

void xyl_plan_free(xyl_plan *p);

#ifdef __cplusplus
}
#endif

#endif /* XYL_H */
