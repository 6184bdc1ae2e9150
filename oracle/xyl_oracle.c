/*
 * xyl_oracle.c -- plain, sequential, FP64 reference sampler for the XY model on
 * dilute Levy graphs (Ibanez Berganza & Leuzzi, "Critical behavior of the XY
 * model in complex topologies").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file; only the test-suite, the package smoke check and the
 * benchmark's CPU-baseline leg do.  It shares no code, header or table with the
 * CUDA path: every routine below is written out here on its own.
 *
 * What it computes, in the order the method runs:
 *   philox()            Philox4x32-10 counter-based generator (Salmon, Moraes,
 *                       Dror & Shaw, SC'11), the random source of every step.
 *   disp_table_*()      Link-length law of the dilute Levy graph, Eq. (Levyi):
 *                       P(J_ij = 1) proportional to |r_i - r_j|^-rho, minimum
 *                       image distances on the periodic L x L lattice (Sec. II).
 *   orc_levy_graph()    Fixed-degree (every site exactly z links) sequential
 *                       pairing of unsaturated sites, each new link drawn with
 *                       the law above among the eligible partners.
 *   orc_levy_bonds()    The paper's own ensemble: exactly M bonds (M = 2N, mean
 *                       degree 4), each pair drawn with the same law, periodic
 *                       or free boundaries (Sec. II).
 *   orc_walk_returns()  Self-return counts of simple random walks, whose decay
 *                       gives the spectral dimension (App. A).
 *   orc_slo_color()     Smallest-last-ordering colouring (App. B, "Graph
 *                       coloring").
 *   orc_csr()           Colour-sorted CSR (App. B, "Memory management": sites of
 *                       one colour stored consecutively).
 *   orc_sincos_series() sin/cos of the Metropolis step by their Maclaurin series.
 *   orc_reflect()       The overrelaxation map (App. B, Creutz reflection).
 *   orc_sim_set_dim()   O(3) spins (three components), the first of the "other
 *                       continuous models" the method carries over to (App. B).
 *   orc_sim_*()         Monte Carlo sweeps of H = -sum_{i<j} J_ij S_i.S_j,
 *                       Eq. (HXY): single-spin Metropolis over the colour classes
 *                       in sequence (App. B), overrelaxation (App. B, "Improved
 *                       equilibrium dynamics"), parallel-tempering swaps every
 *                       sweep (same passage), and the observables of Sec. III
 *                       (energy, magnetisation m, |m|, m^2, m^4, and the
 *                       Fourier sum at k_min = 2 pi / L used by xi_2).
 *
 * Spins are FP64 unit vectors, the form in which Eq. (HXY) is written.  The
 * overrelaxation map is chaotic (rounding differences grow about tenfold per
 * sweep), so every arithmetic step of a sweep is fixed here -- operand order,
 * no contraction, the series for sin/cos -- and an implementation doing the
 * same steps reproduces the trajectory bit for bit.
 *
 * Readings of points the paper leaves open are listed with each routine.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_PI 3.14159265358979323846

/* ------------------------------------------------------------------------- */
/* Philox4x32-10 (Salmon et al., SC'11): 10 rounds of the 4x32 Philox S-box,
 * multipliers 0xD2511F53 / 0xCD9E8D57, key schedule Weyl increments
 * 0x9E3779B9 / 0xBB67AE85 applied between rounds.                            */
/* ------------------------------------------------------------------------- */
void orc_philox(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
        uint32_t n1 = (uint32_t)p1;
        uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
        uint32_t n3 = (uint32_t)p0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Random-stream purposes, stored in the top byte of counter word 2. */
enum { PURPOSE_GRAPH = 0, PURPOSE_INIT = 1, PURPOSE_MET = 2, PURPOSE_PT = 3 };

static void draw_block(uint32_t w0, uint32_t w1, uint32_t purpose, uint32_t sub,
                       uint32_t sample, const uint32_t key[2], uint32_t out[4])
{
    uint32_t ctr[4] = { w0, w1, (purpose << 24) | (sub & 0xFFFFFFu), sample };
    orc_philox(ctr, key, out);
}

/* 53-bit uniform in [0,1) from two words (hi word first). */
static double u53(uint32_t hi, uint32_t lo)
{
    uint64_t v = (((uint64_t)hi << 32) | (uint64_t)lo) >> 11;
    return (double)v * 0x1.0p-53;
}

/* 24-bit uniform in [0,1) from one word. */
static double u24(uint32_t x)
{
    return (double)(x >> 8) * 0x1.0p-24;
}

static uint64_t mulhi64(uint64_t a, uint64_t b)
{
    return (uint64_t)(((unsigned __int128)a * (unsigned __int128)b) >> 64);
}

/* ------------------------------------------------------------------------- */
/* Link-length law, Eq. (Levyi).                                              */
/*                                                                            */
/* Reading: the normalisation runs over partner SITES, so a distance r that   */
/* occurs g(r) times around a site carries total weight g(r) r^-rho; this is  */
/* the only reading under which the per-pair law P(J_ij) ~ |r_i-r_j|^-rho     */
/* holds.  Displacements (dx,dy) take dx,dy in {-L/2+1,...,L/2} (even L), so  */
/* every other site appears exactly once and r_max = (L/2) sqrt(2) as in      */
/* Sec. II.  Table order: the "near" displacements (dx^2+dy^2 <= 8) first,    */
/* then the rest, each group in raster order (dy outer, dx inner, ascending). */
/* Integer boundaries B_k = floor(2^64 * S_k / S), S_k the FP64 running sum   */
/* of the weights before entry k, make every later decision an integer one.   */
/* ------------------------------------------------------------------------- */
#define NEAR_R2 8

typedef struct {
    int L, n;          /* lattice size, number of displacements (L*L - 1) */
    int n_near;        /* entries [0, n_near) are the near group */
    int *dx, *dy;      /* displacement of entry k */
    uint64_t *B;       /* B[k] = lower boundary of entry k, B[0] = 0 */
    int *index_of;     /* raster cell (dy+L/2-1)*L + (dx+L/2-1) -> entry, -1 at origin */
} disp_table;

static void disp_table_free(disp_table *t)
{
    free(t->dx); free(t->dy); free(t->B); free(t->index_of);
}

static int disp_table_build(disp_table *t, int L, double rho)
{
    memset(t, 0, sizeof(*t));
    t->L = L;
    t->n = L * L - 1;
    t->dx = (int *)malloc(sizeof(int) * (size_t)t->n);
    t->dy = (int *)malloc(sizeof(int) * (size_t)t->n);
    t->B = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)t->n);
    t->index_of = (int *)malloc(sizeof(int) * (size_t)L * (size_t)L);
    if (!t->dx || !t->dy || !t->B || !t->index_of) { disp_table_free(t); return -1; }
    int half = L / 2, k = 0;
    for (int pass = 0; pass < 2; ++pass) {
        for (int dy = -half + 1; dy <= half; ++dy) {
            for (int dx = -half + 1; dx <= half; ++dx) {
                int r2 = dx * dx + dy * dy;
                if (r2 == 0) continue;
                int near = r2 <= NEAR_R2;
                if ((pass == 0) != near) continue;
                t->dx[k] = dx; t->dy[k] = dy;
                t->index_of[(dy + half - 1) * L + (dx + half - 1)] = k;
                ++k;
            }
        }
        if (pass == 0) t->n_near = k;
    }
    t->index_of[(half - 1) * L + (half - 1)] = -1;
    /* running FP64 sums of r^-rho in table order */
    double *S = (double *)malloc(sizeof(double) * (size_t)(t->n + 1));
    if (!S) { disp_table_free(t); return -1; }
    S[0] = 0.0;
    for (int m = 0; m < t->n; ++m) {
        double r2 = (double)(t->dx[m] * t->dx[m] + t->dy[m] * t->dy[m]);
        S[m + 1] = S[m] + pow(r2, -0.5 * rho);
    }
    const double two64 = 18446744073709551616.0;
    t->B[0] = 0;
    for (int m = 1; m < t->n; ++m) {
        double q = (S[m] / S[t->n]) * two64;
        t->B[m] = (q >= two64) ? UINT64_MAX : (uint64_t)q;
    }
    free(S);
    return 0;
}

/* integer weight of entry k: B[k+1] - B[k], with B[n] = 2^64 */
static uint64_t disp_weight(const disp_table *t, int k)
{
    uint64_t hi = (k + 1 < t->n) ? t->B[k + 1] : 0; /* 2^64 wraps to 0 */
    return hi - t->B[k];
}

/* entry whose interval [B_k, B_{k+1}) holds u, searched among [lo, n) */
static int disp_locate(const disp_table *t, uint64_t u, int lo)
{
    /* largest k in [lo, n) with B[k] <= u (B is non-decreasing, B[lo] <= u) */
    int a = lo, b = t->n - 1;
    while (a < b) {
        int mid = a + (b - a + 1) / 2;
        if (t->B[mid] <= u) a = mid; else b = mid - 1;
    }
    return a;
}

/* table entry of the displacement from site i to site j */
static int disp_between(const disp_table *t, int i, int j)
{
    int L = t->L, half = L / 2;
    int dx = (j % L) - (i % L), dy = (j / L) - (i / L);
    if (dx > half) dx -= L;
    if (dx <= -half) dx += L;
    if (dy > half) dy -= L;
    if (dy <= -half) dy += L;
    return t->index_of[(dy + half - 1) * L + (dx + half - 1)];
}

/* Exported for the link-law tests: the table in table order. */
int orc_disp_table(int L, double rho, int32_t *dx, int32_t *dy, uint64_t *B, int32_t *n_near)
{
    if (L < 4 || (L & 1)) return -1;
    disp_table t;
    if (disp_table_build(&t, L, rho)) return -1;
    for (int k = 0; k < t.n; ++k) { dx[k] = t.dx[k]; dy[k] = t.dy[k]; B[k] = t.B[k]; }
    *n_near = t.n_near;
    disp_table_free(&t);
    return 0;
}

/* Exported for the proposal-law test: n_draws table samples from one stream. */
int orc_disp_sample(int L, double rho, uint64_t seed, uint32_t sample, int64_t n_draws, int32_t *entry)
{
    if (L < 4 || (L & 1)) return -1;
    disp_table t;
    if (disp_table_build(&t, L, rho)) return -1;
    uint32_t key[2] = { (uint32_t)seed, (uint32_t)(seed >> 32) };
    for (int64_t d = 0; d < n_draws; d += 2) {
        uint32_t x[4];
        draw_block((uint32_t)(d >> 1), (uint32_t)((uint64_t)d >> 33), PURPOSE_GRAPH, 0, sample, key, x);
        entry[d] = disp_locate(&t, ((uint64_t)x[1] << 32) | x[0], 0);
        if (d + 1 < n_draws) entry[d + 1] = disp_locate(&t, ((uint64_t)x[3] << 32) | x[2], 0);
    }
    disp_table_free(&t);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Fixed-degree Levy graph by sequential pairing of unsaturated sites.        */
/*                                                                            */
/* Reading (the paper gives no construction procedure): while some site has  */
/* fewer than z links, pick a site i uniformly among the unsaturated ones,    */
/* then pick its partner j among the ELIGIBLE sites (j != i, fewer than z     */
/* links, not yet linked to i) with probability proportional to the integer   */
/* weight of the displacement i -> j; add the link.  If i has no eligible     */
/* partner the attempt is a dead end and the whole graph restarts with the    */
/* restart count in the random counter.  The draw protocol (identical in any  */
/* implementation that must reproduce the same graph):                        */
/*   * one stream of 64-bit draws U_0, U_1, ...: block b of Philox with       */
/*     counter (b_lo, b_hi, GRAPH<<24 | restart, sample) gives                */
/*     U_2b = w1:w0 and U_2b+1 = w3:w2;                                       */
/*   * i = unsat[mulhi(U, M)], M = number of unsaturated sites;               */
/*   * E = total weight of eligible near entries, F = total weight of far     */
/*     entries; up to 64 times: t = floor(U (E+F) / 2^64); t < E selects the  */
/*     near entry by cumulative weight (near order); otherwise the far entry  */
/*     whose interval holds B[n_near] + t - E is proposed and kept if         */
/*     eligible (a rejection costs one attempt);                              */
/*   * after 64 rejections: enumerate the unsaturated sites in list order,    */
/*     S = sum of eligible weights, t = mulhi(U, S), pick by cumulative       */
/*     weight; S == 0 is the dead end.                                        */
/* All three branches draw j with the same law: weight of i -> j over the     */
/* eligible sites.  The unsaturated list starts as 0..N-1; a site that        */
/* saturates is replaced by the last entry (i before j).                      */
/* ------------------------------------------------------------------------- */
#define PAIR_MAX_REJECT 64

typedef struct {
    uint32_t key[2];
    uint32_t sample, restart;
    uint64_t block;
    int half;
    uint32_t buf[4];
    uint64_t n_draws;
} u64_stream;

static uint64_t stream_next(u64_stream *s)
{
    uint64_t v;
    if (s->half == 0) {
        draw_block((uint32_t)s->block, (uint32_t)(s->block >> 32), PURPOSE_GRAPH, s->restart,
                   s->sample, s->key, s->buf);
        v = ((uint64_t)s->buf[1] << 32) | s->buf[0];
        s->half = 1;
    } else {
        v = ((uint64_t)s->buf[3] << 32) | s->buf[2];
        s->half = 0;
        s->block++;
    }
    s->n_draws++;
    return v;
}

typedef struct {
    int n, z;
    int *deg;
    int *adj;       /* n * z */
    int *unsat;     /* unsaturated sites */
    int *where;     /* position in unsat, -1 when saturated */
    int m;          /* number of unsaturated sites */
} pair_state;

static int adjacent(const pair_state *p, int i, int j)
{
    for (int a = 0; a < p->deg[i]; ++a)
        if (p->adj[(size_t)i * p->z + a] == j) return 1;
    return 0;
}

static int eligible(const pair_state *p, int i, int j)
{
    return j != i && p->deg[j] < p->z && !adjacent(p, i, j);
}

static void saturate_check(pair_state *p, int v)
{
    if (p->deg[v] < p->z) return;
    int pos = p->where[v], last = p->unsat[p->m - 1];
    p->unsat[pos] = last;
    p->where[last] = pos;
    p->where[v] = -1;
    p->m--;
}

static int site_shift(int L, int i, int dx, int dy)
{
    int x = ((i % L) + dx + L) % L, y = ((i / L) + dy + L) % L;
    return x + L * y;
}

/* Partner of site i, or -1 at a dead end. */
static int pick_partner(const disp_table *t, const pair_state *p, int i, u64_stream *s)
{
    int L = t->L;
    unsigned __int128 E = 0;
    for (int k = 0; k < t->n_near; ++k) {
        int j = site_shift(L, i, t->dx[k], t->dy[k]);
        if (eligible(p, i, j)) E += disp_weight(t, k);
    }
    unsigned __int128 F = (t->n_near < t->n) ? ((unsigned __int128)1 << 64) - t->B[t->n_near] : 0;
    if (E + F > 0) {
        for (int attempt = 0; attempt < PAIR_MAX_REJECT; ++attempt) {
            uint64_t u = stream_next(s);
            unsigned __int128 tt = ((unsigned __int128)u * (E + F)) >> 64;
            if (tt < E) {
                unsigned __int128 cum = 0;
                for (int k = 0; k < t->n_near; ++k) {
                    int j = site_shift(L, i, t->dx[k], t->dy[k]);
                    if (!eligible(p, i, j)) continue;
                    cum += disp_weight(t, k);
                    if (cum > tt) return j;
                }
                return -2; /* unreachable: cumulative weight covers tt */
            }
            uint64_t pos = t->B[t->n_near] + (uint64_t)(tt - E);
            int k = disp_locate(t, pos, t->n_near);
            int j = site_shift(L, i, t->dx[k], t->dy[k]);
            if (eligible(p, i, j)) return j;
        }
    }
    /* exhaustive fallback over the unsaturated list */
    unsigned __int128 S = 0;
    for (int a = 0; a < p->m; ++a) {
        int j = p->unsat[a];
        if (eligible(p, i, j)) S += disp_weight(t, disp_between(t, i, j));
    }
    if (S == 0) return -1;
    uint64_t u = stream_next(s);
    unsigned __int128 tt = ((unsigned __int128)u * S) >> 64;
    unsigned __int128 cum = 0;
    for (int a = 0; a < p->m; ++a) {
        int j = p->unsat[a];
        if (!eligible(p, i, j)) continue;
        cum += disp_weight(t, disp_between(t, i, j));
        if (cum > tt) return j;
    }
    return -2;
}

/*
 * Test hook for the partner law: from a given pairing state (deg, adjacency
 * rows of width z, unsaturated list), draw the partner of site i n_trials times
 * from one graph stream and count the outcomes (counts[n] = dead ends).
 */
int orc_pick_partner_counts(int L, int z, double rho, uint64_t seed, const int32_t *deg, const int32_t *adj,
                            const int32_t *unsat, int m, int i, int64_t n_trials, int64_t *counts)
{
    if (L < 4 || (L & 1)) return -1;
    disp_table t;
    if (disp_table_build(&t, L, rho)) return -1;
    int n = L * L;
    pair_state p;
    p.n = n; p.z = z; p.m = m;
    p.deg = (int *)malloc(sizeof(int) * (size_t)n);
    p.adj = (int *)malloc(sizeof(int) * (size_t)n * (size_t)z);
    p.unsat = (int *)malloc(sizeof(int) * (size_t)n);
    p.where = (int *)malloc(sizeof(int) * (size_t)n);
    for (int v = 0; v < n; ++v) { p.deg[v] = deg[v]; p.where[v] = -1; }
    for (int64_t a = 0; a < (int64_t)n * z; ++a) p.adj[a] = adj[a];
    for (int a = 0; a < m; ++a) { p.unsat[a] = unsat[a]; p.where[unsat[a]] = a; }
    u64_stream s;
    memset(&s, 0, sizeof(s));
    s.key[0] = (uint32_t)seed; s.key[1] = (uint32_t)(seed >> 32);
    for (int64_t k = 0; k < n_trials; ++k) {
        int j = pick_partner(&t, &p, i, &s);
        counts[j < 0 ? n : j]++;
    }
    free(p.deg); free(p.adj); free(p.unsat); free(p.where);
    disp_table_free(&t);
    return 0;
}

/*
 * Build one fixed-degree Levy graph.  Writes the N*z/2 links in the order they
 * were made (ei[e], ej[e]; ei is the site that chose).  Returns 0, or -1 on bad
 * arguments, -3 when max_restarts attempts all ended in a dead end.
 */
int orc_levy_graph(int L, int z, double rho, uint64_t seed, uint32_t sample, int max_restarts,
                   int32_t *ei, int32_t *ej, int32_t *restarts_out, uint64_t *draws_out)
{
    if (L < 4 || (L & 1) || z < 1 || z > L * L - 1 || ((int64_t)L * L * z) % 2) return -1;
    disp_table t;
    if (disp_table_build(&t, L, rho)) return -1;
    int n = L * L;
    pair_state p;
    p.n = n; p.z = z;
    p.deg = (int *)malloc(sizeof(int) * (size_t)n);
    p.adj = (int *)malloc(sizeof(int) * (size_t)n * (size_t)z);
    p.unsat = (int *)malloc(sizeof(int) * (size_t)n);
    p.where = (int *)malloc(sizeof(int) * (size_t)n);
    int rc = -3;
    uint64_t total_draws = 0;
    for (int restart = 0; restart < max_restarts; ++restart) {
        for (int v = 0; v < n; ++v) { p.deg[v] = 0; p.unsat[v] = v; p.where[v] = v; }
        p.m = n;
        u64_stream s;
        memset(&s, 0, sizeof(s));
        s.key[0] = (uint32_t)seed; s.key[1] = (uint32_t)(seed >> 32);
        s.sample = sample; s.restart = (uint32_t)restart;
        int64_t e = 0, dead = 0;
        while (p.m > 0) {
            int i = p.unsat[mulhi64(stream_next(&s), (uint64_t)p.m)];
            int j = pick_partner(&t, &p, i, &s);
            if (j < 0) { dead = 1; break; }
            p.adj[(size_t)i * z + p.deg[i]++] = j;
            p.adj[(size_t)j * z + p.deg[j]++] = i;
            ei[e] = i; ej[e] = j; ++e;
            saturate_check(&p, i);
            saturate_check(&p, j);
        }
        total_draws += s.n_draws;
        if (!dead) {
            if (restarts_out) *restarts_out = restart;
            rc = 0;
            break;
        }
    }
    if (draws_out) *draws_out = total_draws;
    free(p.deg); free(p.adj); free(p.unsat); free(p.where);
    disp_table_free(&t);
    return rc;
}

/* ------------------------------------------------------------------------- */
/* The paper's own ensemble (Sec. II, Eq. (Levyi)): exactly M bonds in all    */
/* (M = 2N gives the mean degree 4 the paper uses), each a pair of sites      */
/* drawn with probability proportional to |r_i - r_j|^-rho among all pairs of */
/* the lattice; degrees are free (Poisson with mean 4 at rho = 0, the         */
/* Erdos-Renyi limit).  Boundary conditions:                                  */
/*   PBC  minimum-image displacements, the table above (r_max = (L/2) sqrt2); */
/*   FBC  plain displacements |dx|, |dy| <= L-1 inside the L x L square       */
/*        (r_max = L sqrt 2), table in raster order (dy outer, dx inner)      */
/*        with the same integer boundaries.                                   */
/* Reading of the draw (the paper gives no procedure):                        */
/*   * attempt a uses Philox block a with counter                             */
/*     (a_lo, a_hi, GRAPH<<24 | BONDS_SUB | fbc, sample):                     */
/*     i = mulhi(w1:w0, N), displacement entry k = the one whose interval     */
/*     holds w3:w2, j = i + d_k (wrapped for PBC);                            */
/*   * an FBC partner outside the square, or a pair already bonded, is        */
/*     rejected and the next attempt drawn;                                   */
/*   * the first M accepted pairs are the bonds (ei = i, ej = j).             */
/* Each ordered pair (i, j) has one table entry and one choice of i, so an    */
/* accepted pair is drawn with probability proportional to r_ij^-rho among    */
/* the pairs not yet bonded; at rho = 0 the graph is uniform among graphs     */
/* with M edges.                                                              */
/* ------------------------------------------------------------------------- */
#define BONDS_SUB 0x400000u

static int fbc_table_build(disp_table *t, int L, double rho)
{
    memset(t, 0, sizeof(*t));
    t->L = L;
    t->n = (2 * L - 1) * (2 * L - 1) - 1;
    t->n_near = 0;
    t->dx = (int *)malloc(sizeof(int) * (size_t)t->n);
    t->dy = (int *)malloc(sizeof(int) * (size_t)t->n);
    t->B = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)t->n);
    double *S = (double *)malloc(sizeof(double) * (size_t)(t->n + 1));
    if (!t->dx || !t->dy || !t->B || !S) { free(S); disp_table_free(t); return -1; }
    int k = 0;
    for (int dy = -(L - 1); dy <= L - 1; ++dy)
        for (int dx = -(L - 1); dx <= L - 1; ++dx) {
            if (dx == 0 && dy == 0) continue;
            t->dx[k] = dx; t->dy[k] = dy; ++k;
        }
    S[0] = 0.0;
    for (int m = 0; m < t->n; ++m) {
        double r2 = (double)(t->dx[m] * t->dx[m] + t->dy[m] * t->dy[m]);
        S[m + 1] = S[m] + pow(r2, -0.5 * rho);
    }
    const double two64 = 18446744073709551616.0;
    t->B[0] = 0;
    for (int m = 1; m < t->n; ++m) {
        double q = (S[m] / S[t->n]) * two64;
        t->B[m] = (q >= two64) ? UINT64_MAX : (uint64_t)q;
    }
    free(S);
    return 0;
}

/* Exported for the FBC link-law tests: the table in table order. */
int orc_fbc_table(int L, double rho, int32_t *dx, int32_t *dy, uint64_t *B)
{
    if (L < 2) return -1;
    disp_table t;
    if (fbc_table_build(&t, L, rho)) return -1;
    for (int k = 0; k < t.n; ++k) { dx[k] = t.dx[k]; dy[k] = t.dy[k]; B[k] = t.B[k]; }
    disp_table_free(&t);
    return 0;
}

/*
 * Build one graph of the M-bond ensemble.  Writes the M bonds in the order
 * they were accepted.  Returns 0; -1 on bad arguments (PBC needs even L >= 4,
 * FBC L >= 2, 0 <= M <= N(N-1)/2); -3 when 64 M + 10^6 attempts did not give M
 * distinct bonds.  attempts_out (may be NULL) receives the attempts used.
 */
int orc_levy_bonds(int L, double rho, int64_t n_bonds, int fbc, uint64_t seed, uint32_t sample,
                   int32_t *ei, int32_t *ej, uint64_t *attempts_out)
{
    if (fbc ? L < 2 : (L < 4 || (L & 1))) return -1;
    const int64_t n = (int64_t)L * L;
    if (n_bonds < 0 || n_bonds > n * (n - 1) / 2) return -1;
    disp_table t;
    if (fbc ? fbc_table_build(&t, L, rho) : disp_table_build(&t, L, rho)) return -1;
    int *deg = (int *)calloc((size_t)n, sizeof(int));
    int *cap = (int *)calloc((size_t)n, sizeof(int));
    int **nbr = (int **)calloc((size_t)n, sizeof(int *));
    int rc = (deg && cap && nbr) ? -3 : -1;
    const uint32_t key[2] = { (uint32_t)seed, (uint32_t)(seed >> 32) };
    const uint64_t max_attempts = 64u * (uint64_t)n_bonds + 1000000u;
    int64_t e = 0;
    uint64_t a = 0;
    while (rc == -3 && a < max_attempts) {
        if (e == n_bonds) { rc = 0; break; }
        uint32_t x[4];
        draw_block((uint32_t)a, (uint32_t)(a >> 32), PURPOSE_GRAPH, BONDS_SUB | (fbc ? 1u : 0u), sample, key, x);
        ++a;
        int i = (int)mulhi64(((uint64_t)x[1] << 32) | x[0], (uint64_t)n);
        int k = disp_locate(&t, ((uint64_t)x[3] << 32) | x[2], 0);
        int j;
        if (fbc) {
            int xj = i % L + t.dx[k], yj = i / L + t.dy[k];
            if (xj < 0 || xj >= L || yj < 0 || yj >= L) continue;
            j = xj + L * yj;
        } else {
            j = site_shift(L, i, t.dx[k], t.dy[k]);
        }
        int bonded = 0;
        for (int b = 0; b < deg[i] && !bonded; ++b) bonded = nbr[i][b] == j;
        if (bonded) continue;
        int ends[2] = { i, j };
        for (int q = 0; q < 2 && rc == -3; ++q) {
            int v = ends[q];
            if (deg[v] == cap[v]) {
                int *grown = (int *)realloc(nbr[v], sizeof(int) * (size_t)(cap[v] ? 2 * cap[v] : 8));
                if (!grown) { rc = -1; break; }
                cap[v] = cap[v] ? 2 * cap[v] : 8;
                nbr[v] = grown;
            }
            nbr[v][deg[v]++] = ends[1 - q];
        }
        if (rc != -3) break;
        ei[e] = i; ej[e] = j; ++e;
    }
    if (rc == -3 && e == n_bonds) rc = 0;
    if (attempts_out) *attempts_out = a;
    if (nbr) for (int64_t v = 0; v < n; ++v) free(nbr[v]);
    free(nbr); free(cap); free(deg);
    disp_table_free(&t);
    return rc;
}

/* ------------------------------------------------------------------------- */
/* Random walks for the spectral dimension (Sec. "Spectral dimension",        */
/* App. A): the probability P(tau) that a simple random walker is back on its */
/* starting node after tau steps decays as tau^(-dbar/2).                     */
/* Reading (the paper gives the observable, not the walk's details): at each  */
/* step a walker on a node of degree k > 0 moves to one of its k neighbours   */
/* chosen uniformly (CSR row order); on a node without neighbours it stays.   */
/* Step tau (0-based) of walker w takes word tau mod 4 of Philox block        */
/* floor(tau / 4) with counter (w, floor(tau / 4), WALK<<24, 0): neighbour    */
/* index floor(word * k / 2^32).  returns[tau] counts the walkers on their    */
/* starting node after tau steps (returns[0] = number of walkers).            */
/* ------------------------------------------------------------------------- */
#define PURPOSE_WALK 4

int orc_walk_returns(int n, const int32_t *row_ptr, const int32_t *col, int64_t n_walkers, const int32_t *start,
                     int32_t n_steps, uint64_t seed, uint64_t *returns)
{
    if (n < 1 || n_walkers < 0 || n_steps < 0 || n_walkers > 0xFFFFFFFFll) return -1;
    for (int64_t w = 0; w < n_walkers; ++w)
        if (start[w] < 0 || start[w] >= n) return -1;
    const uint32_t key[2] = { (uint32_t)seed, (uint32_t)(seed >> 32) };
    for (int32_t t = 0; t <= n_steps; ++t) returns[t] = 0;
    returns[0] = (uint64_t)n_walkers;
    for (int64_t w = 0; w < n_walkers; ++w) {
        int v = start[w];
        uint32_t x[4] = { 0, 0, 0, 0 };
        for (int32_t t = 0; t < n_steps; ++t) {
            if (t % 4 == 0) draw_block((uint32_t)w, (uint32_t)(t / 4), PURPOSE_WALK, 0, 0, key, x);
            const int k = row_ptr[v + 1] - row_ptr[v];
            if (k > 0) v = col[row_ptr[v] + (int)(((uint64_t)x[t % 4] * (uint64_t)k) >> 32)];
            if (v == start[w]) returns[t + 1]++;
        }
    }
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Smallest-last-ordering colouring (App. B "Graph coloring"; Matula & Beck). */
/* Reading of the unpublished variant: repeatedly remove a vertex of minimum  */
/* degree in the remaining graph (ties: smallest id), then colour vertices in */
/* reverse removal order with the smallest colour no coloured neighbour has.  */
/* A binary heap of (degree, id) with stale entries skipped does the removal. */
/* ------------------------------------------------------------------------- */
typedef struct { int deg, id; } heap_item;

static int heap_less(heap_item a, heap_item b)
{
    return a.deg < b.deg || (a.deg == b.deg && a.id < b.id);
}

static void heap_push(heap_item *h, int64_t *size, heap_item v)
{
    int64_t k = (*size)++;
    h[k] = v;
    while (k > 0) {
        int64_t up = (k - 1) / 2;
        if (!heap_less(h[k], h[up])) break;
        heap_item tmp = h[k]; h[k] = h[up]; h[up] = tmp;
        k = up;
    }
}

static heap_item heap_pop(heap_item *h, int64_t *size)
{
    heap_item top = h[0];
    h[0] = h[--(*size)];
    int64_t k = 0;
    for (;;) {
        int64_t l = 2 * k + 1, r = l + 1, best = k;
        if (l < *size && heap_less(h[l], h[best])) best = l;
        if (r < *size && heap_less(h[r], h[best])) best = r;
        if (best == k) break;
        heap_item tmp = h[k]; h[k] = h[best]; h[best] = tmp;
        k = best;
    }
    return top;
}

/* adjacency (any order) from an edge list */
static int build_adjacency(int n, int64_t ne, const int32_t *ei, const int32_t *ej, int **ptr_out, int **nbr_out)
{
    int *ptr = (int *)calloc((size_t)n + 1, sizeof(int));
    int *nbr = (int *)malloc(sizeof(int) * (size_t)(2 * ne + 1));
    int *fill = (int *)calloc((size_t)n, sizeof(int));
    if (!ptr || !nbr || !fill) { free(ptr); free(nbr); free(fill); return -1; }
    for (int64_t e = 0; e < ne; ++e) { ptr[ei[e] + 1]++; ptr[ej[e] + 1]++; }
    for (int v = 0; v < n; ++v) ptr[v + 1] += ptr[v];
    for (int64_t e = 0; e < ne; ++e) {
        nbr[ptr[ei[e]] + fill[ei[e]]++] = ej[e];
        nbr[ptr[ej[e]] + fill[ej[e]]++] = ei[e];
    }
    free(fill);
    *ptr_out = ptr; *nbr_out = nbr;
    return 0;
}

int orc_slo_color(int n, int64_t ne, const int32_t *ei, const int32_t *ej, int32_t *color)
{
    int *ptr, *nbr;
    if (build_adjacency(n, ne, ei, ej, &ptr, &nbr)) return -1;
    int *deg = (int *)malloc(sizeof(int) * (size_t)n);
    char *gone = (char *)calloc((size_t)n, 1);
    int *order = (int *)malloc(sizeof(int) * (size_t)n);
    heap_item *h = (heap_item *)malloc(sizeof(heap_item) * (size_t)(n + 2 * ne + 1));
    int64_t hs = 0;
    for (int v = 0; v < n; ++v) {
        deg[v] = ptr[v + 1] - ptr[v];
        heap_item it = { deg[v], v };
        heap_push(h, &hs, it);
    }
    int removed = 0;
    while (removed < n) {
        heap_item it = heap_pop(h, &hs);
        if (gone[it.id] || it.deg != deg[it.id]) continue;
        int v = it.id;
        gone[v] = 1;
        order[removed++] = v;
        for (int a = ptr[v]; a < ptr[v + 1]; ++a) {
            int u = nbr[a];
            if (gone[u]) continue;
            deg[u]--;
            heap_item nu = { deg[u], u };
            heap_push(h, &hs, nu);
        }
    }
    for (int v = 0; v < n; ++v) color[v] = -1;
    int n_colors = 0;
    char *used = (char *)calloc((size_t)n + 2, 1);
    for (int k = n - 1; k >= 0; --k) {
        int v = order[k];
        for (int a = ptr[v]; a < ptr[v + 1]; ++a)
            if (color[nbr[a]] >= 0) used[color[nbr[a]]] = 1;
        int c = 0;
        while (used[c]) ++c;
        color[v] = c;
        if (c + 1 > n_colors) n_colors = c + 1;
        for (int a = ptr[v]; a < ptr[v + 1]; ++a)
            if (color[nbr[a]] >= 0) used[color[nbr[a]]] = 0;
    }
    free(used); free(h); free(order); free(gone); free(deg); free(ptr); free(nbr);
    return n_colors;
}

/* ------------------------------------------------------------------------- */
/* Colour-sorted CSR (App. B "Memory management").  New id = rank of the site */
/* by (colour, original id); perm[new] = original id; rows list neighbour new */
/* ids ascending; color_ptr[c] = first new id of colour c.                    */
/* ------------------------------------------------------------------------- */
static int cmp_int(const void *a, const void *b)
{
    int x = *(const int *)a, y = *(const int *)b;
    return (x > y) - (x < y);
}

int orc_csr(int n, int64_t ne, const int32_t *ei, const int32_t *ej, const int32_t *color, int n_colors,
            int32_t *perm, int32_t *row_ptr, int32_t *col, int32_t *color_ptr)
{
    int *ptr, *nbr;
    if (build_adjacency(n, ne, ei, ej, &ptr, &nbr)) return -1;
    int *inv = (int *)malloc(sizeof(int) * (size_t)n);
    int k = 0;
    for (int c = 0; c < n_colors; ++c) {
        color_ptr[c] = k;
        for (int v = 0; v < n; ++v)
            if (color[v] == c) { perm[k] = v; inv[v] = k; ++k; }
    }
    color_ptr[n_colors] = k;
    row_ptr[0] = 0;
    for (int a = 0; a < n; ++a) {
        int v = perm[a], d = ptr[v + 1] - ptr[v];
        for (int b = 0; b < d; ++b) col[row_ptr[a] + b] = inv[nbr[ptr[v] + b]];
        qsort(col + row_ptr[a], (size_t)d, sizeof(int32_t), cmp_int);
        row_ptr[a + 1] = row_ptr[a] + d;
    }
    free(inv); free(ptr); free(nbr);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* sin and cos of |x| <= pi (about) by their Maclaurin series:                */
/*   sin x = x sum_k (-1)^k x^2k / (2k+1)!,  k = 0..14                        */
/*   cos x =   sum_k (-1)^k x^2k / (2k)!,    k = 0..15                        */
/* coefficients by the factorial recurrence a_k = a_{k-1} / (n (n+1)), Horner */
/* in y = x^2 with IEEE fused multiply-add.  Truncation < 3e-17 at |x| = pi;  */
/* pinned against libm to 2e-15 absolute.  Every rounding step is fixed, so   */
/* any implementation of these steps gives the same bits.                     */
/* ------------------------------------------------------------------------- */
#define SIN_TERMS 15
#define COS_TERMS 16
static double sin_coef[SIN_TERMS], cos_coef[COS_TERMS];
static int series_ready = 0;

static void series_init(void)
{
    if (series_ready) return;
    double a = 1.0;
    sin_coef[0] = 1.0;
    for (int k = 1; k < SIN_TERMS; ++k) {
        a = a / (double)((2 * k) * (2 * k + 1));
        sin_coef[k] = (k & 1) ? -a : a;
    }
    a = 1.0;
    cos_coef[0] = 1.0;
    for (int k = 1; k < COS_TERMS; ++k) {
        a = a / (double)((2 * k - 1) * (2 * k));
        cos_coef[k] = (k & 1) ? -a : a;
    }
    series_ready = 1;
}

void orc_sincos_series(double x, double *sn, double *cs)
{
    series_init();
    const double y = x * x;
    double p = sin_coef[SIN_TERMS - 1];
    for (int k = SIN_TERMS - 2; k >= 0; --k) p = fma(p, y, sin_coef[k]);
    double q = cos_coef[COS_TERMS - 1];
    for (int k = COS_TERMS - 2; k >= 0; --k) q = fma(q, y, cos_coef[k]);
    *sn = x * p;
    *cs = q;
}

/* ------------------------------------------------------------------------- */
/* Monte Carlo sampler.                                                       */
/*                                                                            */
/* Spins are FP64 unit vectors S_i = (x_i, y_i), as in Eq. (HXY),             */
/* H = -sum_{i<j} J_ij S_i . S_j.                                             */
/*                                                                            */
/* Sweep t (App. B; readings where the paper is silent):                      */
/*   1. Metropolis pass: colours c = 0..Q-1 in turn; within a colour the      */
/*      sites are mutually unlinked, so the order inside it does not matter   */
/*      (ascending id here).  The local field h = sum_j S_j is summed over    */
/*      the neighbours in ascending colour-sorted id.  Proposal: S rotated by */
/*      delta = Delta (2u - 1), Delta per temperature slot:                   */
/*        x' = c x - s y,  y' = s x + c y   (c, s = cos, sin of delta);       */
/*      dE = -((x' - x) h_x + (y' - y) h_y); accept iff dE <= 0 or            */
/*      u' < exp(-beta dE).                                                   */
/*   2. Overrelaxation pass, same colour order: reflection about the local    */
/*      field, k = 2 (x h_x + y h_y) / (h_x^2 + h_y^2), S' = k h - S; the spin */
/*      is left as it is when h = 0.  One Metropolis and one OR pass a sweep. */
/*   3. Parallel tempering after the sweep: pairs of slots (k, k+1) with      */
/*      k = t mod 2, 4, ...; accept iff u < exp((beta_k - beta_{k+1})         */
/*      (E_k - E_{k+1})) where E_k is the energy of the replica at slot k;    */
/*      an accepted swap exchanges which replica sits at the two slots.       */
/*   4. Measurement when (t+1) is a multiple of measure_every, per slot.      */
/* Every expression is evaluated as written (no contraction): products, then  */
/* sums, left to right.                                                       */
/* Random draws: Metropolis of site i (original id), sweep t, replica r:      */
/* Philox counter (i, t, MET<<24 | r, sample); 53-bit mode uses u53(w0,w1)    */
/* for the step and u53(w2,w3) for the test.  24-bit mode: counter            */
/* (i, t, MET<<24 | r/2, sample) serves replicas 2p and 2p+1, the even one    */
/* taking u24(w0), u24(w1) and the odd one u24(w2), u24(w3).                  */
/* Initial angle theta = 2 pi u - pi from counter (i, 0, INIT<<24 | r,        */
/* sample), S = (cos theta, sin theta) by the series above.  PT pair k at     */
/* sweep t: counter (k, t, PT<<24, sample), u53(w0,w1).                       */
/* ------------------------------------------------------------------------- */
enum { OP_MET = 1u, OP_OR = 2u, OP_PT = 4u, OP_MEASURE = 8u };

/* One near-tie decision: replica (or -1 for PT), original site id (PT: pair k),
 * sweep index and the outcome the test took. */
typedef struct { int32_t rep, site; int64_t sweep; int32_t accepted; } orc_tie;
enum { ACC_N, ACC_E, ACC_E2, ACC_ABSM, ACC_MX, ACC_MY, ACC_M2, ACC_M4, ACC_CHIK, ACC_MZ, ACC_COUNT };

typedef struct {
    int n, R, L, Q;
    int *ptr, *nbr;           /* neighbours of each original id, ascending colour-sorted id */
    int *cls_ptr, *cls;       /* colour classes, ascending id inside a class */
    int64_t n_bonds;
    int *bi, *bj;             /* bond list */
    double *cx, *sx, *cy, *sy;/* Fourier phases cos/sin(2 pi x/L), (2 pi y/L) */
    double *beta, *delta;     /* per slot */
    uint32_t key[2], sample;
    int u24_mode;
    double *vx, *vy;          /* spin vectors [R][n] */
    int *slot_of, *rep_at;
    uint64_t t;
    double *E;                /* per replica energy after the last sweep */
    double *acc;              /* [R][ACC_COUNT] per slot */
    uint64_t *met_acc, *met_try, *pt_acc, *pt_try;
    double tie_eps;
    int64_t *first_tie;       /* per replica: first sweep with a near-tie Metropolis test */
    int64_t *n_ties;          /* per replica: near-tie Metropolis tests since the last clear */
    int64_t first_pt_tie;
    double min_margin;        /* smallest Metropolis margin seen */
    double *jb;               /* coupling of each bond, or NULL (all J = 1) */
    double *jn;               /* coupling of each neighbour entry (aligned with nbr), or NULL */
    double *hx, *hy;          /* field on each site, or NULL */
    double *hz;               /* third field component (O(3) fields), or NULL */
    int dim;                  /* spin components: 2 (XY) or 3 (O(3)) */
    double *vz;               /* third spin component [R][n] (zero for XY) */
    /* checking aids (none changes a decision unless a test sets it):          */
    orc_tie *tie_log;         /* near-tie Metropolis tests since the last clear */
    int64_t tie_len, tie_cap;
    orc_tie *pt_log;          /* near-tie PT tests since the last clear (site = pair k) */
    int64_t pt_len, pt_cap;
    int8_t *forced;           /* [R][n] Metropolis outcome to take instead of the test's (-1: none), or NULL */
    int8_t *pt_forced;        /* [R] PT outcome of pair k to take instead of the test's (-1: none), or NULL */
    uint8_t *active;          /* [R] replicas the sweeps update, or NULL (all) */
} orc_sim;

void orc_sim_free(orc_sim *s)
{
    if (!s) return;
    free(s->ptr); free(s->nbr); free(s->cls_ptr); free(s->cls); free(s->bi); free(s->bj);
    free(s->cx); free(s->sx); free(s->cy); free(s->sy); free(s->beta); free(s->delta);
    free(s->vx); free(s->vy); free(s->slot_of); free(s->rep_at); free(s->E); free(s->acc);
    free(s->met_acc); free(s->met_try); free(s->pt_acc); free(s->pt_try); free(s->first_tie); free(s->n_ties);
    free(s->jb); free(s->jn); free(s->hx); free(s->hy); free(s->hz); free(s->vz);
    free(s->tie_log); free(s->pt_log); free(s->forced); free(s->pt_forced); free(s->active);
    free(s);
}

static const int *g_rank_for_sort;
static int cmp_by_rank(const void *a, const void *b)
{
    int x = g_rank_for_sort[*(const int *)a], y = g_rank_for_sort[*(const int *)b];
    return (x > y) - (x < y);
}

/* xy: 2n lattice coordinates (x, y) or NULL (then x = id, y = 0, period L = n). */
orc_sim *orc_sim_new(int n, int64_t ne, const int32_t *ei, const int32_t *ej, const int32_t *color,
                     const int32_t *xy, int L, int R, const double *beta, const double *delta,
                     uint64_t seed, uint32_t sample, int u24_mode)
{
    series_init();
    orc_sim *s = (orc_sim *)calloc(1, sizeof(orc_sim));
    if (!s) return NULL;
    s->n = n; s->R = R; s->u24_mode = u24_mode;
    s->key[0] = (uint32_t)seed; s->key[1] = (uint32_t)(seed >> 32); s->sample = sample;
    if (build_adjacency(n, ne, ei, ej, &s->ptr, &s->nbr)) { orc_sim_free(s); return NULL; }
    int Q = 0;
    for (int v = 0; v < n; ++v) if (color[v] + 1 > Q) Q = color[v] + 1;
    s->Q = Q;
    s->cls_ptr = (int *)calloc((size_t)Q + 1, sizeof(int));
    s->cls = (int *)malloc(sizeof(int) * (size_t)n);
    int k = 0;
    for (int c = 0; c < Q; ++c) {
        s->cls_ptr[c] = k;
        for (int v = 0; v < n; ++v) if (color[v] == c) s->cls[k++] = v;
    }
    s->cls_ptr[Q] = k;
    /* colour-sorted id of each site = its position in the class list; order each
     * neighbour list by it */
    int *rank = (int *)malloc(sizeof(int) * (size_t)n);
    for (int a = 0; a < n; ++a) rank[s->cls[a]] = a;
    g_rank_for_sort = rank;
    for (int v = 0; v < n; ++v)
        qsort(s->nbr + s->ptr[v], (size_t)(s->ptr[v + 1] - s->ptr[v]), sizeof(int), cmp_by_rank);
    free(rank);
    s->n_bonds = ne;
    s->bi = (int *)malloc(sizeof(int) * (size_t)(ne + 1));
    s->bj = (int *)malloc(sizeof(int) * (size_t)(ne + 1));
    for (int64_t e = 0; e < ne; ++e) { s->bi[e] = ei[e]; s->bj[e] = ej[e]; }
    s->L = xy ? L : n;
    s->cx = (double *)malloc(sizeof(double) * (size_t)n);
    s->sx = (double *)malloc(sizeof(double) * (size_t)n);
    s->cy = (double *)malloc(sizeof(double) * (size_t)n);
    s->sy = (double *)malloc(sizeof(double) * (size_t)n);
    for (int v = 0; v < n; ++v) {
        int x = xy ? xy[2 * v] : v, y = xy ? xy[2 * v + 1] : 0;
        double ax = 2.0 * ORC_PI * (double)x / (double)s->L;
        double ay = 2.0 * ORC_PI * (double)y / (double)s->L;
        s->cx[v] = cos(ax); s->sx[v] = sin(ax);
        s->cy[v] = cos(ay); s->sy[v] = sin(ay);
    }
    s->beta = (double *)malloc(sizeof(double) * (size_t)R);
    s->delta = (double *)malloc(sizeof(double) * (size_t)R);
    for (int r = 0; r < R; ++r) { s->beta[r] = beta[r]; s->delta[r] = delta[r]; }
    s->vx = (double *)calloc((size_t)R * (size_t)n, sizeof(double));
    s->vy = (double *)calloc((size_t)R * (size_t)n, sizeof(double));
    s->vz = (double *)calloc((size_t)R * (size_t)n, sizeof(double));
    s->dim = 2;
    s->slot_of = (int *)malloc(sizeof(int) * (size_t)R);
    s->rep_at = (int *)malloc(sizeof(int) * (size_t)R);
    s->E = (double *)calloc((size_t)R, sizeof(double));
    s->acc = (double *)calloc((size_t)R * ACC_COUNT, sizeof(double));
    s->met_acc = (uint64_t *)calloc((size_t)R, sizeof(uint64_t));
    s->met_try = (uint64_t *)calloc((size_t)R, sizeof(uint64_t));
    s->pt_acc = (uint64_t *)calloc((size_t)R, sizeof(uint64_t));
    s->pt_try = (uint64_t *)calloc((size_t)R, sizeof(uint64_t));
    s->first_tie = (int64_t *)malloc(sizeof(int64_t) * (size_t)R);
    s->n_ties = (int64_t *)calloc((size_t)R, sizeof(int64_t));
    s->tie_eps = 0.0;
    for (int r = 0; r < R; ++r) { s->slot_of[r] = r; s->rep_at[r] = r; s->first_tie[r] = -1; s->vx[(size_t)r * n] = 1.0; }
    s->first_pt_tie = -1;
    s->min_margin = INFINITY;
    return s;
}

void orc_sim_set_delta(orc_sim *s, const double *delta)
{
    for (int k = 0; k < s->R; ++k) s->delta[k] = delta[k];
}

void orc_sim_set_tie_eps(orc_sim *s, double eps) { s->tie_eps = eps; }

static double energy_of(const orc_sim *s, int r)
{
    const double *x = s->vx + (size_t)r * s->n, *y = s->vy + (size_t)r * s->n;
    double E = 0.0;
    if (s->dim == 3) {
        const double *z = s->vz + (size_t)r * s->n;
        for (int64_t e = 0; e < s->n_bonds; ++e) {
            int i = s->bi[e], j = s->bj[e];
            double d = x[i] * x[j] + y[i] * y[j] + z[i] * z[j];
            E -= s->jb ? s->jb[e] * d : d;
        }
        if (s->hz)
            for (int v = 0; v < s->n; ++v) E -= s->hx[v] * x[v] + s->hy[v] * y[v] + s->hz[v] * z[v];
        return E;
    }
    for (int64_t e = 0; e < s->n_bonds; ++e) {
        int i = s->bi[e], j = s->bj[e];
        if (s->jb) E -= s->jb[e] * (x[i] * x[j] + y[i] * y[j]);
        else E -= x[i] * x[j] + y[i] * y[j];
    }
    if (s->hx)
        for (int v = 0; v < s->n; ++v) E -= s->hx[v] * x[v] + s->hy[v] * y[v];
    return E;
}

static void refresh_energies(orc_sim *s)
{
    for (int r = 0; r < s->R; ++r) s->E[r] = energy_of(s, r);
}

/* aligned != 0: every spin (1, 0); else the INIT draws.  Resets the sweep count,
 * the slot labels and every accumulator. */
static void init_o3(orc_sim *s, int aligned);

void orc_sim_init(orc_sim *s, int aligned)
{
    if (s->dim == 3) init_o3(s, aligned);
    for (int r = 0; r < s->R && s->dim == 2; ++r) {
        for (int v = 0; v < s->n; ++v) {
            double sn = 0.0, cs = 1.0;
            if (!aligned) {
                uint32_t x[4];
                draw_block((uint32_t)v, 0, PURPOSE_INIT, (uint32_t)r, s->sample, s->key, x);
                double u = s->u24_mode ? u24(x[0]) : u53(x[0], x[1]);
                double th = 2.0 * ORC_PI * u - ORC_PI;
                orc_sincos_series(th, &sn, &cs);
            }
            s->vx[(size_t)r * s->n + v] = cs;
            s->vy[(size_t)r * s->n + v] = sn;
        }
    }
    for (int r = 0; r < s->R; ++r) {
        s->slot_of[r] = r; s->rep_at[r] = r; s->first_tie[r] = -1; s->n_ties[r] = 0;
    }
    s->t = 0;
    s->first_pt_tie = -1;
    s->tie_len = 0;
    s->pt_len = 0;
    s->min_margin = INFINITY;
    memset(s->acc, 0, sizeof(double) * (size_t)s->R * ACC_COUNT);
    memset(s->met_acc, 0, sizeof(uint64_t) * (size_t)s->R);
    memset(s->met_try, 0, sizeof(uint64_t) * (size_t)s->R);
    memset(s->pt_acc, 0, sizeof(uint64_t) * (size_t)s->R);
    memset(s->pt_try, 0, sizeof(uint64_t) * (size_t)s->R);
    refresh_energies(s);
}

static void log_tie(orc_tie **log, int64_t *len, int64_t *cap, int r, int site, int64_t t, int accepted)
{
    if (*len == *cap) {
        int64_t nc = *cap ? 2 * *cap : 64;
        orc_tie *grown = (orc_tie *)realloc(*log, sizeof(orc_tie) * (size_t)nc);
        if (!grown) return;  /* the count of n_ties still records it */
        *log = grown;
        *cap = nc;
    }
    orc_tie e = { r, site, t, accepted };
    (*log)[(*len)++] = e;
}

/* margin: distance of the test from flipping (|u - exp(-beta dE)|, or |dE|
 * near dE = 0); a test closer than tie_eps is counted and logged with the
 * outcome the test took. */
static void note_tie(orc_sim *s, int r, int v, double margin, int accepted)
{
    if (margin < s->min_margin) s->min_margin = margin;
    if (margin < s->tie_eps) {
        s->n_ties[r]++;
        if (s->first_tie[r] < 0) s->first_tie[r] = (int64_t)s->t;
        log_tie(&s->tie_log, &s->tie_len, &s->tie_cap, r, v, (int64_t)s->t, accepted);
    }
}

/* the outcome a test set for (r, v), else the test's own */
static int forced_outcome(const orc_sim *s, int r, int v, int accept)
{
    if (s->forced) {
        const int8_t f = s->forced[(size_t)r * s->n + v];
        if (f >= 0) return f;
    }
    return accept;
}

static void local_field(const orc_sim *s, const double *x, const double *y, int v, double *hx, double *hy)
{
    double ax = 0.0, ay = 0.0;
    if (s->jn) {
        for (int a = s->ptr[v]; a < s->ptr[v + 1]; ++a) {
            ax += s->jn[a] * x[s->nbr[a]];
            ay += s->jn[a] * y[s->nbr[a]];
        }
    } else {
        for (int a = s->ptr[v]; a < s->ptr[v + 1]; ++a) {
            ax += x[s->nbr[a]];
            ay += y[s->nbr[a]];
        }
    }
    if (s->hx) {
        /* the site's own field, added after the neighbours */
        ax += s->hx[v];
        ay += s->hy[v];
    }
    *hx = ax; *hy = ay;
}

/*
 * Random fields (the paper's "random fields" variant, App. B): H gains
 * -sum_i h_i . S_i with one field vector per site (original ids, hxy[2i],
 * hxy[2i+1]); the local field becomes sum_j J_ij S_j + h_i and the energy
 * includes the field term.  NULL removes the fields.  Recomputes the energies.
 */
int orc_sim_set_fields(orc_sim *s, const double *hxy)
{
    if (hxy && s->dim != 2) return -2;  /* 2-vectors: XY spins (orc_sim_set_fields3 for O(3)) */
    free(s->hx); free(s->hy); free(s->hz);
    s->hx = s->hy = s->hz = NULL;
    if (hxy) {
        s->hx = (double *)malloc(sizeof(double) * (size_t)s->n);
        s->hy = (double *)malloc(sizeof(double) * (size_t)s->n);
        if (!s->hx || !s->hy) return -1;
        for (int v = 0; v < s->n; ++v) { s->hx[v] = hxy[2 * v]; s->hy[v] = hxy[2 * v + 1]; }
    }
    refresh_energies(s);
    return 0;
}

/*
 * Random fields on O(3) spins: one 3-vector per site (original ids, hxyz[3i],
 * hxyz[3i+1], hxyz[3i+2]); H gains -sum_i h_i . S_i as for XY, the local
 * field becomes sum_j J_ij S_j + h_i (the field added after the neighbours)
 * and the energy includes the field term.  Needs dim 3; NULL removes the
 * fields.  Recomputes the energies.
 */
int orc_sim_set_fields3(orc_sim *s, const double *hxyz)
{
    if (hxyz && s->dim != 3) return -2;
    free(s->hx); free(s->hy); free(s->hz);
    s->hx = s->hy = s->hz = NULL;
    if (hxyz) {
        s->hx = (double *)malloc(sizeof(double) * (size_t)s->n);
        s->hy = (double *)malloc(sizeof(double) * (size_t)s->n);
        s->hz = (double *)malloc(sizeof(double) * (size_t)s->n);
        if (!s->hx || !s->hy || !s->hz) return -1;
        for (int v = 0; v < s->n; ++v) {
            s->hx[v] = hxyz[3 * v];
            s->hy[v] = hxyz[3 * v + 1];
            s->hz[v] = hxyz[3 * v + 2];
        }
    }
    refresh_energies(s);
    return 0;
}

/*
 * Random bonds (the paper's "other continuous models with random bonds",
 * App. B): H = -sum_(ij) J_ij S_i . S_j with one coupling per bond (J = +1 or
 * -1 for the XY spin glass; any value works), in the order of the bond list.
 * The local field becomes h_i = sum_j J_ij S_j and the energy sums J_ij S_i.S_j;
 * the sweep is otherwise unchanged.  NULL restores J = 1.  Recomputes the
 * energies of the current spins.
 */
int orc_sim_set_couplings(orc_sim *s, const double *j_per_bond)
{
    free(s->jb); free(s->jn);
    s->jb = s->jn = NULL;
    if (!j_per_bond) { refresh_energies(s); return 0; }
    s->jb = (double *)malloc(sizeof(double) * (size_t)(s->n_bonds + 1));
    s->jn = (double *)malloc(sizeof(double) * (size_t)(s->ptr[s->n] + 1));
    if (!s->jb || !s->jn) return -1;
    for (int64_t e = 0; e < s->n_bonds; ++e) {
        s->jb[e] = j_per_bond[e];
        const int ends[2] = { s->bi[e], s->bj[e] };
        for (int q = 0; q < 2; ++q) {
            const int v = ends[q], u = ends[1 - q];
            for (int a = s->ptr[v]; a < s->ptr[v + 1]; ++a)
                if (s->nbr[a] == u) { s->jn[a] = j_per_bond[e]; break; }
        }
    }
    refresh_energies(s);
    return 0;
}

static void metropolis_site_o3(orc_sim *s, int r, int v);
static void overrelax_site_o3(orc_sim *s, int r, int v);
void orc_reflect(int dim, const double *sv, const double *h, double *out);

static void metropolis_site(orc_sim *s, int r, int v)
{
    if (s->dim == 3) { metropolis_site_o3(s, r, v); return; }
    double *x = s->vx + (size_t)r * s->n, *y = s->vy + (size_t)r * s->n;
    int slot = s->slot_of[r];
    uint32_t w[4];
    double ud, ua;
    if (s->u24_mode) {
        /* one block serves replicas 2p and 2p+1: (w0, w1) for the even one, (w2, w3) for the odd */
        draw_block((uint32_t)v, (uint32_t)s->t, PURPOSE_MET, (uint32_t)(r >> 1), s->sample, s->key, w);
        ud = u24(w[(r & 1) ? 2 : 0]);
        ua = u24(w[(r & 1) ? 3 : 1]);
    } else {
        draw_block((uint32_t)v, (uint32_t)s->t, PURPOSE_MET, (uint32_t)r, s->sample, s->key, w);
        ud = u53(w[0], w[1]);
        ua = u53(w[2], w[3]);
    }
    double hx, hy;
    local_field(s, x, y, v, &hx, &hy);
    double d = s->delta[slot] * (2.0 * ud - 1.0);
    double sn, cs;
    orc_sincos_series(d, &sn, &cs);
    double nx = cs * x[v] - sn * y[v];
    double ny = sn * x[v] + cs * y[v];
    double dE = -((nx - x[v]) * hx + (ny - y[v]) * hy);
    int accept;
    if (dE <= 0.0) {
        accept = 1;
        note_tie(s, r, v, -dE, accept);
    } else {
        double a = exp(-s->beta[slot] * dE);
        accept = ua < a;
        double margin = fabs(ua - a);
        if (dE < margin) margin = dE;
        note_tie(s, r, v, margin, accept);
    }
    accept = forced_outcome(s, r, v, accept);
    s->met_try[slot]++;
    if (accept) {
        x[v] = nx;
        y[v] = ny;
        s->met_acc[slot]++;
    }
}

/*
 * Overrelaxation map (App. B, "Improved equilibrium dynamics", Creutz): the
 * reflection of a spin about its local field, s' = 2 (s.h) h / |h|^2 - s, for
 * dim = 2 or 3 components (sums left to right); s is returned unchanged when
 * h = 0.  It conserves s.h (hence the energy) and |s|, and applying it twice
 * gives s back.
 */
void orc_reflect(int dim, const double *sv, const double *h, double *out)
{
    double h2 = h[0] * h[0] + h[1] * h[1];
    double sh = sv[0] * h[0] + sv[1] * h[1];
    if (dim == 3) {
        h2 += h[2] * h[2];
        sh += sv[2] * h[2];
    }
    if (!(h2 > 0.0)) {
        for (int a = 0; a < dim; ++a) out[a] = sv[a];
        return;
    }
    const double k = 2.0 * sh / h2;
    for (int a = 0; a < dim; ++a) out[a] = k * h[a] - sv[a];
}

static void overrelax_site(orc_sim *s, int r, int v)
{
    if (s->dim == 3) { overrelax_site_o3(s, r, v); return; }
    double *x = s->vx + (size_t)r * s->n, *y = s->vy + (size_t)r * s->n;
    double h[2], sv[2] = { x[v], y[v] }, out[2];
    local_field(s, x, y, v, &h[0], &h[1]);
    orc_reflect(2, sv, h, out);
    x[v] = out[0];
    y[v] = out[1];
}

static void parallel_tempering(orc_sim *s)
{
    for (int k = (int)(s->t & 1u); k + 1 < s->R; k += 2) {
        int a = s->rep_at[k], b = s->rep_at[k + 1];
        double x = (s->beta[k] - s->beta[k + 1]) * (s->E[a] - s->E[b]);
        uint32_t w[4];
        draw_block((uint32_t)k, (uint32_t)s->t, PURPOSE_PT, 0, s->sample, s->key, w);
        double u = u53(w[0], w[1]);
        double p = exp(x);
        int accept = u < p;
        if (x < 0.0 && fabs(u - p) < s->tie_eps) {
            if (s->first_pt_tie < 0) s->first_pt_tie = (int64_t)s->t;
            log_tie(&s->pt_log, &s->pt_len, &s->pt_cap, -1, k, (int64_t)s->t, accept);
        }
        if (s->pt_forced && s->pt_forced[k] >= 0) accept = s->pt_forced[k];
        s->pt_try[k]++;
        if (accept) {
            s->rep_at[k] = b; s->rep_at[k + 1] = a;
            s->slot_of[b] = k; s->slot_of[a] = k + 1;
            s->pt_acc[k]++;
        }
    }
}

/* Observables of Sec. III for replica r: e, m, |F(k_min)|^2 (two directions). */
static void observe(const orc_sim *s, int r, double out[ACC_COUNT])
{
    const double *x = s->vx + (size_t)r * s->n, *y = s->vy + (size_t)r * s->n, *z = s->vz + (size_t)r * s->n;
    double mx = 0, my = 0, mz = 0;
    double fxr_a = 0, fxi_a = 0, fyr_a = 0, fyi_a = 0; /* k along x: spin x / y comps */
    double fxr_b = 0, fxi_b = 0, fyr_b = 0, fyi_b = 0; /* k along y */
    double fzr_a = 0, fzi_a = 0, fzr_b = 0, fzi_b = 0; /* spin z component (O(3)) */
    for (int v = 0; v < s->n; ++v) {
        double c = x[v], sn = y[v];
        mx += c; my += sn;
        fxr_a += c * s->cx[v]; fxi_a += c * s->sx[v];
        fyr_a += sn * s->cx[v]; fyi_a += sn * s->sx[v];
        fxr_b += c * s->cy[v]; fxi_b += c * s->sy[v];
        fyr_b += sn * s->cy[v]; fyi_b += sn * s->sy[v];
        if (s->dim == 3) {
            mz += z[v];
            fzr_a += z[v] * s->cx[v]; fzi_a += z[v] * s->sx[v];
            fzr_b += z[v] * s->cy[v]; fzi_b += z[v] * s->sy[v];
        }
    }
    double N = (double)s->n;
    double e = s->E[r] / N;
    mx /= N; my /= N; mz /= N;
    double m2 = mx * mx + my * my;
    double fa = fxr_a * fxr_a + fxi_a * fxi_a + fyr_a * fyr_a + fyi_a * fyi_a;
    double fb = fxr_b * fxr_b + fxi_b * fxi_b + fyr_b * fyr_b + fyi_b * fyi_b;
    if (s->dim == 3) {
        m2 += mz * mz;
        fa += fzr_a * fzr_a + fzi_a * fzi_a;
        fb += fzr_b * fzr_b + fzi_b * fzi_b;
    }
    out[ACC_N] = 1.0;
    out[ACC_E] = e;
    out[ACC_E2] = e * e;
    out[ACC_ABSM] = sqrt(m2);
    out[ACC_MX] = mx;
    out[ACC_MY] = my;
    out[ACC_M2] = m2;
    out[ACC_M4] = m2 * m2;
    out[ACC_CHIK] = (fa + fb) / (2.0 * N);
    out[ACC_MZ] = mz;
}

void orc_sim_sweeps(orc_sim *s, int n_sweeps, unsigned ops, int measure_every)
{
    for (int it = 0; it < n_sweeps; ++it) {
        for (int r = 0; r < s->R; ++r) {
            if (s->active && !s->active[r]) continue;
            if (ops & OP_MET)
                for (int c = 0; c < s->Q; ++c)
                    for (int a = s->cls_ptr[c]; a < s->cls_ptr[c + 1]; ++a) metropolis_site(s, r, s->cls[a]);
            if (ops & OP_OR)
                for (int c = 0; c < s->Q; ++c)
                    for (int a = s->cls_ptr[c]; a < s->cls_ptr[c + 1]; ++a) overrelax_site(s, r, s->cls[a]);
            s->E[r] = energy_of(s, r);
        }
        if (ops & OP_PT) parallel_tempering(s);
        if ((ops & OP_MEASURE) && measure_every > 0 && ((s->t + 1) % (uint64_t)measure_every) == 0) {
            for (int k = 0; k < s->R; ++k) {
                double o[ACC_COUNT];
                observe(s, s->rep_at[k], o);
                for (int q = 0; q < ACC_COUNT; ++q) s->acc[(size_t)k * ACC_COUNT + q] += o[q];
            }
        }
        s->t++;
    }
}

/* angles atan2(y, x) of every spin, [R][n] */
void orc_sim_get_angles(const orc_sim *s, double *out)
{
    for (size_t q = 0; q < (size_t)s->R * (size_t)s->n; ++q) out[q] = atan2(s->vy[q], s->vx[q]);
}

/* spins from angles in (-pi, pi] via the series; energies refreshed */
void orc_sim_set_angles(orc_sim *s, const double *in)
{
    for (size_t q = 0; q < (size_t)s->R * (size_t)s->n; ++q) {
        double th = in[q];
        while (th > ORC_PI) th -= 2.0 * ORC_PI;
        while (th < -ORC_PI) th += 2.0 * ORC_PI;
        orc_sincos_series(th, &s->vy[q], &s->vx[q]);
    }
    refresh_energies(s);
}

/* spin vectors, [R][n][dim] */
void orc_sim_get_vectors(const orc_sim *s, double *out)
{
    const size_t d = (size_t)s->dim;
    for (size_t q = 0; q < (size_t)s->R * (size_t)s->n; ++q) {
        out[d * q] = s->vx[q];
        out[d * q + 1] = s->vy[q];
        if (d == 3) out[d * q + 2] = s->vz[q];
    }
}

void orc_sim_set_vectors(orc_sim *s, const double *in)
{
    const size_t d = (size_t)s->dim;
    for (size_t q = 0; q < (size_t)s->R * (size_t)s->n; ++q) {
        s->vx[q] = in[d * q];
        s->vy[q] = in[d * q + 1];
        if (d == 3) s->vz[q] = in[d * q + 2];
    }
    refresh_energies(s);
}

/* replica at each slot, and the sweep index of the next sweep */
void orc_sim_set_labels(orc_sim *s, const int32_t *rep_at, uint64_t t)
{
    for (int k = 0; k < s->R; ++k) { s->rep_at[k] = rep_at[k]; s->slot_of[rep_at[k]] = k; }
    s->t = t;
}

void orc_sim_get_energies(const orc_sim *s, double *out)
{
    for (int r = 0; r < s->R; ++r) out[r] = s->E[r];
}

void orc_sim_get_labels(const orc_sim *s, int32_t *rep_at)
{
    for (int k = 0; k < s->R; ++k) rep_at[k] = s->rep_at[k];
}

void orc_sim_get_acc(const orc_sim *s, double *acc, uint64_t *met_acc, uint64_t *met_try,
                     uint64_t *pt_acc, uint64_t *pt_try)
{
    memcpy(acc, s->acc, sizeof(double) * (size_t)s->R * ACC_COUNT);
    memcpy(met_acc, s->met_acc, sizeof(uint64_t) * (size_t)s->R);
    memcpy(met_try, s->met_try, sizeof(uint64_t) * (size_t)s->R);
    memcpy(pt_acc, s->pt_acc, sizeof(uint64_t) * (size_t)s->R);
    memcpy(pt_try, s->pt_try, sizeof(uint64_t) * (size_t)s->R);
}

void orc_sim_reset_acc(orc_sim *s)
{
    memset(s->acc, 0, sizeof(double) * (size_t)s->R * ACC_COUNT);
    memset(s->met_acc, 0, sizeof(uint64_t) * (size_t)s->R);
    memset(s->met_try, 0, sizeof(uint64_t) * (size_t)s->R);
    memset(s->pt_acc, 0, sizeof(uint64_t) * (size_t)s->R);
    memset(s->pt_try, 0, sizeof(uint64_t) * (size_t)s->R);
}

void orc_sim_get_ties(const orc_sim *s, int64_t *first_tie, int64_t *first_pt_tie, double *min_margin)
{
    for (int r = 0; r < s->R; ++r) first_tie[r] = s->first_tie[r];
    *first_pt_tie = s->first_pt_tie;
    *min_margin = s->min_margin;
}

void orc_sim_get_tie_counts(const orc_sim *s, int64_t *n_ties)
{
    for (int r = 0; r < s->R; ++r) n_ties[r] = s->n_ties[r];
}

void orc_sim_clear_ties(orc_sim *s)
{
    for (int r = 0; r < s->R; ++r) { s->first_tie[r] = -1; s->n_ties[r] = 0; }
    s->tie_len = 0;
    s->pt_len = 0;
    s->first_pt_tie = -1;
    s->min_margin = INFINITY;
}

uint64_t orc_sim_sweep_index(const orc_sim *s) { return s->t; }

/* ------------------------------------------------------------------------- */
/* Checking aids for the single-precision parity tests.  A single-precision   */
/* kernel evaluates exp(-beta dE) and the PT energies with rounding errors    */
/* far below 1e-5, so it can only take a different outcome where the test is  */
/* that close to flipping.  The log lists every such near-tie test (replica,  */
/* original site id, sweep, outcome); a test then re-runs a sweep with chosen */
/* near-tie outcomes forced the other way, to show that a mismatch comes from */
/* exactly those decisions.  The replica mask lets it re-run one replica      */
/* alone (the others keep their spins and energies; PT then compares stale    */
/* energies, so a masked run is for spins and energies only).                */
/* ------------------------------------------------------------------------- */

/* copy up to max entries of the Metropolis (pt = 0) or PT (pt = 1) near-tie
 * log; returns the number of entries logged since the last clear */
int64_t orc_sim_get_tie_log(const orc_sim *s, int pt, int64_t max, int32_t *rep, int32_t *site, int64_t *sweep,
                            int32_t *accepted)
{
    const orc_tie *log = pt ? s->pt_log : s->tie_log;
    const int64_t len = pt ? s->pt_len : s->tie_len;
    for (int64_t q = 0; q < len && q < max; ++q) {
        rep[q] = log[q].rep; site[q] = log[q].site; sweep[q] = log[q].sweep; accepted[q] = log[q].accepted;
    }
    return len;
}

/* Metropolis outcomes to take at (replica, original site) in the sweeps that
 * follow, instead of the test's; n = 0 removes them all.  Returns -1 on bad
 * input or allocation failure. */
int orc_sim_force(orc_sim *s, int64_t n, const int32_t *rep, const int32_t *site, const int32_t *accept)
{
    if (n <= 0) { free(s->forced); s->forced = NULL; return 0; }
    if (!s->forced) {
        s->forced = (int8_t *)malloc((size_t)s->R * (size_t)s->n);
        if (!s->forced) return -1;
    }
    memset(s->forced, -1, (size_t)s->R * (size_t)s->n);
    for (int64_t q = 0; q < n; ++q) {
        if (rep[q] < 0 || rep[q] >= s->R || site[q] < 0 || site[q] >= s->n) return -1;
        s->forced[(size_t)rep[q] * s->n + site[q]] = accept[q] ? 1 : 0;
    }
    return 0;
}

/* PT outcomes to take for pair k (slots k, k+1) instead of the test's; n = 0 removes them. */
int orc_sim_force_pt(orc_sim *s, int64_t n, const int32_t *pair, const int32_t *accept)
{
    if (n <= 0) { free(s->pt_forced); s->pt_forced = NULL; return 0; }
    if (!s->pt_forced) {
        s->pt_forced = (int8_t *)malloc((size_t)s->R);
        if (!s->pt_forced) return -1;
    }
    memset(s->pt_forced, -1, (size_t)s->R);
    for (int64_t q = 0; q < n; ++q) {
        if (pair[q] < 0 || pair[q] + 1 >= s->R) return -1;
        s->pt_forced[pair[q]] = accept[q] ? 1 : 0;
    }
    return 0;
}

/* mask[r] != 0: the sweeps update replica r; NULL: every replica */
int orc_sim_set_active(orc_sim *s, const uint8_t *mask)
{
    if (!mask) { free(s->active); s->active = NULL; return 0; }
    if (!s->active) {
        s->active = (uint8_t *)malloc((size_t)s->R);
        if (!s->active) return -1;
    }
    memcpy(s->active, mask, (size_t)s->R);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* O(3) spins (App. B: the method carries over to other continuous models;    */
/* O(3) is the paper's example).  S_i = (x, y, z) unit vectors, the same      */
/* Hamiltonian with the three-component dot product, the same sweep, PT and   */
/* measurement; m^2 and chi(k) take all three components, ACC_MZ sums m_z.    */
/* Readings where the paper fixes nothing:                                    */
/*   init: uniform on the sphere (Archimedes): z = 2u - 1, phi = 2 pi u' - pi,*/
/*     rho = sqrt((1 - z)(1 + z)), S = (rho cos phi, rho sin phi, z).          */
/*     53-bit: u = u53(w0,w1), u' = u53(w2,w3) of the INIT block of (i, r);   */
/*     24-bit: u24(w0), u24(w1).  aligned: S = (1, 0, 0).                      */
/*   Metropolis: S' uniform on the spherical cap of angular radius Delta      */
/*     around S (Delta <= pi; Delta = pi is the whole sphere): with            */
/*     w = u (1 - cos Delta) = u * 2 sin^2(Delta / 2), cos theta = 1 - w and  */
/*     sin theta = sqrt(w (2 - w)); azimuth phi = 2 pi u'' - pi in the frame  */
/*     (e1, e2) orthogonal to S of Duff et al. (JCGT 6(1), 2017), its first   */
/*     vector times g:                                                        */
/*       g = +1 if z >= 0 else -1, a = -1 / (g + z), b = x y a,               */
/*       e1 = (g + x^2 a, b, -x),  e2 = (b, g + y^2 a, -y);                    */
/*     S' = cos theta S + sin theta (cos phi e1 + sin phi e2).  The proposal   */
/*     density depends on the angle between S and S' only, so it is          */
/*     symmetric; and the frame of -S is minus the frame of S, bit for bit,   */
/*     so the proposal from -S is minus the proposal from S (the gauge        */
/*     symmetry S -> -S, J -> -J then holds step by step, as for XY).         */
/*     dE = -(S' - S) . h; the test as for XY.                                */
/*     53-bit draws: block (i, t, MET<<24 | r): u = u53(w0,w1), test u53(w2,w3);*/
/*     block (i, t, MET<<24 | 0x800000 | r): u'' = u53(w0,w1).                */
/*     24-bit draws: one block (i, t, MET<<24 | r) per replica: u24(w0) for   */
/*     the cap, u24(w1) for phi, u24(w2) for the test.                        */
/*   Overrelaxation: S' = 2 (S.h) h / |h|^2 - S (rotation by pi about h).     */
/* Random fields: 3-vectors per site (orc_sim_set_fields3), added to the     */
/* local field after the neighbours, -h.S in the energy, as for XY.          */
/* ------------------------------------------------------------------------- */
#define MET_SECOND_BLOCK 0x800000u

int orc_sim_set_dim(orc_sim *s, int dim)
{
    if (dim != 2 && dim != 3) return -1;
    if (s->hx && (s->hz != NULL) != (dim == 3)) return -2;  /* fields keep their component count */
    s->dim = dim;
    memset(s->vz, 0, sizeof(double) * (size_t)s->R * (size_t)s->n);
    refresh_energies(s);
    return 0;
}

int orc_sim_dim(const orc_sim *s) { return s->dim; }

static void init_o3(orc_sim *s, int aligned)
{
    for (int r = 0; r < s->R; ++r) {
        for (int v = 0; v < s->n; ++v) {
            const size_t q = (size_t)r * s->n + v;
            if (aligned) { s->vx[q] = 1.0; s->vy[q] = 0.0; s->vz[q] = 0.0; continue; }
            uint32_t w[4];
            draw_block((uint32_t)v, 0, PURPOSE_INIT, (uint32_t)r, s->sample, s->key, w);
            double u = s->u24_mode ? u24(w[0]) : u53(w[0], w[1]);
            double up = s->u24_mode ? u24(w[1]) : u53(w[2], w[3]);
            double z = 2.0 * u - 1.0;
            double phi = 2.0 * ORC_PI * up - ORC_PI;
            double rho = sqrt((1.0 - z) * (1.0 + z));
            double sn, cs;
            orc_sincos_series(phi, &sn, &cs);
            s->vx[q] = rho * cs;
            s->vy[q] = rho * sn;
            s->vz[q] = z;
        }
    }
}

static void local_field3(const orc_sim *s, int r, int v, double *hx, double *hy, double *hz)
{
    const double *x = s->vx + (size_t)r * s->n, *y = s->vy + (size_t)r * s->n, *z = s->vz + (size_t)r * s->n;
    double ax = 0.0, ay = 0.0, az = 0.0;
    for (int a = s->ptr[v]; a < s->ptr[v + 1]; ++a) {
        const int j = s->nbr[a];
        if (s->jn) {
            ax += s->jn[a] * x[j];
            ay += s->jn[a] * y[j];
            az += s->jn[a] * z[j];
        } else {
            ax += x[j];
            ay += y[j];
            az += z[j];
        }
    }
    if (s->hz) {
        /* the site's own field, added after the neighbours */
        const double f[3] = { s->hx[v], s->hy[v], s->hz[v] };
        ax += f[0];
        ay += f[1];
        az += f[2];
    }
    *hx = ax; *hy = ay; *hz = az;
}

/* the cap proposal of the header above, every step as written there */
void orc_o3_propose(double x, double y, double z, double half_width, double u, double uphi,
                    double *nx, double *ny, double *nz)
{
    double sh, ch;
    orc_sincos_series(0.5 * half_width, &sh, &ch);
    const double w = u * (2.0 * (sh * sh));
    const double ct = 1.0 - w;
    const double st = sqrt(w * (2.0 - w));
    double sp, cp;
    orc_sincos_series(2.0 * ORC_PI * uphi - ORC_PI, &sp, &cp);
    const double g = z >= 0.0 ? 1.0 : -1.0;
    const double a = -1.0 / (g + z);
    const double b = x * y * a;
    const double e1x = g + (x * x) * a, e1y = b, e1z = -x;
    const double e2x = b, e2y = g + (y * y) * a, e2z = -y;
    const double tx = cp * e1x + sp * e2x, ty = cp * e1y + sp * e2y, tz = cp * e1z + sp * e2z;
    *nx = ct * x + st * tx;
    *ny = ct * y + st * ty;
    *nz = ct * z + st * tz;
}

static void metropolis_site_o3(orc_sim *s, int r, int v)
{
    const size_t q = (size_t)r * s->n + v;
    const int slot = s->slot_of[r];
    uint32_t w[4];
    double ud, up, ua;
    draw_block((uint32_t)v, (uint32_t)s->t, PURPOSE_MET, (uint32_t)r, s->sample, s->key, w);
    if (s->u24_mode) {
        ud = u24(w[0]);
        up = u24(w[1]);
        ua = u24(w[2]);
    } else {
        ud = u53(w[0], w[1]);
        ua = u53(w[2], w[3]);
        draw_block((uint32_t)v, (uint32_t)s->t, PURPOSE_MET, MET_SECOND_BLOCK | (uint32_t)r, s->sample, s->key, w);
        up = u53(w[0], w[1]);
    }
    double hx, hy, hz;
    local_field3(s, r, v, &hx, &hy, &hz);
    const double x = s->vx[q], y = s->vy[q], z = s->vz[q];
    double nx, ny, nz;
    orc_o3_propose(x, y, z, s->delta[slot], ud, up, &nx, &ny, &nz);
    const double dE = -((nx - x) * hx + (ny - y) * hy + (nz - z) * hz);
    int accept;
    if (dE <= 0.0) {
        accept = 1;
        note_tie(s, r, v, -dE, accept);
    } else {
        double p = exp(-s->beta[slot] * dE);
        accept = ua < p;
        double margin = fabs(ua - p);
        if (dE < margin) margin = dE;
        note_tie(s, r, v, margin, accept);
    }
    accept = forced_outcome(s, r, v, accept);
    s->met_try[slot]++;
    if (accept) {
        s->vx[q] = nx;
        s->vy[q] = ny;
        s->vz[q] = nz;
        s->met_acc[slot]++;
    }
}

static void overrelax_site_o3(orc_sim *s, int r, int v)
{
    const size_t q = (size_t)r * s->n + v;
    double h[3], sv[3] = { s->vx[q], s->vy[q], s->vz[q] }, out[3];
    local_field3(s, r, v, &h[0], &h[1], &h[2]);
    orc_reflect(3, sv, h, out);
    s->vx[q] = out[0];
    s->vy[q] = out[1];
    s->vz[q] = out[2];
}
