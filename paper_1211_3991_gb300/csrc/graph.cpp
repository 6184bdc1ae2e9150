// Host-side graph construction of libxyl: dilute Levy graphs (Eq. (Levyi)) with
// a fixed degree on the periodic L x L lattice, or with a fixed number of bonds
// on the periodic or free lattice (the paper's own ensemble, Sec. II),
// smallest-last-ordering
// colouring and the colour-sorted CSR (App. B, "Graph coloring" and "Memory
// management").  Compiled without FP contraction so that every decision taken
// from the FP64 link-law table is reproducible bit for bit.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <queue>
#include <set>
#include <utility>

#include "internal.h"
#include "philox.cuh"

namespace xyl {

static thread_local std::string g_last_error;

int fail(int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return code;
}

void clear_error() { g_last_error.clear(); }

namespace {

// ---------------------------------------------------------------------------
// Link-length law on the periodic lattice.  Displacements (dx, dy) with
// dx, dy in {-L/2+1, ..., L/2} reach every other site once (r_max = L/sqrt(2),
// Sec. II).  Entries with dx^2 + dy^2 <= 8 form the "near" group and come
// first; the rest follow, each group in raster order (dy outer, dx inner).
// Weight r^-rho per partner site; the FP64 running sum S_k before entry k maps
// to the 64-bit boundary floor(2^64 S_k / S_total).  Every draw compares
// 64-bit integers against these boundaries.
// ---------------------------------------------------------------------------
constexpr int kNearR2 = 8;
constexpr int kMaxReject = 64;
constexpr int kMaxRestarts = 100;

struct LinkLaw {
    int L = 0;
    int entries = 0;
    int near = 0;
    std::vector<int32_t> ddx, ddy;
    std::vector<uint64_t> lower;      // lower boundary of each entry
    std::vector<int32_t> entry_of;    // (dy+L/2-1)*L + (dx+L/2-1) -> entry

    uint64_t weight(int k) const
    {
        const uint64_t upper = (k + 1 < entries) ? lower[k + 1] : 0;  // 2^64 == 0 (mod 2^64)
        return upper - lower[k];
    }
    // entry whose [lower_k, lower_k+1) holds u, searching from `first`
    int find(uint64_t u, int first) const
    {
        auto it = std::upper_bound(lower.begin() + first, lower.end(), u);
        return (int)(it - lower.begin()) - 1;
    }
    int between(int i, int j) const
    {
        const int h = L / 2;
        int dx = (j % L) - (i % L), dy = (j / L) - (i / L);
        if (dx > h) dx -= L; else if (dx <= -h) dx += L;
        if (dy > h) dy -= L; else if (dy <= -h) dy += L;
        return entry_of[(dy + h - 1) * L + (dx + h - 1)];
    }
    int shift(int i, int k) const
    {
        const int x = ((i % L) + ddx[k] + L) % L;
        const int y = ((i / L) + ddy[k] + L) % L;
        return x + L * y;
    }
};

LinkLaw make_law(int L, double rho)
{
    LinkLaw law;
    law.L = L;
    law.entries = L * L - 1;
    law.ddx.reserve(law.entries);
    law.ddy.reserve(law.entries);
    law.entry_of.assign((size_t)L * L, -1);
    const int h = L / 2;
    for (int group = 0; group < 2; ++group) {
        for (int dy = 1 - h; dy <= h; ++dy)
            for (int dx = 1 - h; dx <= h; ++dx) {
                const int r2 = dx * dx + dy * dy;
                if (r2 == 0 || (r2 <= kNearR2) != (group == 0)) continue;
                law.entry_of[(dy + h - 1) * L + (dx + h - 1)] = (int)law.ddx.size();
                law.ddx.push_back(dx);
                law.ddy.push_back(dy);
            }
        if (group == 0) law.near = (int)law.ddx.size();
    }
    std::vector<double> run(law.entries + 1, 0.0);
    for (int k = 0; k < law.entries; ++k) {
        const double r2 = (double)(law.ddx[k] * law.ddx[k] + law.ddy[k] * law.ddy[k]);
        run[k + 1] = run[k] + std::pow(r2, -0.5 * rho);
    }
    const double two64 = 18446744073709551616.0;
    law.lower.assign(law.entries, 0);
    for (int k = 1; k < law.entries; ++k) {
        const double q = (run[k] / run[law.entries]) * two64;
        law.lower[k] = (q >= two64) ? ~0ull : (uint64_t)q;
    }
    return law;
}

// 64-bit draws: block b gives (w1:w0) then (w3:w2).
class DrawStream {
  public:
    DrawStream(uint64_t key, uint32_t sample, uint32_t restart) : key_(key), sample_(sample), restart_(restart) {}
    uint64_t next()
    {
        if (!have_second_) {
            cur_ = philox_draw((uint32_t)block_, (uint32_t)(block_ >> 32), kPurposeGraph, restart_, sample_, key_);
            have_second_ = true;
            return ((uint64_t)cur_.w1 << 32) | cur_.w0;
        }
        have_second_ = false;
        ++block_;
        return ((uint64_t)cur_.w3 << 32) | cur_.w2;
    }

  private:
    uint64_t key_;
    uint32_t sample_, restart_;
    uint64_t block_ = 0;
    bool have_second_ = false;
    Words4 cur_{};
};

inline uint64_t scale_u64(uint64_t u, uint64_t m) { return (uint64_t)(((unsigned __int128)u * m) >> 64); }

struct Pairing {
    int n, z;
    std::vector<int32_t> degree;
    std::vector<int32_t> links;     // n * z
    std::vector<int32_t> open;      // unsaturated sites
    std::vector<int32_t> open_pos;  // index in `open`, -1 once saturated

    Pairing(int n_, int z_) : n(n_), z(z_), degree(n_), links((size_t)n_ * z_), open(n_), open_pos(n_) {}

    void reset()
    {
        open.resize(n);
        for (int v = 0; v < n; ++v) { degree[v] = 0; open[v] = v; open_pos[v] = v; }
    }
    bool linked(int i, int j) const
    {
        const int32_t *row = &links[(size_t)i * z];
        for (int a = 0; a < degree[i]; ++a)
            if (row[a] == j) return true;
        return false;
    }
    bool can_link(int i, int j) const { return j != i && degree[j] < z && !linked(i, j); }
    void link(int i, int j)
    {
        links[(size_t)i * z + degree[i]++] = j;
        links[(size_t)j * z + degree[j]++] = i;
        close_if_full(i);
        close_if_full(j);
    }
    void close_if_full(int v)
    {
        if (degree[v] < z) return;
        const int at = open_pos[v];
        const int moved = open.back();
        open[at] = moved;
        open_pos[moved] = at;
        open.pop_back();
        open_pos[v] = -1;
    }
};

// Partner of i drawn with the link law restricted to eligible sites; -1 = dead end.
int draw_partner(const LinkLaw &law, const Pairing &pr, int i, DrawStream &ds)
{
    unsigned __int128 near_w = 0;
    for (int k = 0; k < law.near; ++k)
        if (pr.can_link(i, law.shift(i, k))) near_w += law.weight(k);
    const unsigned __int128 far_w =
        (law.near < law.entries) ? (((unsigned __int128)1 << 64) - law.lower[law.near]) : 0;
    const unsigned __int128 total = near_w + far_w;
    if (total != 0) {
        for (int attempt = 0; attempt < kMaxReject; ++attempt) {
            const unsigned __int128 t = ((unsigned __int128)ds.next() * total) >> 64;
            if (t < near_w) {
                unsigned __int128 acc = 0;
                for (int k = 0; k < law.near; ++k) {
                    const int j = law.shift(i, k);
                    if (!pr.can_link(i, j)) continue;
                    acc += law.weight(k);
                    if (acc > t) return j;
                }
            }
            const uint64_t where = law.lower[law.near] + (uint64_t)(t - near_w);
            const int j = law.shift(i, law.find(where, law.near));
            if (pr.can_link(i, j)) return j;
        }
    }
    // exhaustive draw over the open list (list order)
    unsigned __int128 sum = 0;
    for (int32_t j : pr.open)
        if (pr.can_link(i, j)) sum += law.weight(law.between(i, j));
    if (sum == 0) return -1;
    const unsigned __int128 t = ((unsigned __int128)ds.next() * sum) >> 64;
    unsigned __int128 acc = 0;
    for (int32_t j : pr.open) {
        if (!pr.can_link(i, j)) continue;
        acc += law.weight(law.between(i, j));
        if (acc > t) return j;
    }
    return -1;
}

// ---------------------------------------------------------------------------
// Free boundaries: displacements |dx|, |dy| <= L-1 inside the L x L square
// (r_max = L sqrt 2, Sec. II), raster order (dy outer, dx inner), weight
// r^-rho per displacement, boundaries from the FP64 running sum as above.
// ---------------------------------------------------------------------------
LinkLaw make_free_law(int L, double rho)
{
    LinkLaw law;
    law.L = L;
    law.entries = (2 * L - 1) * (2 * L - 1) - 1;
    law.near = 0;
    law.ddx.reserve(law.entries);
    law.ddy.reserve(law.entries);
    for (int dy = 1 - L; dy <= L - 1; ++dy)
        for (int dx = 1 - L; dx <= L - 1; ++dx) {
            if (dx == 0 && dy == 0) continue;
            law.ddx.push_back(dx);
            law.ddy.push_back(dy);
        }
    std::vector<double> run(law.entries + 1, 0.0);
    for (int k = 0; k < law.entries; ++k) {
        const double r2 = (double)(law.ddx[k] * law.ddx[k] + law.ddy[k] * law.ddy[k]);
        run[k + 1] = run[k] + std::pow(r2, -0.5 * rho);
    }
    const double two64 = 18446744073709551616.0;
    law.lower.assign(law.entries, 0);
    for (int k = 1; k < law.entries; ++k) {
        const double q = (run[k] / run[law.entries]) * two64;
        law.lower[k] = (q >= two64) ? ~0ull : (uint64_t)q;
    }
    return law;
}

// Stream id of the M-bond ensemble in counter word 2 (below the purpose byte),
// apart from the pairing restarts of the fixed-degree ensemble.
constexpr uint32_t kBondStream = 0x400000u;

// M distinct bonds, each attempt one Philox block: the first site from
// w1:w0, the displacement from w3:w2; a free-boundary partner outside the
// square or an existing bond rejects the attempt.
bool draw_bonds(const LinkLaw &law, bool free_bc, int64_t n_bonds, uint64_t seed, uint32_t sample, xyl_graph &g,
                uint64_t *attempts)
{
    const int L = law.L;
    const uint64_t n = (uint64_t)L * L;
    std::vector<std::vector<int32_t>> nbr(n);
    const uint64_t limit = 64u * (uint64_t)n_bonds + 1000000u;
    int64_t e = 0;
    uint64_t a = 0;
    for (; e < n_bonds && a < limit; ++a) {
        const Words4 w = philox_draw((uint32_t)a, (uint32_t)(a >> 32), kPurposeGraph, kBondStream | (free_bc ? 1u : 0u),
                                     sample, seed);
        const int i = (int)scale_u64(((uint64_t)w.w1 << 32) | w.w0, n);
        const int k = law.find(((uint64_t)w.w3 << 32) | w.w2, 0);
        int j;
        if (free_bc) {
            const int x = i % L + law.ddx[k], y = i / L + law.ddy[k];
            if (x < 0 || x >= L || y < 0 || y >= L) continue;
            j = x + L * y;
        } else {
            j = law.shift(i, k);
        }
        if (std::find(nbr[i].begin(), nbr[i].end(), j) != nbr[i].end()) continue;
        nbr[i].push_back(j);
        nbr[j].push_back(i);
        g.ei[e] = i;
        g.ej[e] = j;
        ++e;
    }
    *attempts = a;
    return e == n_bonds;
}

// ---------------------------------------------------------------------------
// Smallest-last ordering: peel a vertex of least remaining degree (ties: least
// id) until none is left, then colour in the reverse peeling order with the
// least colour absent among already-coloured neighbours.
// ---------------------------------------------------------------------------
int colour_slo(int n, const std::vector<int32_t> &adj_ptr, const std::vector<int32_t> &adj,
               std::vector<int32_t> &colour)
{
    std::vector<int32_t> remaining(n);
    std::vector<char> peeled(n, 0);
    using Key = std::pair<int32_t, int32_t>;  // (remaining degree, id)
    std::priority_queue<Key, std::vector<Key>, std::greater<Key>> heap;
    for (int v = 0; v < n; ++v) {
        remaining[v] = adj_ptr[v + 1] - adj_ptr[v];
        heap.push({remaining[v], v});
    }
    std::vector<int32_t> order;
    order.reserve(n);
    while ((int)order.size() < n) {
        const Key top = heap.top();
        heap.pop();
        const int v = top.second;
        if (peeled[v] || top.first != remaining[v]) continue;
        peeled[v] = 1;
        order.push_back(v);
        for (int a = adj_ptr[v]; a < adj_ptr[v + 1]; ++a) {
            const int u = adj[a];
            if (!peeled[u]) heap.push({--remaining[u], u});
        }
    }
    colour.assign(n, -1);
    int n_colors = 0;
    std::vector<int32_t> seen_at(n + 1, -1);
    for (int idx = n - 1; idx >= 0; --idx) {
        const int v = order[idx];
        for (int a = adj_ptr[v]; a < adj_ptr[v + 1]; ++a)
            if (colour[adj[a]] >= 0) seen_at[colour[adj[a]]] = v;
        int c = 0;
        while (seen_at[c] == v) ++c;
        colour[v] = c;
        n_colors = std::max(n_colors, c + 1);
    }
    return n_colors;
}

void finish_graph(xyl_graph &g)
{
    const int n = g.n;
    std::vector<int32_t> adj_ptr(n + 1, 0), adj(2 * g.n_edges);
    for (int64_t e = 0; e < g.n_edges; ++e) { adj_ptr[g.ei[e] + 1]++; adj_ptr[g.ej[e] + 1]++; }
    for (int v = 0; v < n; ++v) adj_ptr[v + 1] += adj_ptr[v];
    std::vector<int32_t> fill(adj_ptr.begin(), adj_ptr.end() - 1);
    for (int64_t e = 0; e < g.n_edges; ++e) {
        adj[fill[g.ei[e]]++] = g.ej[e];
        adj[fill[g.ej[e]]++] = g.ei[e];
    }
    g.n_colors = colour_slo(n, adj_ptr, adj, g.color);
    // colour-sorted ids: stable counting sort by colour keeps original order inside a class
    g.color_ptr.assign(g.n_colors + 1, 0);
    for (int v = 0; v < n; ++v) g.color_ptr[g.color[v] + 1]++;
    for (int c = 0; c < g.n_colors; ++c) g.color_ptr[c + 1] += g.color_ptr[c];
    std::vector<int32_t> next(g.color_ptr.begin(), g.color_ptr.end() - 1), sorted_id(n);
    g.perm.assign(n, 0);
    for (int v = 0; v < n; ++v) {
        const int s = next[g.color[v]]++;
        g.perm[s] = v;
        sorted_id[v] = s;
    }
    g.row_ptr.assign(n + 1, 0);
    g.col.assign(2 * g.n_edges, 0);
    g.max_deg = 0;
    for (int s = 0; s < n; ++s) {
        const int v = g.perm[s];
        const int d = adj_ptr[v + 1] - adj_ptr[v];
        g.row_ptr[s + 1] = g.row_ptr[s] + d;
        g.max_deg = std::max(g.max_deg, d);
        int32_t *row = &g.col[g.row_ptr[s]];
        for (int a = 0; a < d; ++a) row[a] = sorted_id[adj[adj_ptr[v] + a]];
        std::sort(row, row + d);
    }
}

}  // namespace
}  // namespace xyl

using namespace xyl;

extern "C" {

const char *xyl_last_error(void) { return g_last_error.c_str(); }

int xyl_version(void) { return 100; }

int xyl_build_graph_csr(int32_t L, int32_t z, double rho, uint64_t seed, uint32_t sample_id, xyl_graph **out)
{
    clear_error();
    if (!out) return fail(XYL_EINVAL, "xyl_build_graph_csr: out is NULL");
    *out = nullptr;
    if (L < 4 || (L & 1) || L > 4096) return fail(XYL_EINVAL, "xyl_build_graph_csr: L=%d must be even in [4,4096]", L);
    const int64_t n = (int64_t)L * L;
    if (z < 1 || z >= n || (n * z) % 2) return fail(XYL_EINVAL, "xyl_build_graph_csr: bad z=%d for N=%lld", z, (long long)n);
    if (!std::isfinite(rho)) return fail(XYL_EINVAL, "xyl_build_graph_csr: rho must be finite");
    try {
        const LinkLaw law = make_law(L, rho);
        Pairing pr((int)n, z);
        auto *g = new xyl_graph();
        g->n = (int32_t)n; g->L = L; g->z = z; g->n_edges = n * z / 2;
        g->ei.resize(g->n_edges); g->ej.resize(g->n_edges);
        bool done = false;
        for (int restart = 0; restart < kMaxRestarts && !done; ++restart) {
            pr.reset();
            DrawStream ds(seed, sample_id, (uint32_t)restart);
            int64_t e = 0;
            bool dead = false;
            while (!pr.open.empty()) {
                const int i = pr.open[scale_u64(ds.next(), pr.open.size())];
                const int j = draw_partner(law, pr, i, ds);
                if (j < 0) { dead = true; break; }
                pr.link(i, j);
                g->ei[e] = i; g->ej[e] = j; ++e;
            }
            if (!dead) { done = true; g->restarts = restart; }
        }
        if (!done) {
            delete g;
            return fail(XYL_EGRAPH, "xyl_build_graph_csr: every one of %d attempts hit a dead end", kMaxRestarts);
        }
        g->xy.resize(2 * n);
        for (int64_t v = 0; v < n; ++v) { g->xy[2 * v] = (int32_t)(v % L); g->xy[2 * v + 1] = (int32_t)(v / L); }
        finish_graph(*g);
        *out = g;
        return XYL_OK;
    } catch (const std::exception &ex) {
        return fail(XYL_EINVAL, "xyl_build_graph_csr: %s", ex.what());
    }
}

int xyl_build_levy_bonds(int32_t L, double rho, int64_t n_bonds, int32_t boundary, uint64_t seed, uint32_t sample_id,
                         xyl_graph **out)
{
    clear_error();
    if (!out) return fail(XYL_EINVAL, "xyl_build_levy_bonds: out is NULL");
    *out = nullptr;
    if (boundary != XYL_PBC && boundary != XYL_FBC)
        return fail(XYL_EINVAL, "xyl_build_levy_bonds: boundary=%d is neither XYL_PBC nor XYL_FBC", boundary);
    const bool free_bc = boundary == XYL_FBC;
    if (free_bc ? (L < 2 || L > 4096) : (L < 4 || (L & 1) || L > 4096))
        return fail(XYL_EINVAL, "xyl_build_levy_bonds: L=%d must be %s", L,
                    free_bc ? "in [2,4096]" : "even in [4,4096]");
    const int64_t n = (int64_t)L * L;
    if (n_bonds < 0 || n_bonds > n * (n - 1) / 2)
        return fail(XYL_EINVAL, "xyl_build_levy_bonds: n_bonds=%lld outside [0, N(N-1)/2]", (long long)n_bonds);
    if (!std::isfinite(rho)) return fail(XYL_EINVAL, "xyl_build_levy_bonds: rho must be finite");
    try {
        const LinkLaw law = free_bc ? make_free_law(L, rho) : make_law(L, rho);
        auto *g = new xyl_graph();
        g->n = (int32_t)n; g->L = L; g->z = 0; g->n_edges = n_bonds;
        g->ei.resize(n_bonds); g->ej.resize(n_bonds);
        uint64_t attempts = 0;
        if (!draw_bonds(law, free_bc, n_bonds, seed, sample_id, *g, &attempts)) {
            delete g;
            return fail(XYL_EGRAPH, "xyl_build_levy_bonds: %llu attempts gave fewer than %lld distinct bonds",
                        (unsigned long long)attempts, (long long)n_bonds);
        }
        g->xy.resize(2 * n);
        for (int64_t v = 0; v < n; ++v) { g->xy[2 * v] = (int32_t)(v % L); g->xy[2 * v + 1] = (int32_t)(v / L); }
        finish_graph(*g);
        *out = g;
        return XYL_OK;
    } catch (const std::exception &ex) {
        return fail(XYL_EINVAL, "xyl_build_levy_bonds: %s", ex.what());
    }
}

int xyl_graph_from_edges(int32_t n, int64_t n_edges, const int32_t *edges, const int32_t *xy, int32_t L,
                         xyl_graph **out)
{
    clear_error();
    if (!out) return fail(XYL_EINVAL, "xyl_graph_from_edges: out is NULL");
    *out = nullptr;
    if (n < 1 || n_edges < 0 || (n_edges > 0 && !edges)) return fail(XYL_EINVAL, "xyl_graph_from_edges: bad sizes");
    if (xy && L < 1) return fail(XYL_EINVAL, "xyl_graph_from_edges: L must be >= 1 with coordinates");
    std::set<std::pair<int32_t, int32_t>> seen;
    for (int64_t e = 0; e < n_edges; ++e) {
        const int32_t a = edges[2 * e], b = edges[2 * e + 1];
        if (a < 0 || b < 0 || a >= n || b >= n) return fail(XYL_EINVAL, "xyl_graph_from_edges: id out of range at edge %lld", (long long)e);
        if (a == b) return fail(XYL_EINVAL, "xyl_graph_from_edges: self-loop at edge %lld", (long long)e);
        if (!seen.insert({std::min(a, b), std::max(a, b)}).second)
            return fail(XYL_EINVAL, "xyl_graph_from_edges: repeated pair at edge %lld", (long long)e);
    }
    auto *g = new xyl_graph();
    g->n = n; g->n_edges = n_edges; g->z = 0;
    g->ei.resize(n_edges); g->ej.resize(n_edges);
    for (int64_t e = 0; e < n_edges; ++e) { g->ei[e] = edges[2 * e]; g->ej[e] = edges[2 * e + 1]; }
    g->xy.resize(2 * (size_t)n);
    for (int v = 0; v < n; ++v) {
        g->xy[2 * v] = xy ? xy[2 * v] : v;
        g->xy[2 * v + 1] = xy ? xy[2 * v + 1] : 0;
    }
    g->L = xy ? L : n;
    finish_graph(*g);
    *out = g;
    return XYL_OK;
}

int xyl_graph_info(const xyl_graph *g, int32_t *n, int64_t *n_edges, int32_t *n_colors, int32_t *max_deg,
                   int32_t *restarts)
{
    if (!g) return fail(XYL_EINVAL, "xyl_graph_info: NULL graph");
    if (n) *n = g->n;
    if (n_edges) *n_edges = g->n_edges;
    if (n_colors) *n_colors = g->n_colors;
    if (max_deg) *max_deg = g->max_deg;
    if (restarts) *restarts = g->restarts;
    return XYL_OK;
}

int xyl_graph_export_csr(const xyl_graph *g, int32_t *perm, int32_t *row_ptr, int32_t *col, int32_t *color_ptr)
{
    if (!g) return fail(XYL_EINVAL, "xyl_graph_export_csr: NULL graph");
    if (perm) std::memcpy(perm, g->perm.data(), sizeof(int32_t) * g->perm.size());
    if (row_ptr) std::memcpy(row_ptr, g->row_ptr.data(), sizeof(int32_t) * g->row_ptr.size());
    if (col) std::memcpy(col, g->col.data(), sizeof(int32_t) * g->col.size());
    if (color_ptr) std::memcpy(color_ptr, g->color_ptr.data(), sizeof(int32_t) * g->color_ptr.size());
    return XYL_OK;
}

int xyl_graph_export_edges(const xyl_graph *g, int32_t *ei, int32_t *ej)
{
    if (!g) return fail(XYL_EINVAL, "xyl_graph_export_edges: NULL graph");
    if (ei) std::memcpy(ei, g->ei.data(), sizeof(int32_t) * g->ei.size());
    if (ej) std::memcpy(ej, g->ej.data(), sizeof(int32_t) * g->ej.size());
    return XYL_OK;
}

int xyl_graph_set_couplings(xyl_graph *g, const int8_t *j)
{
    clear_error();
    if (!g) return fail(XYL_EINVAL, "xyl_graph_set_couplings: NULL graph");
    if (!j) {
        g->jlink.clear();
        g->jcsr.clear();
        return XYL_OK;
    }
    for (int64_t e = 0; e < g->n_edges; ++e)
        if (j[e] != 1 && j[e] != -1) return fail(XYL_EINVAL, "xyl_graph_set_couplings: J[%lld] = %d is not +1 or -1",
                                                 (long long)e, (int)j[e]);
    // colour-sorted id of each original id, then the entry of each link in both rows
    std::vector<int32_t> sorted(g->n);
    for (int s = 0; s < g->n; ++s) sorted[g->perm[s]] = s;
    std::vector<int8_t> csr(g->col.size(), 1);
    for (int64_t e = 0; e < g->n_edges; ++e) {
        const int a = sorted[g->ei[e]], b = sorted[g->ej[e]];
        const int ends[2][2] = {{a, b}, {b, a}};
        for (const auto &rb : ends) {
            const int32_t *lo = g->col.data() + g->row_ptr[rb[0]], *hi = g->col.data() + g->row_ptr[rb[0] + 1];
            const int32_t *at = std::lower_bound(lo, hi, rb[1]);
            csr[at - g->col.data()] = j[e];
        }
    }
    g->jlink.assign(j, j + g->n_edges);
    g->jcsr.swap(csr);
    return XYL_OK;
}

static int set_fields(xyl_graph *g, const double *h, int dim, const char *who)
{
    clear_error();
    if (!g) return fail(XYL_EINVAL, "%s: NULL graph", who);
    if (!h) {
        g->field.clear();
        g->field_dim = 0;
        return XYL_OK;
    }
    for (int64_t k = 0; k < dim * (int64_t)g->n; ++k)
        if (!std::isfinite(h[k])) return fail(XYL_EINVAL, "%s: component %lld is not finite", who, (long long)k);
    g->field.assign(h, h + dim * (size_t)g->n);
    g->field_dim = dim;
    return XYL_OK;
}

int xyl_graph_set_fields(xyl_graph *g, const double *hxy) { return set_fields(g, hxy, 2, "xyl_graph_set_fields"); }

int xyl_graph_set_fields3(xyl_graph *g, const double *hxyz)
{
    return set_fields(g, hxyz, 3, "xyl_graph_set_fields3");
}

int xyl_graph_export_couplings(const xyl_graph *g, int8_t *j_csr)
{
    if (!g || !j_csr) return fail(XYL_EINVAL, "xyl_graph_export_couplings: NULL argument");
    for (size_t k = 0; k < g->col.size(); ++k) j_csr[k] = g->jcsr.empty() ? (int8_t)1 : g->jcsr[k];
    return XYL_OK;
}

void xyl_graph_free(xyl_graph *g) { delete g; }

}  // extern "C"
