"""Pins of the oracle's graph construction, colouring and CSR.

Checks against what the definitions fix: the link law of Eq. (Levyi) through an
independent brute-force count of minimum-image distances, the exact conditional
partner law in every branch of the draw, exact degree / symmetry / simplicity,
properness and the degeneracy bound of smallest-last colouring, and hand-derived
colourings of small graphs.
"""
import numpy as np
import pytest
from scipy import stats

from helpers import min_image_r2_counts


def _law_by_r2(L, rho):
    counts = min_image_r2_counts(L)
    r2 = np.array(sorted(counts))
    p = np.array([counts[v] * float(v) ** (-rho / 2) for v in r2])
    return r2, p / p.sum()


@pytest.mark.parametrize("L", [4, 8, 16, 64])
def test_disp_table_covers_each_partner_once(orc, L):
    dx, dy, B, n_near = orc.disp_table(L, 3.5)
    assert len(dx) == L * L - 1
    cells = set(zip(((dx % L)).tolist(), ((dy % L)).tolist()))
    assert len(cells) == L * L - 1 and (0, 0) not in cells
    # the table's squared lengths equal the minimum-image distances, as a multiset
    r2_tab = np.unique(dx.astype(np.int64) ** 2 + dy.astype(np.int64) ** 2, return_counts=True)
    want = min_image_r2_counts(L)
    assert dict(zip(r2_tab[0].tolist(), r2_tab[1].tolist())) == want
    # boundaries non-decreasing from 0; near group = squared length <= 8
    assert B[0] == 0 and np.all(np.diff(B.astype(object)) >= 0)
    r2 = dx.astype(np.int64) ** 2 + dy.astype(np.int64) ** 2
    assert np.all(r2[:n_near] <= 8) and np.all(r2[n_near:] > 8)


@pytest.mark.parametrize("L,rho", [(16, 3.5), (32, 2.5), (32, 4.5)])
def test_proposal_law_chi2(orc, L, rho):
    """Eq. (Levyi): proposals follow g(r) r^-rho exactly (g = multiplicity)."""
    dx, dy, B, _ = orc.disp_table(L, rho)
    ent = orc.disp_sample(L, rho, seed=99, sample=3, n_draws=400_000)
    r2_of = dx.astype(np.int64) ** 2 + dy.astype(np.int64) ** 2
    r2, p = _law_by_r2(L, rho)
    drawn = r2_of[ent]
    obs = np.array([(drawn == v).sum() for v in r2])
    exp = p * len(ent)
    keep = exp >= 20
    obs_k = np.append(obs[keep], obs[~keep].sum())
    exp_k = np.append(exp[keep], exp[~keep].sum())
    assert stats.chisquare(obs_k, exp_k).pvalue > 1e-4


def _r2_between(L, i, j):
    dx = abs(i % L - j % L)
    dy = abs(i // L - j // L)
    dx = min(dx, L - dx)
    dy = min(dy, L - dy)
    return dx * dx + dy * dy


def _exact_partner_law(L, z, rho, deg, adj, i):
    n = L * L
    p = np.zeros(n)
    for j in range(n):
        if j == i or deg[j] >= z or j in adj[i][: deg[i]]:
            continue
        p[j] = float(_r2_between(L, i, j)) ** (-rho / 2)
    return p / p.sum() if p.sum() > 0 else p


def _state(L, z, saturated, i, i_links):
    n = L * L
    deg = np.zeros(n, np.int32)
    adj = -np.ones((n, z), np.int32)
    for v in saturated:
        deg[v] = z
    for a, j in enumerate(i_links):
        adj[i, a] = j
    deg[i] = len(i_links)
    unsat = np.array([v for v in range(n) if deg[v] < z], np.int32)
    return deg, adj, unsat


@pytest.mark.parametrize("case", ["fresh", "near_full", "few_left", "dead"])
def test_partner_law_every_branch(orc, case):
    """Each branch of the partner draw reproduces the exact conditional law."""
    L, z, rho, i = 16, 6, 3.5, 5 + 16 * 7
    rng = np.random.default_rng(1)
    n = L * L
    if case == "fresh":
        deg, adj, unsat = _state(L, z, [], i, [])
    elif case == "near_full":
        # every site within squared distance 8 of i saturated, 70% of the rest too
        near = [j for j in range(n) if j != i and _r2_between(L, i, j) <= 8]
        rest = [j for j in range(n) if j != i and j not in near]
        sat = near + list(rng.choice(rest, size=int(0.7 * len(rest)), replace=False))
        free = [j for j in rest if j not in sat]
        deg, adj, unsat = _state(L, z, sat, i, [free[0], free[1]])
    elif case == "few_left":
        others = [j for j in range(n) if j != i]
        keep = [j for j in others if _r2_between(L, i, j) >= 32][:4]
        sat = [j for j in others if j not in keep]
        deg, adj, unsat = _state(L, z, sat, i, [keep[0]])
    else:
        others = [j for j in range(n) if j != i]
        keep = [others[100]]
        sat = [j for j in others if j not in keep]
        deg, adj, unsat = _state(L, z, sat, i, [keep[0]])
    trials = 200_000
    counts = orc.pick_partner_counts(L, z, rho, 1234, deg, adj.reshape(-1), unsat, i, trials)
    p = _exact_partner_law(L, z, rho, deg, adj, i)
    if case == "dead":
        assert counts[n] == trials
        return
    assert counts[n] == 0
    assert np.all(counts[:n][p == 0] == 0)
    nz = p > 0
    exp = p[nz] * trials
    obs = counts[:n][nz]
    keep = exp >= 20
    obs_k = np.append(obs[keep], obs[~keep].sum())
    exp_k = np.append(exp[keep], exp[~keep].sum())
    if (~keep).sum() == 0:
        obs_k, exp_k = obs_k[:-1], exp_k[:-1]
    if len(obs_k) == 1:
        assert obs_k[0] == trials
    else:
        assert stats.chisquare(obs_k, exp_k).pvalue > 1e-4


def _check_simple_regular(L, z, ei, ej):
    n = L * L
    assert len(ei) == n * z // 2
    assert np.all(ei != ej)
    deg = np.bincount(np.concatenate([ei, ej]), minlength=n)
    assert np.all(deg == z)
    pairs = set()
    for a, b in zip(ei.tolist(), ej.tolist()):
        key = (min(a, b), max(a, b))
        assert key not in pairs
        pairs.add(key)


@pytest.mark.parametrize("L,rho", [(4, 3.5), (8, 3.0), (16, 3.5), (32, 2.5), (32, 4.5), (64, 3.0)])
def test_graph_is_simple_and_z_regular(orc, L, rho):
    for seed in range(3):
        ei, ej, restarts, _ = orc.levy_graph(L, 6, rho, seed)
        _check_simple_regular(L, 6, ei, ej)


def test_graph_is_deterministic_and_seeded(orc):
    a = orc.levy_graph(16, 6, 3.5, 7, sample=2)
    b = orc.levy_graph(16, 6, 3.5, 7, sample=2)
    c = orc.levy_graph(16, 6, 3.5, 7, sample=3)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    assert not (np.array_equal(a[0], c[0]) and np.array_equal(a[1], c[1]))


def test_first_link_law(orc):
    """First link of a fresh graph: chooser uniform over sites, length law exact."""
    L, rho = 8, 3.0
    firsts_i, r2s = [], []
    for seed in range(3000):
        ei, ej, _, _ = orc.levy_graph(L, 6, rho, seed, max_restarts=1000)
        firsts_i.append(ei[0])
        r2s.append(_r2_between(L, int(ei[0]), int(ej[0])))
    r2, p = _law_by_r2(L, rho)
    r2s = np.array(r2s)
    obs = np.array([(r2s == v).sum() for v in r2])
    exp = p * len(r2s)
    keep = exp >= 20
    obs_k = np.append(obs[keep], obs[~keep].sum())
    exp_k = np.append(exp[keep], exp[~keep].sum())
    assert stats.chisquare(obs_k, exp_k).pvalue > 1e-4
    hist = np.bincount(np.array(firsts_i), minlength=L * L)
    assert stats.chisquare(hist).pvalue > 1e-4


def _r2_links(L, ei, ej):
    a, b = np.asarray(ei), np.asarray(ej)
    dx = np.abs(a % L - b % L)
    dy = np.abs(a // L - b // L)
    dx = np.minimum(dx, L - dx)
    dy = np.minimum(dy, L - dy)
    return dx * dx + dy * dy


@pytest.mark.parametrize("rho", [2.5, 3.5, 4.5])
def test_early_links_follow_law(orc, rho):
    """The first 5% of links (few sites saturated yet) follow the exact law."""
    L = 128
    r2, p = _law_by_r2(L, rho)
    r2s = []
    for seed in range(3):
        ei, ej, _, _ = orc.levy_graph(L, 6, rho, 21 + seed)
        k = len(ei) // 20
        r2s.append(_r2_links(L, ei[:k], ej[:k]))
    r2s = np.concatenate(r2s)
    obs = np.array([(r2s == v).sum() for v in r2])
    exp = p * len(r2s)
    keep = exp >= 20
    obs_k = np.append(obs[keep], obs[~keep].sum())
    exp_k = np.append(exp[keep], exp[~keep].sum())
    # saturation already conditions a few late draws of this window: loose threshold
    assert stats.chisquare(obs_k, exp_k).pvalue > 1e-6


def test_accepted_link_bias_is_size_stable(orc):
    """Whole-graph link law: saturation (4 nearest neighbours for z = 6) pulls the
    accepted law away from the proposal law by a fixed, size-independent amount."""
    rho = 3.0
    fr = {}
    for L in (64, 128):
        ei, ej, _, _ = orc.levy_graph(L, 6, rho, 11)
        r2s = _r2_links(L, ei, ej)
        r2, p = _law_by_r2(L, rho)
        fr[L] = ((r2s <= 8).mean(), p[r2 <= 8].sum())
        print(f"L={L}: near-link fraction accepted {fr[L][0]:.4f}, law {fr[L][1]:.4f}")
    assert abs(fr[64][0] - fr[128][0]) < 0.02
    for L in fr:
        assert 0.0 < fr[L][1] - fr[L][0] < 0.1


# ---------------------------------------------------------------- colouring
def _proper(n, ei, ej, col):
    return np.all(col[np.asarray(ei)] != col[np.asarray(ej)]) and col.min() >= 0


def test_slo_hand_derived_colourings(orc):
    # path 0-1-2-3: removal 0,1,2,3 (min degree, smallest id); reverse greedy 3:0 2:1 1:0 0:1
    col, q = orc.slo_color(4, [0, 1, 2], [1, 2, 3])
    assert col.tolist() == [1, 0, 1, 0] and q == 2
    # triangle: removal 0,1,2; colours 2:0 1:1 0:2
    col, q = orc.slo_color(3, [0, 1, 0], [1, 2, 2])
    assert col.tolist() == [2, 1, 0] and q == 3
    # star with centre 0: removal 1,2,3,0,4; colours 4:0 0:1 3:0 2:0 1:0
    col, q = orc.slo_color(5, [0, 0, 0, 0], [1, 2, 3, 4])
    assert col.tolist() == [1, 0, 0, 0, 0] and q == 2
    # K4 needs 4 colours; removal 0,1,2,3 -> colours 3:0 2:1 1:2 0:3
    ei = [0, 0, 0, 1, 1, 2]
    ej = [1, 2, 3, 2, 3, 3]
    col, q = orc.slo_color(4, ei, ej)
    assert col.tolist() == [3, 2, 1, 0] and q == 4
    # isolated vertices take colour 0
    col, q = orc.slo_color(3, [], [])
    assert col.tolist() == [0, 0, 0] and q == 1


@pytest.mark.parametrize("L,rho", [(16, 3.5), (64, 2.5), (64, 4.5)])
def test_slo_proper_and_degeneracy_bound(orc, L, rho):
    nx = pytest.importorskip("networkx")
    ei, ej, _, _ = orc.levy_graph(L, 6, rho, 5)
    n = L * L
    col, q = orc.slo_color(n, ei, ej)
    assert _proper(n, ei, ej, col)
    assert q == col.max() + 1 and q <= 7
    G = nx.Graph()
    G.add_edges_from(zip(ei.tolist(), ej.tolist()))
    degeneracy = max(nx.core_number(G).values())
    assert q <= degeneracy + 1


def test_csr_layout(orc):
    L = 16
    ei, ej, _, _ = orc.levy_graph(L, 6, 3.5, 5)
    n = L * L
    col, q = orc.slo_color(n, ei, ej)
    perm, row_ptr, cidx, cptr = orc.csr(n, ei, ej, col, q)
    assert sorted(perm.tolist()) == list(range(n))
    inv = np.empty(n, np.int64)
    inv[perm] = np.arange(n)
    # classes contiguous, ascending original id inside a class
    for c in range(q):
        members = perm[cptr[c]:cptr[c + 1]]
        assert np.all(col[members] == c) and np.all(np.diff(members) > 0)
    assert cptr[0] == 0 and cptr[q] == n
    # rows sorted, symmetric, and equal to the original edges
    got = set()
    for a in range(n):
        row = cidx[row_ptr[a]:row_ptr[a + 1]]
        assert np.all(np.diff(row) > 0)
        for b in row.tolist():
            got.add((min(perm[a], perm[b]), max(perm[a], perm[b])))
    want = {(min(a, b), max(a, b)) for a, b in zip(ei.tolist(), ej.tolist())}
    assert got == want
