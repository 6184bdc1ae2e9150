"""Pins of the oracle's M-bond Levy graphs (the paper's own ensemble, Sec. II).

Eq. (Levyi) with a fixed total of bonds: every bond is a pair of sites drawn with
probability proportional to |r_i - r_j|^-rho among all pairs of the lattice
(minimum image for periodic boundaries, plain distance inside the square for
free ones), pairs already bonded drawn again.  Checked against brute-force pair
counts of the lattice, the exact law of the first bond, and the exact
hypergeometric degree law of the uniform graph at rho = 0 (the Erdos-Renyi limit).
"""
import numpy as np
import pytest
from scipy import stats

from helpers import min_image_r2_counts


def _pairs_by_r2(L, fbc):
    """Brute force: number of ordered site pairs at each squared distance."""
    n = L * L
    x, y = np.arange(n) % L, np.arange(n) // L
    dx = np.abs(x[:, None] - x[None, :])
    dy = np.abs(y[:, None] - y[None, :])
    if not fbc:
        dx = np.minimum(dx, L - dx)
        dy = np.minimum(dy, L - dy)
    r2 = (dx ** 2 + dy ** 2).reshape(-1)
    r2 = r2[r2 > 0]
    vals, counts = np.unique(r2, return_counts=True)
    return vals, counts


def _bond_r2(L, ei, ej, fbc):
    dx = np.abs(ei % L - ej % L)
    dy = np.abs(ei // L - ej // L)
    if not fbc:
        dx = np.minimum(dx, L - dx)
        dy = np.minimum(dy, L - dy)
    return dx.astype(np.int64) ** 2 + dy.astype(np.int64) ** 2


def _chi2_p(obs, exp, min_exp=10.0):
    keep = exp >= min_exp
    o = np.append(obs[keep], obs[~keep].sum())
    e = np.append(exp[keep], exp[~keep].sum())
    if e[-1] == 0:
        o, e = o[:-1], e[:-1]
    return stats.chisquare(o, e * o.sum() / e.sum()).pvalue


@pytest.mark.parametrize("L", [2, 3, 8])
def test_fbc_table_brute_force(orc, L):
    dx, dy, B = orc.fbc_table(L, 2.5)
    want = {(a, b) for a in range(-(L - 1), L) for b in range(-(L - 1), L)} - {(0, 0)}
    assert len(dx) == len(want) and set(zip(dx.tolist(), dy.tolist())) == want
    # raster order (dy outer, dx inner)
    assert list(zip(dy.tolist(), dx.tolist())) == sorted(zip(dy.tolist(), dx.tolist()))
    # integer boundaries: entry widths proportional to r^-rho
    upper = np.append(B[1:].astype(object), 2 ** 64)
    width = np.array([float(u - b) for u, b in zip(upper, B.astype(object))])
    w = (dx.astype(float) ** 2 + dy.astype(float) ** 2) ** -1.25
    np.testing.assert_allclose(width / 2.0 ** 64, w / w.sum(), rtol=1e-9)
    assert B[0] == 0


@pytest.mark.parametrize("fbc", [False, True])
@pytest.mark.parametrize("L,rho", [(8, 0.0), (16, 2.5), (16, 4.5), (32, 3.5)])
def test_bonds_simple_counted_seeded(orc, L, rho, fbc):
    n = L * L
    ei, ej, attempts = orc.levy_bonds(L, rho, seed=5, sample=2, fbc=fbc)
    assert len(ei) == 2 * n and attempts >= 2 * n
    assert np.all(ei != ej) and np.all((ei >= 0) & (ei < n)) and np.all((ej >= 0) & (ej < n))
    key = np.minimum(ei, ej).astype(np.int64) * n + np.maximum(ei, ej)
    assert len(np.unique(key)) == len(key)
    deg = np.bincount(np.concatenate([ei, ej]), minlength=n)
    assert deg.sum() == 4 * n
    a2, b2, _ = orc.levy_bonds(L, rho, seed=5, sample=2, fbc=fbc)
    assert np.array_equal(a2, ei) and np.array_equal(b2, ej)
    a3, _, _ = orc.levy_bonds(L, rho, seed=5, sample=3, fbc=fbc)
    assert not np.array_equal(a3, ei)


def test_bond_count_limits(orc):
    n = 16
    ei, _, _ = orc.levy_bonds(4, 1.0, seed=1, n_bonds=0)
    assert len(ei) == 0
    # every pair of a 4 x 4 lattice: the complete graph
    ei, ej, _ = orc.levy_bonds(4, 1.0, seed=1, n_bonds=n * (n - 1) // 2)
    assert len(np.unique(np.minimum(ei, ej) * n + np.maximum(ei, ej))) == n * (n - 1) // 2
    with pytest.raises(ValueError):
        orc.levy_bonds(4, 1.0, seed=1, n_bonds=n * (n - 1) // 2 + 1)
    with pytest.raises(ValueError):
        orc.levy_bonds(5, 1.0, seed=1)          # periodic lattices need an even side
    orc.levy_bonds(5, 1.0, seed=1, fbc=True)     # free boundaries take any side


@pytest.mark.parametrize("fbc", [False, True])
@pytest.mark.parametrize("rho", [0.0, 2.5, 4.5])
def test_first_bond_law(orc, rho, fbc):
    """The first bond of a graph has no earlier bond to avoid, so over many
    independent streams it follows P({i,j}) ~ r_ij^-rho exactly: by squared
    distance (brute-force pair counts) and by site (uniform at rho = 0, edge
    effects of free boundaries otherwise)."""
    L, K = 8, 12000
    n = L * L
    first = np.array([orc.levy_bonds(L, rho, seed=11, sample=s, n_bonds=1, fbc=fbc)[:2] for s in range(K)])[:, :, 0]
    ei, ej = first[:, 0], first[:, 1]
    vals, counts = _pairs_by_r2(L, fbc)
    p = counts * vals.astype(float) ** (-rho / 2)
    r2 = _bond_r2(L, ei, ej, fbc)
    obs = np.array([(r2 == v).sum() for v in vals])
    assert obs.sum() == K
    assert _chi2_p(obs, p / p.sum() * K) > 1e-4
    # per site: P(site v is an endpoint) = sum over its partners of the pair law
    x, y = np.arange(n) % L, np.arange(n) // L
    dx = np.abs(x[:, None] - x[None, :])
    dy = np.abs(y[:, None] - y[None, :])
    if not fbc:
        dx, dy = np.minimum(dx, L - dx), np.minimum(dy, L - dy)
    w = np.where(dx + dy > 0, (dx ** 2 + dy ** 2 + (dx + dy == 0)).astype(float) ** (-rho / 2), 0.0)
    site_p = w.sum(1) / w.sum() * 2          # each bond has two endpoints
    ends = np.bincount(np.concatenate([ei, ej]), minlength=n)
    assert _chi2_p(ends, site_p * K) > 1e-4


@pytest.mark.parametrize("fbc", [False, True])
def test_uniform_graph_at_rho_zero(orc, fbc):
    """rho = 0: every pair equally likely and M = 2N pairs drawn without
    replacement, i.e. the uniform graph with M edges (the Erdos-Renyi limit of
    Sec. II).  A site's degree is then hypergeometric (the M bonds among the
    N(N-1)/2 pairs, N-1 of which contain the site) and the bond lengths follow
    the lattice's pair-distance counts, whatever the boundaries."""
    L = 32
    n = L * L
    degs, r2s = [], []
    for s in range(6):
        ei, ej, _ = orc.levy_bonds(L, 0.0, seed=21, sample=s, fbc=fbc)
        degs.append(np.bincount(np.concatenate([ei, ej]), minlength=n))
        r2s.append(_bond_r2(L, ei, ej, fbc))
    deg = np.concatenate(degs)
    hyper = stats.hypergeom(n * (n - 1) // 2, n - 1, 2 * n)
    kmax = deg.max() + 1
    obs = np.bincount(deg, minlength=kmax)
    exp = np.array([hyper.pmf(k) for k in range(kmax)]) * len(deg)
    assert _chi2_p(obs, exp) > 1e-4
    # Poisson(4) is the large-N limit the paper quotes
    assert abs(hyper.pmf(4) - stats.poisson(4).pmf(4)) < 2e-3
    vals, counts = _pairs_by_r2(L, fbc)
    r2 = np.concatenate(r2s)
    obs = np.array([(r2 == v).sum() for v in vals])
    assert _chi2_p(obs, counts / counts.sum() * len(r2)) > 1e-4


def test_pbc_table_is_the_pairing_table(orc):
    """Periodic bonds draw displacements from the same minimum-image table as
    the fixed-degree ensemble (each partner site once)."""
    dx, dy, B, _ = orc.disp_table(8, 3.0)
    assert len(dx) == 63
    r2 = dict(zip(*np.unique(dx.astype(np.int64) ** 2 + dy.astype(np.int64) ** 2, return_counts=True)))
    assert {int(k): int(v) for k, v in r2.items()} == min_image_r2_counts(8)
