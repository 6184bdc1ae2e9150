"""Pins of the oracle's O(3) spins (App. B: the method carries over to other
continuous models; O(3) is the paper's example).  None of them re-evaluates the
oracle's own formulas:

* Initial spins are uniform on the sphere: unit norm, z and the azimuth uniform
  (Archimedes), second moments I/3.
* The Metropolis proposal is uniform on the spherical cap of angular radius
  Delta: 1 - S.S' = u (1 - cos Delta) against numpy's cosine, unit norm for
  every azimuth, and an isotropic spread about S (equal second moments along
  two orthogonal axes perpendicular to S).
* Trees, exactly: each bond variable J_b S_i.S_j is independent with density
  proportional to exp(beta y) on [-1, 1] (mean coth(beta) - 1/beta, the
  Langevin function), and <S_i.S_j> is the product of J_b L(beta) along the
  path; this gives <e>, <e^2> and <m^2>.
* Rings, exactly: expanding each bond weight in Legendre polynomials,
  exp(t x) = sum_l (2l+1) i_l(t) P_l(x) (modified spherical Bessel i_l), the
  normalised partition function of a ring is sum_l (2l+1) prod_b i_l(beta J_b),
  and <E>, <E^2> follow from its beta derivatives; one frustrated ring.
* beta = 0: <m^2> = 1/N and <m^4> = (N^2 + 2N(N-1)/3) / N^4 for independent
  uniform unit 3-vectors (the XY value would be 2N(N-1)/2 in the second term).
* Overrelaxation alone conserves the energy; gauge invariance is exact.
* Random fields (3-vectors): a spin without links follows the Langevin law
  <S> = L(beta|h|) h/|h|; a bond with fields against quadrature over one spin
  with the other integrated out exactly (itself checked by brute-force
  sampling); overrelaxation still conserves the energy.
"""
import numpy as np
import pytest
from scipy import special, stats

from helpers import ACC, bin_means, jackknife, run_bins

ALL = 1 | 2 | 4 | 8
NO_PT = 1 | 2 | 8


def _langevin(beta):
    return 1.0 / np.tanh(beta) - 1.0 / beta


def _second(beta):
    # <y^2> for density exp(beta y) on [-1, 1]: variance + mean^2
    return 1.0 / beta ** 2 - 1.0 / np.sinh(beta) ** 2 + _langevin(beta) ** 2


@pytest.mark.parametrize("u24", [False, True])
def test_initial_spins_are_uniform_on_the_sphere(orc, u24):
    n = 20000
    sim = orc.graph_sim(np.zeros(0, np.int32), np.zeros(0, np.int32), n, [1.0, 1.0], [1.0, 1.0], 5, u24=u24, dim=3)
    sim.init()
    v = sim.vectors().reshape(-1, 3)
    assert np.abs(np.linalg.norm(v, axis=1) - 1.0).max() < 1e-15
    assert stats.kstest(v[:, 2], stats.uniform(-1, 2).cdf).pvalue > 1e-3
    phi = np.arctan2(v[:, 1], v[:, 0])
    assert stats.kstest(phi, stats.uniform(-np.pi, 2 * np.pi).cdf).pvalue > 1e-3
    np.testing.assert_allclose(v.T @ v / len(v), np.eye(3) / 3, atol=0.01)
    sim.init(aligned=True)
    assert np.array_equal(sim.vectors().reshape(-1, 3), np.tile([1.0, 0.0, 0.0], (2 * n, 1)))


@pytest.mark.parametrize("delta", [0.3, 1.7, np.pi])
def test_cap_proposal_is_uniform_on_the_cap(orc, delta):
    rng = np.random.default_rng(3)
    for s in [np.array([0.0, 0.0, 1.0]), np.array([0.0, 0.0, -1.0]), np.array([1.0, 0.0, 0.0]),
              rng.normal(size=3)]:
        s = s / np.linalg.norm(s)
        u, uphi = rng.random(4000), rng.random(4000)
        p = np.array([orc.o3_propose(s, delta, a, b) for a, b in zip(u, uphi)])
        assert np.abs(np.linalg.norm(p, axis=1) - 1.0).max() < 1e-14
        np.testing.assert_allclose(1.0 - p @ s, u * (1.0 - np.cos(delta)), atol=2e-15)
        # spread about s is isotropic: two orthogonal directions perpendicular to s
        a = np.cross(s, [0.3, 0.5, 0.7])
        a /= np.linalg.norm(a)
        b = np.cross(s, a)
        var_a, var_b = ((p @ a) ** 2).mean(), ((p @ b) ** 2).mean()
        sin2 = 1.0 - (1.0 - u * (1.0 - np.cos(delta))) ** 2
        assert abs(var_a - sin2.mean() / 2) < 0.05 * sin2.mean() + 1e-3
        assert abs(var_b - sin2.mean() / 2) < 0.05 * sin2.mean() + 1e-3
        assert abs((p @ a).mean()) < 4 * np.sqrt(var_a / len(p)) + 1e-12


def _random_tree(n, rng):
    return [(int(rng.integers(0, i)), i) for i in range(1, n)]


@pytest.mark.parametrize("signs", [False, True])
def test_tree_moments_are_exact(orc, signs):
    rng = np.random.default_rng(11 + signs)
    n, beta = 10, 1.2
    edges = _random_tree(n, rng)
    J = rng.choice([-1.0, 1.0], len(edges)) if signs else np.ones(len(edges))
    sim = orc.graph_sim([a for a, _ in edges], [b for _, b in edges], n, [beta], [2.2], 9, dim=3)
    if signs:
        sim.set_couplings(J)
    sim.init()
    sim.sweeps(200, NO_PT)
    sim.reset_acc()
    bins = bin_means(run_bins(sim, 100, 400, NO_PT))
    Lb, y2 = _langevin(beta), _second(beta)
    nb = n - 1
    e = -nb * Lb / n
    e2 = (nb * y2 + nb * (nb - 1) * Lb ** 2) / n ** 2
    # <S_i.S_j> = product of J_b L(beta) along the tree path
    adj = {i: [] for i in range(n)}
    for (a, b), j in zip(edges, J):
        adj[a].append((b, j))
        adj[b].append((a, j))
    corr = np.zeros((n, n))
    for i in range(n):
        stack, seen = [(i, 1.0)], {i}
        while stack:
            v, c = stack.pop()
            corr[i, v] = c
            for w, j in adj[v]:
                if w not in seen:
                    seen.add(w)
                    stack.append((w, c * j * Lb))
    m2 = corr.sum() / n ** 2
    for key, want in (("e", e), ("e2", e2), ("m2", m2)):
        got, err = jackknife(bins[:, 0, :], lambda m: m[ACC[key]])
        assert abs(got - want) < 4.5 * err + 1e-9, (key, got, want, err)


def _ring_moments(J, beta, lmax=40):
    """<E>, <E^2> of an O(3) ring with couplings J (E = -sum J_b S_b.S_b+1)."""
    Z = Z1 = Z2 = 0.0
    for l in range(lmax):
        f = np.array([special.spherical_in(l, beta * j) for j in J])
        x = beta * np.asarray(J)
        fp = np.array([special.spherical_in(l, xi, derivative=True) for xi in x]) * np.asarray(J)
        # i_l'' from x^2 i'' + 2 x i' - (x^2 + l(l+1)) i = 0, times J^2 = 1
        ip = fp * np.asarray(J)
        fpp = f * (1.0 + l * (l + 1) / x ** 2) - 2.0 * ip / x
        w = 2 * l + 1
        Z += w * np.prod(f)
        s1 = s2 = 0.0
        for b in range(len(J)):
            rest = np.prod(np.delete(f, b))
            s1 += fp[b] * rest
            s2 += fpp[b] * rest
            for c in range(len(J)):
                if c != b:
                    s2 += fp[b] * fp[c] * np.prod(np.delete(f, [b, c]))
        Z1 += w * s1
        Z2 += w * s2
    return -Z1 / Z, Z2 / Z


def test_ring_closed_form_against_brute_force_sampling():
    """The ring formula itself against plain importance sampling of 3 spins."""
    rng = np.random.default_rng(0)
    J, beta = [1.0, -1.0, 1.0], 0.9
    v = rng.normal(size=(400000, 3, 3))
    v /= np.linalg.norm(v, axis=2, keepdims=True)
    E = -sum(J[b] * (v[:, b] * v[:, (b + 1) % 3]).sum(1) for b in range(3))
    w = np.exp(-beta * E)
    e1, e2 = _ring_moments(J, beta)
    assert abs((w * E).sum() / w.sum() - e1) < 0.01
    assert abs((w * E * E).sum() / w.sum() - e2) < 0.02


@pytest.mark.parametrize("J", [[1.0] * 5, [1.0, -1.0, 1.0, 1.0, 1.0]])
def test_ring_moments_are_exact(orc, J):
    n, beta = len(J), 1.1
    ei, ej = list(range(n)), [(i + 1) % n for i in range(n)]
    sim = orc.graph_sim(ei, ej, n, [beta], [2.0], 4, dim=3)
    sim.set_couplings(J)
    sim.init()
    sim.sweeps(200, NO_PT)
    sim.reset_acc()
    bins = bin_means(run_bins(sim, 100, 400, NO_PT))
    E1, E2 = _ring_moments(J, beta)
    for key, want in (("e", E1 / n), ("e2", E2 / n ** 2)):
        got, err = jackknife(bins[:, 0, :], lambda m: m[ACC[key]])
        assert abs(got - want) < 4.5 * err + 1e-9, (key, got, want, err)


def test_infinite_temperature_cumulant(orc):
    L = 6
    n = L * L
    ei, ej, _, _ = orc.levy_graph(L, 4, 3.0, 1, 0)
    sim = orc.graph_sim(ei, ej, n, [0.0], [np.pi], 2, xy=orc.lattice_xy(L), L=L, dim=3)
    sim.init()
    sim.sweeps(10, NO_PT)
    sim.reset_acc()
    bins = bin_means(run_bins(sim, 50, 400, NO_PT))
    m2, m2e = jackknife(bins[:, 0, :], lambda m: m[ACC["m2"]])
    m4, m4e = jackknife(bins[:, 0, :], lambda m: m[ACC["m4"]])
    assert abs(m2 - 1.0 / n) < 4.5 * m2e
    assert abs(m4 - (n * n + 2 * n * (n - 1) / 3) / n ** 4) < 4.5 * m4e
    # every proposal is accepted at beta = 0
    st = sim.accumulators()
    assert np.array_equal(st["met_acc"], st["met_try"])


def test_overrelaxation_conserves_energy(orc):
    L = 16
    ei, ej, _, _ = orc.levy_graph(L, 6, 3.5, 1, 0)
    sim = orc.graph_sim(ei, ej, L * L, [0.7, 1.3], [1.0, 1.0], 6, dim=3)
    sim.set_couplings(np.random.default_rng(2).choice([-1.0, 1.0], len(ei)))
    sim.init()
    sim.sweeps(5, 1)
    E0 = sim.energies().copy()
    v0 = sim.vectors().copy()
    sim.sweeps(20, 2)
    np.testing.assert_allclose(sim.energies(), E0, rtol=1e-12)
    assert np.abs(sim.vectors() - v0).max() > 0.1
    assert np.abs(np.linalg.norm(sim.vectors(), axis=2) - 1.0).max() < 1e-12


def test_gauge_invariance_is_exact(orc):
    L = 16
    n = L * L
    ei, ej, _, _ = orc.levy_graph(L, 6, 3.5, 1, 0)
    rng = np.random.default_rng(5)
    J = rng.choice([-1.0, 1.0], len(ei))
    tau = rng.choice([-1.0, 1.0], n)
    sims = []
    for jj in (J, tau[ei] * tau[ej] * J):
        s = orc.graph_sim(ei, ej, n, [0.6, 0.9, 1.3], [2.0, 1.5, 1.0], 7, xy=orc.lattice_xy(L), L=L, dim=3)
        s.set_couplings(jj)
        s.init()
        sims.append(s)
    a, b = sims
    b.set_vectors(a.vectors() * tau[None, :, None])
    for _ in range(8):
        a.sweeps(1, ALL)
        b.sweeps(1, ALL)
        np.testing.assert_array_equal(b.vectors(), a.vectors() * tau[None, :, None])
        np.testing.assert_array_equal(a.energies(), b.energies())
        np.testing.assert_array_equal(a.labels(), b.labels())


def test_fields_keep_the_spins_component_count(orc):
    sim = orc.graph_sim([0], [1], 2, [1.0], [1.0], 1, dim=3)
    with pytest.raises(ValueError):
        sim.set_fields(np.ones((2, 2)))
    xy = orc.graph_sim([0], [1], 2, [1.0], [1.0], 1)
    with pytest.raises(ValueError):
        xy.set_fields(np.ones((2, 3)))
    with pytest.raises(ValueError):
        orc.graph_sim([0], [1], 2, [1.0], [1.0], 1, dim=4)


def _unit(v):
    v = np.asarray(v, np.float64)
    return v / np.linalg.norm(v, axis=-1, keepdims=True)


def test_free_spins_in_fields_follow_the_langevin_law(orc):
    """A spin with no links in a field h: <S> = L(beta|h|) h/|h| and its energy
    -|h| L(beta|h|), L(x) = coth x - 1/x (one-spin partition function
    4 pi sinh(beta|h|) / (beta|h|)); field directions with all three components."""
    n, beta = 6, 1.3
    mags = np.array([0.2, 0.5, 1.0, 1.5, 2.5, 4.0])
    dirs = _unit(np.random.default_rng(4).normal(size=(n, 3)))
    h = mags[:, None] * dirs
    sim = orc.graph_sim(np.zeros(0, np.int32), np.zeros(0, np.int32), n, [beta], [np.pi], 5, dim=3)
    sim.set_fields(h)
    sim.init()
    sim.sweeps(200, NO_PT)
    sim.reset_acc()
    bins = bin_means(run_bins(sim, 100, 400, NO_PT))
    Lh = _langevin(beta * mags)
    want = {"e": -(mags * Lh).sum() / n}
    for a, key in enumerate(("mx", "my", "mz")):
        want[key] = (Lh * dirs[:, a]).sum() / n
    for key, w in want.items():
        got, err = jackknife(bins[:, 0, :], lambda m: m[ACC[key]])
        assert abs(got - w) < 4.5 * err + 1e-9, (key, got, w, err)


def _bond_with_fields(J, h1, h2, beta, M=64):
    """<e>, <e^2>, <m_x>, <m_z> of two O(3) spins, H = -J S1.S2 - h1.S1 - h2.S2.
    S2 is integrated out exactly: given S1 it has density ~ exp(beta a.S2),
    a = J S1 + h2, so <a.S2> = |a| L(beta|a|) and <(a.S2)^2> = |a|^2 y2(beta|a|);
    S1 runs over a Gauss-Legendre (cos theta) x periodic (phi) grid."""
    x, wx = np.polynomial.legendre.leggauss(M)
    phi = 2 * np.pi * np.arange(2 * M) / (2 * M)
    ct, ph = np.meshgrid(x, phi, indexing="ij")
    st = np.sqrt(1 - ct ** 2)
    S1 = np.stack([st * np.cos(ph), st * np.sin(ph), ct], -1)
    wq = wx[:, None] * np.ones_like(ph)
    b = S1 @ np.asarray(h1)
    a = J * S1 + np.asarray(h2)
    A = np.linalg.norm(a, axis=-1)
    # log of exp(beta b) sinh(beta A) / (beta A), kept finite
    logw = beta * b + beta * A + np.log1p(-np.exp(-2 * beta * A)) - np.log(2 * beta * A)
    w = wq * np.exp(logw - logw.max())
    LA, y2 = _langevin(beta * A), _second(beta * A)
    E = -(b + A * LA)
    E2 = b ** 2 + 2 * b * A * LA + A ** 2 * y2
    S2 = LA[..., None] * a / A[..., None]
    m = 0.5 * (S1 + S2)
    Z = w.sum()
    return {"e": (w * E).sum() / Z / 2, "e2": (w * E2).sum() / Z / 4, "mx": (w * m[..., 0]).sum() / Z,
            "mz": (w * m[..., 2]).sum() / Z}


def test_bond_integration_against_brute_force_sampling():
    """The bond quadrature itself against plain importance sampling."""
    rng = np.random.default_rng(1)
    J, h1, h2, beta = -1.0, [0.3, -0.8, 0.5], [0.9, 0.2, -0.4], 1.1
    v = _unit(rng.normal(size=(1000000, 2, 3)))
    E = -(J * (v[:, 0] * v[:, 1]).sum(1) + v[:, 0] @ np.array(h1) + v[:, 1] @ np.array(h2))
    w = np.exp(-beta * E)
    q = _bond_with_fields(J, h1, h2, beta)
    assert abs((w * E).sum() / w.sum() / 2 - q["e"]) < 0.003
    assert abs((w * E * E).sum() / w.sum() / 4 - q["e2"]) < 0.006
    assert abs((w * (v[:, 0, 2] + v[:, 1, 2]) / 2).sum() / w.sum() - q["mz"]) < 0.003


@pytest.mark.parametrize("J", [1.0, -1.0])
def test_bond_with_fields_against_quadrature(orc, J):
    h1, h2, beta = [0.3, -0.8, 0.5], [0.9, 0.2, -0.4], 1.1
    sim = orc.graph_sim([0], [1], 2, [beta], [2.5], 8, dim=3)
    sim.set_couplings([J])
    sim.set_fields(np.array([h1, h2]))
    sim.init()
    sim.sweeps(100, NO_PT)
    sim.reset_acc()
    bins = bin_means(run_bins(sim, 100, 400, NO_PT))
    q = _bond_with_fields(J, h1, h2, beta)
    for key in ("e", "e2", "mx", "mz"):
        got, err = jackknife(bins[:, 0, :], lambda m: m[ACC[key]])
        assert abs(got - q[key]) < 4.5 * err + 1e-9, (key, got, q[key], err)


def test_overrelaxation_with_fields_conserves_energy(orc):
    L = 16
    ei, ej, _, _ = orc.levy_graph(L, 6, 3.5, 1, 0)
    sim = orc.graph_sim(ei, ej, L * L, [0.7, 1.3], [1.0, 1.0], 6, dim=3)
    sim.set_fields(0.5 * _unit(np.random.default_rng(3).normal(size=(L * L, 3))))
    sim.init()
    sim.sweeps(5, 1)
    E0 = sim.energies().copy()
    sim.sweeps(20, 2)
    np.testing.assert_allclose(sim.energies(), E0, rtol=1e-12)
