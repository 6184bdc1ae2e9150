"""Pins of the oracle's random bonds (H = -sum J_ij S_i.S_j, the paper's "random
bonds" variant of the method, App. B).

* Gauge invariance, exact: with tau_i = +-1, the couplings J'_ij = tau_i tau_j J_ij
  and spins S'_i = tau_i S_i describe the same system; every step of the sweep
  (local field, rotation, reflection, energy) maps term by term, so from the
  same random streams the two trajectories are negatives of each other on the
  tau = -1 sites bit for bit, with identical energies and PT labels.
* Frustrated small graphs against numerical quadrature (<e>, <e^2>, <m^2>).
* The fully frustrated triangle (all J = -1) orders at 120 degrees: e -> -1/2
  at low temperature (the ferromagnet's is -1).
"""
import numpy as np
import pytest

from helpers import ACC, bin_means, jackknife, quadrature_moments, run_bins

ALL = 1 | 2 | 4 | 8
NO_PT = 1 | 2 | 8


def _sim(orc, ei, ej, n, beta, delta, xy=None, L=None):
    return orc.graph_sim(np.asarray(ei, np.int32), np.asarray(ej, np.int32), n, beta, delta, 3, xy=xy, L=L)


@pytest.mark.parametrize("u24", [False, True])
def test_gauge_invariance_is_exact(orc, u24):
    L = 16
    n = L * L
    ei, ej, _, _ = orc.levy_graph(L, 6, 3.5, 1, 0)
    rng = np.random.default_rng(4)
    J = rng.choice([-1.0, 1.0], len(ei))
    tau = rng.choice([-1.0, 1.0], n)
    betas, deltas = [0.6, 0.9, 1.3], [2.0, 1.5, 1.0]
    sims = []
    for jj in (J, tau[ei] * tau[ej] * J):
        s = orc.graph_sim(ei, ej, n, betas, deltas, 7, xy=orc.lattice_xy(L), L=L, u24=u24)
        s.set_couplings(jj)
        s.init()
        sims.append(s)
    a, b = sims
    v = a.vectors()
    b.set_vectors(v * tau[None, :, None])
    np.testing.assert_array_equal(a.energies(), b.energies())
    for _ in range(12):
        a.sweeps(1, ALL)
        b.sweeps(1, ALL)
        np.testing.assert_array_equal(b.vectors(), a.vectors() * tau[None, :, None])
        np.testing.assert_array_equal(a.energies(), b.energies())
        np.testing.assert_array_equal(a.labels(), b.labels())
    # and the couplings do act: the ferromagnet's trajectory is different
    c = orc.graph_sim(ei, ej, n, betas, deltas, 7, xy=orc.lattice_xy(L), L=L, u24=u24)
    c.init()
    c.sweeps(12, ALL)
    assert not np.array_equal(c.vectors(), a.vectors())


FRUSTRATED = {
    "triangle_one_af": (3, [(0, 1), (1, 2), (2, 0)], [1.0, 1.0, -1.0]),
    "triangle_all_af": (3, [(0, 1), (1, 2), (2, 0)], [-1.0, -1.0, -1.0]),
    "ring4_mixed": (4, [(0, 1), (1, 2), (2, 3), (3, 0)], [1.0, -1.0, 1.0, 1.0]),
    "K4_mixed": (4, [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)], [1.0, -1.0, 1.0, -1.0, 1.0, 1.0]),
}


@pytest.mark.parametrize("name", sorted(FRUSTRATED))
def test_frustrated_small_graphs_against_quadrature(orc, name):
    n, edges, J = FRUSTRATED[name]
    beta = 1.6
    sim = _sim(orc, [a for a, _ in edges], [b for _, b in edges], n, [beta], [2.5])
    sim.set_couplings(J)
    sim.init()
    sim.sweeps(100, NO_PT)
    sim.reset_acc()
    bins = bin_means(run_bins(sim, 100, 200, NO_PT))
    q = quadrature_moments(n, edges, beta, M=40 if n == 4 else 96, couplings=J)
    for key in ("e", "e2", "m2"):
        got, err = jackknife(bins[:, 0, :], lambda m: m[ACC[key]])
        assert abs(got - q[key]) < 4.5 * err + 1e-9, (key, got, q[key], err)


def test_fully_frustrated_triangle_orders_at_120_degrees(orc):
    edges = [(0, 1), (1, 2), (2, 0)]
    ei, ej = [a for a, _ in edges], [b for _, b in edges]
    sim = _sim(orc, ei, ej, 3, [40.0], [0.3])
    sim.set_couplings([-1.0, -1.0, -1.0])
    sim.init()
    sim.sweeps(2000, NO_PT)
    sim.reset_acc()
    sim.sweeps(4000, NO_PT)
    e = sim.accumulators()["acc"][0, ACC["e"]] / sim.accumulators()["acc"][0, ACC["n"]]
    # ground state -1/2 per spin; harmonic fluctuations add about T/2 per spin (2 soft modes of 3 spins)
    assert -0.5 < e < -0.5 + 0.02
    sim.set_couplings(None)
    sim.init()
    sim.sweeps(2000, NO_PT)
    sim.reset_acc()
    sim.sweeps(4000, NO_PT)
    e = sim.accumulators()["acc"][0, ACC["e"]] / sim.accumulators()["acc"][0, ACC["n"]]
    assert -1.0 < e < -1.0 + 0.02
