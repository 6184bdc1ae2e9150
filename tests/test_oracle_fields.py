"""Pins of the oracle's random fields (H = -sum J_ij S_i.S_j - sum h_i.S_i, the
paper's "random fields" variant of the method, App. B).

* A spin with no links in a field h: <S . h/|h|> = I1(beta|h|) / I0(beta|h|),
  its energy -|h| I1/I0 (exact, one-spin partition function 2 pi I0(beta|h|)).
* Small graphs with bonds, couplings and fields against quadrature over all
  angles (the field breaks rotation invariance).
"""
import numpy as np
import pytest
from scipy.special import iv

from helpers import ACC, bin_means, jackknife, quadrature_moments, run_bins

NO_PT = 1 | 2 | 8


def test_free_spins_follow_the_bessel_law(orc):
    n, beta = 6, 1.3
    mags = np.array([0.2, 0.5, 1.0, 1.5, 2.5, 4.0])
    ang = np.linspace(0.3, 5.9, n)
    h = np.stack([mags * np.cos(ang), mags * np.sin(ang)], 1)
    sim = orc.graph_sim(np.zeros(0, np.int32), np.zeros(0, np.int32), n, [beta], [np.pi], 5)
    sim.set_fields(h)
    sim.init()
    sim.sweeps(200, NO_PT)
    sim.reset_acc()
    bins = bin_means(run_bins(sim, 100, 400, NO_PT))
    t = iv(1, beta * mags) / iv(0, beta * mags)
    e_exact = -(mags * t).sum() / n
    mx_exact = (t * np.cos(ang)).sum() / n
    my_exact = (t * np.sin(ang)).sum() / n
    for key, want in (("e", e_exact), ("mx", mx_exact), ("my", my_exact)):
        got, err = jackknife(bins[:, 0, :], lambda m: m[ACC[key]])
        assert abs(got - want) < 4.5 * err + 1e-9, (key, got, want, err)


CASES = {
    "edge_fields": (2, [(0, 1)], [1.0], [(0.8, 0.0), (0.0, -0.5)]),
    "edge_af_field": (2, [(0, 1)], [-1.0], [(1.2, 0.4), (0.0, 0.0)]),
    "triangle_fields": (3, [(0, 1), (1, 2), (2, 0)], [1.0, -1.0, 1.0], [(0.3, 0.9), (-0.7, 0.2), (0.1, -0.4)]),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_small_graphs_with_fields_against_quadrature(orc, name):
    n, edges, J, h = CASES[name]
    beta = 1.4
    ei = np.array([a for a, _ in edges], np.int32)
    ej = np.array([b for _, b in edges], np.int32)
    sim = orc.graph_sim(ei, ej, n, [beta], [2.5], 3)
    sim.set_couplings(J)
    sim.set_fields(np.array(h, np.float64))
    sim.init()
    sim.sweeps(100, NO_PT)
    sim.reset_acc()
    bins = bin_means(run_bins(sim, 100, 200, NO_PT))
    q = quadrature_moments(n, edges, beta, M=96 if n == 2 else 48, couplings=J, fields=h)
    for key in ("e", "e2", "m2", "mx"):
        got, err = jackknife(bins[:, 0, :], lambda m: m[ACC[key]])
        assert abs(got - q[key]) < 4.5 * err + 1e-9, (key, got, q[key], err)
