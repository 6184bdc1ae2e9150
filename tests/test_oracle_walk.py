"""Pins of the oracle's random walks (spectral dimension, App. A).

The walk's self-return probability after t steps from node s is exactly
(P^t)_ss, P = D^-1 A the transition matrix, so on small graphs every count is
binomial around a known probability (and exactly zero where a return is
impossible).  On the square lattice the return probability after 2n < L steps is
the closed form [C(2n, n) / 4^n]^2, odd returns never happen (the lattice is
bipartite), and the decay t^-1 is the spectral dimension 2.
"""
import numpy as np
import pytest
from scipy.special import comb


def csr_of(n, edges):
    adj = [[] for _ in range(n)]
    for a, b in edges:
        adj[a].append(b)
        adj[b].append(a)
    row_ptr = np.zeros(n + 1, np.int32)
    row_ptr[1:] = np.cumsum([len(a) for a in adj])
    col = np.array([j for a in adj for j in a], np.int32)
    return row_ptr, col


def torus_edges(L):
    e = []
    for y in range(L):
        for x in range(L):
            i = x + L * y
            e.append((i, (x + 1) % L + L * y))
            e.append((i, x + L * ((y + 1) % L)))
    return e


def exact_returns(n, edges, s, T):
    A = np.zeros((n, n))
    for a, b in edges:
        A[a, b] = A[b, a] = 1.0
    deg = A.sum(1)
    P = np.where(deg[:, None] > 0, A / np.maximum(deg, 1)[:, None], np.eye(n))
    out, v = [], np.eye(n)[s]
    for _ in range(T + 1):
        out.append(v[s])
        v = v @ P
    return np.array(out)


SMALL = {
    "ring7": (7, [(i, (i + 1) % 7) for i in range(7)], 0),
    "K4": (4, [(a, b) for a in range(4) for b in range(a + 1, 4)], 2),
    "star_leaf": (6, [(0, k) for k in range(1, 6)], 3),
    "irregular": (6, [(0, 1), (1, 2), (2, 0), (2, 3), (3, 4), (4, 5), (5, 3), (1, 4)], 5),
}


@pytest.mark.parametrize("name", sorted(SMALL))
def test_return_counts_match_transition_matrix_powers(orc, name):
    n, edges, s = SMALL[name]
    W, T = 200_000, 14
    row_ptr, col = csr_of(n, edges)
    got = orc.walk_returns(row_ptr, col, np.full(W, s, np.int32), T, seed=17).astype(np.float64)
    p = exact_returns(n, edges, s, T)
    assert got[0] == W
    for t in range(1, T + 1):
        if p[t] == 0.0:
            assert got[t] == 0, (t, got[t])
        else:
            z = (got[t] - W * p[t]) / np.sqrt(W * p[t] * (1 - p[t]) + 1e-300)
            assert abs(z) < 5.0, (name, t, got[t] / W, p[t], z)


def test_square_lattice_closed_form_and_no_odd_returns(orc):
    L, W, T = 32, 200_000, 30
    row_ptr, col = csr_of(L * L, torus_edges(L))
    rng = np.random.default_rng(3)
    got = orc.walk_returns(row_ptr, col, rng.integers(0, L * L, W, dtype=np.int32), T, seed=5).astype(np.float64)
    assert np.all(got[1::2] == 0)
    for n2 in range(2, T + 1, 2):
        p = (comb(n2, n2 // 2, exact=True) / 2.0 ** n2) ** 2   # [C(2n, n) / 4^n]^2 with 2n = n2
        z = (got[n2] - W * p) / np.sqrt(W * p * (1 - p))
        assert abs(z) < 5.0, (n2, got[n2] / W, p)


def test_isolated_start_and_seeding(orc):
    row_ptr, col = csr_of(3, [(0, 1)])
    got = orc.walk_returns(row_ptr, col, np.array([2, 2, 0], np.int32), 9, seed=1)
    # the two walkers on the isolated node return at every step; the one on the
    # edge returns at every even step
    assert list(got) == [3, 2, 3, 2, 3, 2, 3, 2, 3, 2]
    r2, c2 = csr_of(64, torus_edges(8))
    st = np.arange(64, dtype=np.int32)
    a = orc.walk_returns(r2, c2, st, 40, seed=9)
    assert np.array_equal(a, orc.walk_returns(r2, c2, st, 40, seed=9))
    assert not np.array_equal(a, orc.walk_returns(r2, c2, st, 40, seed=10))
    with pytest.raises(ValueError):
        orc.walk_returns(r2, c2, np.array([64], np.int32), 4, seed=1)


def test_large_rho_bond_ensemble_is_the_square_lattice(orc):
    """rho -> infinity: every proposal is a nearest-neighbour pair, so the 2N
    distinct bonds are the 2N links of the periodic square lattice."""
    L = 16
    ei, ej, _ = orc.levy_bonds(L, 200.0, seed=2, sample=0)
    got = {tuple(sorted(p)) for p in zip(ei.tolist(), ej.tolist())}
    want = {tuple(sorted(p)) for p in torus_edges(L)}
    assert got == want
