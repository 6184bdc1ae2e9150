"""GPU random walks (spectral dimension, App. A) against the oracle.

Walks are integer work: the return histograms of the kernel and of the
sequential oracle must be identical, count for count, on the same CSR, seed and
starting nodes.  On the square lattice the self-return probability decays as
tau^-1 (spectral dimension 2, Eq. (eqbard) for rho > d + 2).
"""
import numpy as np
import pytest

from test_oracle_walk import csr_of, torus_edges

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need CUDA")
    from paper_1211_3991_gb300 import build
    build.build()
    from paper_1211_3991_gb300 import workloads, xyl
    xyl.load()
    return torch, xyl, workloads


def _gpu_returns(torch, xyl, row_ptr, col, start, n_steps, seed, first_walker=0):
    dev = torch.device("cuda")
    rp = torch.from_numpy(np.ascontiguousarray(row_ptr, np.int32)).to(dev)
    cl = torch.from_numpy(np.ascontiguousarray(col, np.int32)).to(dev)
    st = torch.from_numpy(np.ascontiguousarray(start, np.int32)).to(dev)
    out = torch.empty(n_steps + 1, dtype=torch.int64, device=dev)
    xyl.walk_returns(rp, cl, st, n_steps, seed, out, first_walker=first_walker)
    return out.cpu().numpy().astype(np.uint64)


def _oracle_csr(orc, L, rho, sample, fbc=False):
    ei, ej, _ = orc.levy_bonds(L, rho, 1, sample, fbc=fbc)
    col, q = orc.slo_color(L * L, ei, ej)
    _, row_ptr, c, _ = orc.csr(L * L, ei, ej, col, q)
    return row_ptr, c


@pytest.mark.parametrize("case", ["bonds_rho0", "bonds_fbc", "fixed_degree", "torus"])
def test_walk_histograms_identical_to_oracle(env, orc, case):
    torch, xyl, wl = env
    rng = np.random.default_rng(7)
    if case == "torus":
        row_ptr, col = csr_of(64 * 64, torus_edges(64))
        start, T = rng.integers(0, 64 * 64, 20000, dtype=np.int32), 300
    elif case == "fixed_degree":
        g = xyl.build_graph_csr(128, 6, 3.5, 1, 0)
        _, row_ptr, col, _ = g.csr()
        ei, ej, _, _ = orc.levy_graph(128, 6, 3.5, 1, 0)
        c, q = orc.slo_color(128 * 128, ei, ej)
        _, orp, ocol, _ = orc.csr(128 * 128, ei, ej, c, q)
        assert np.array_equal(orp, row_ptr) and np.array_equal(ocol, col)
        start, T = rng.integers(0, 128 * 128, 30000, dtype=np.int32), 200
    else:
        fbc = case == "bonds_fbc"
        L, rho = (16, 0.0) if not fbc else (32, 10.0 / 3.0)
        g = xyl.build_levy_bonds(L, rho, 1, 4, fbc=fbc)
        _, row_ptr, col, _ = g.csr()
        orp, ocol = _oracle_csr(orc, L, rho, 4, fbc)
        assert np.array_equal(orp, row_ptr) and np.array_equal(ocol, col)
        start, T = np.repeat(np.arange(L * L, dtype=np.int32), 8), 500
    want = orc.walk_returns(row_ptr, col, start, T, seed=33)
    got = _gpu_returns(torch, xyl, row_ptr, col, start, T, 33)
    assert np.array_equal(got, want)
    assert got[0] == len(start)


def test_walkers_in_pieces_and_invalid_starts(env, orc):
    torch, xyl, _ = env
    row_ptr, col = csr_of(32 * 32, torus_edges(32))
    start = np.arange(1000, dtype=np.int32) % 1024
    whole = _gpu_returns(torch, xyl, row_ptr, col, start, 120, 5)
    a = _gpu_returns(torch, xyl, row_ptr, col, start[:371], 120, 5)
    b = _gpu_returns(torch, xyl, row_ptr, col, start[371:], 120, 5, first_walker=371)
    assert np.array_equal(a + b, whole)
    # starts outside the graph are left out: the oracle on the valid ones, same stream ids
    bad = start.copy()
    bad[[3, 500]] = [-1, 1024]
    got = _gpu_returns(torch, xyl, row_ptr, col, bad, 120, 5)
    assert got[0] == 998
    keep = np.ones(1000, bool)
    keep[[3, 500]] = False
    ref = np.zeros(121, np.uint64)
    for w in np.flatnonzero(keep):
        ref += _gpu_returns(torch, xyl, row_ptr, col, start[w:w + 1], 120, 5, first_walker=int(w))
    assert np.array_equal(got, ref)


def test_square_lattice_spectral_dimension(env):
    """P(tau) ~ tau^(-dbar/2) with dbar = 2 on the square lattice (times well
    below L, so the walk does not feel the torus)."""
    torch, xyl, _ = env
    L, W, T = 512, 1 << 17, 2000
    row_ptr, col = csr_of(L * L, torus_edges(L))
    start = np.random.default_rng(1).integers(0, L * L, W, dtype=np.int32)
    got = _gpu_returns(torch, xyl, row_ptr, col, start, T, 11).astype(np.float64)
    assert np.all(got[1::2] == 0)
    tau = np.arange(100, T + 1, 2)
    slope = np.polyfit(np.log(tau), np.log(got[tau] / W), 1)[0]
    assert abs(-2 * slope - 2.0) < 0.05, slope
