"""Test-side statistics and exact references (no method code from either side).

* ``jackknife``: delete-one-bin jackknife over bins of measurements.
* ``quadrature_moments``: exact thermal moments of an n <= 4 spin XY system by the
  periodic trapezoid rule over relative angles (spectrally convergent for the
  smooth periodic Boltzmann weight), used to pin both samplers.
* ``bessel_*``: closed forms of the open chain and the periodic ring.
* ``paper_critical_temperatures``: the paper's printed T_c table (tests/golden).
"""
from __future__ import annotations

import itertools

import numpy as np
from scipy import special

ACC = {k: i for i, k in enumerate(("n", "e", "e2", "absm", "mx", "my", "m2", "m4", "chik", "mz"))}


def jackknife(bins: np.ndarray, fn):
    """bins: (B, ...) per-bin means; fn: function of the mean -> scalar."""
    bins = np.asarray(bins, dtype=np.float64)
    B = bins.shape[0]
    total = bins.sum(0)
    full = fn(total / B)
    loo = np.array([fn((total - bins[b]) / (B - 1)) for b in range(B)])
    err = np.sqrt((B - 1) / B * ((loo - loo.mean()) ** 2).sum())
    return float(full), float(err)


def bin_means(acc_bins: np.ndarray) -> np.ndarray:
    """(B, R, 9) accumulator sums -> (B, R, 9) per-bin means (column 0 keeps counts)."""
    acc_bins = np.asarray(acc_bins, dtype=np.float64)
    out = acc_bins.copy()
    out[..., 1:] = acc_bins[..., 1:] / acc_bins[..., :1]
    return out


def derived(mean_row: np.ndarray, N: int, T: float, L: int):
    """Sec. III observables from one slot's mean accumulator row."""
    e, e2, m2, m4 = mean_row[ACC["e"]], mean_row[ACC["e2"]], mean_row[ACC["m2"]], mean_row[ACC["m4"]]
    mx, my, chik = mean_row[ACC["mx"]], mean_row[ACC["my"]], mean_row[ACC["chik"]]
    return {
        "e": e,
        "c": N * (e2 - e * e) / T ** 2,
        "chi_conn": N * (m2 - mx * mx - my * my),
        "chi0": N * m2,
        "U4": m4 / m2 ** 2 - 1.0,
        "chik": chik,
        "absm": mean_row[ACC["absm"]],
    }


def run_bins(sim, n_bins: int, bin_sweeps: int, ops: int, measure_every: int = 1):
    """Run a sampler (oracle or library, same method names) in bins; returns (B, R, 9)."""
    out = []
    for _ in range(n_bins):
        sim.sweeps(bin_sweeps, ops, measure_every)
        out.append(sim.accumulators()["acc"].copy())
        sim.reset_acc()
    return np.array(out)


def quadrature_moments(n, edges, beta, M=48, xy=None, L=None, couplings=None, fields=None):
    """Exact <e>, <e^2>, <m^2>, <m^4>, <|m|>, <m_x>, <chi(k_min)> for n <= 4 spins.

    Without fields fix theta_0 = 0 (all quantities are rotation invariant) and
    integrate the other n-1 angles on an M-point periodic grid; with fields
    (n x 2 vectors, energy -sum h_i . S_i) integrate all n angles."""
    grid = 2 * np.pi * np.arange(M) / M - np.pi
    if fields is None:
        mesh = np.meshgrid(*([grid] * (n - 1)), indexing="ij")
        th = [np.zeros_like(mesh[0])] + list(mesh)
    else:
        th = list(np.meshgrid(*([grid] * n), indexing="ij"))
    E = np.zeros_like(th[0])
    J = [1.0] * len(edges) if couplings is None else list(couplings)
    for (i, j), c in zip(edges, J):
        E -= c * np.cos(th[i] - th[j])
    if fields is not None:
        for i in range(n):
            E -= fields[i][0] * np.cos(th[i]) + fields[i][1] * np.sin(th[i])
    w = np.exp(-beta * (E - E.min()))
    Z = w.sum()
    mx = sum(np.cos(t) for t in th) / n
    my = sum(np.sin(t) for t in th) / n
    m2 = mx * mx + my * my
    e = E / n
    out = {
        "e": (w * e).sum() / Z,
        "e2": (w * e * e).sum() / Z,
        "m2": (w * m2).sum() / Z,
        "m4": (w * m2 * m2).sum() / Z,
        "absm": (w * np.sqrt(m2)).sum() / Z,
        "mx": (w * mx).sum() / Z,
    }
    if xy is not None:
        xs = [xy[2 * v] for v in range(n)]
        ys = [xy[2 * v + 1] for v in range(n)]
        tot = 0
        for pos in (xs, ys):
            ph = [np.exp(2j * np.pi * p / L) for p in pos]
            fx = sum(np.cos(th[v]) * ph[v] for v in range(n))
            fy = sum(np.sin(th[v]) * ph[v] for v in range(n))
            tot = tot + np.abs(fx) ** 2 + np.abs(fy) ** 2
        out["chik"] = (w * tot).sum() / Z / (2 * n)
    return out


def chain_closed_form(n: int, beta: float):
    """Open chain of n spins: bond angles are independent with weight e^{beta cos}."""
    i0, i1, i2 = special.iv(0, beta), special.iv(1, beta), special.iv(2, beta)
    t = i1 / i0
    mean_E = -(n - 1) * t
    var_E = (n - 1) * ((1 + i2 / i0) / 2 - t * t)
    return t, mean_E, var_E


def ring_mean_energy(N: int, beta: float, kmax: int = 60):
    """Periodic ring: Z ~ sum_k I_k^N, <E> = -N sum_k I_k^{N-1} I_k' / sum_k I_k^N."""
    ks = np.arange(-kmax, kmax + 1)
    Ik = special.ive(ks, beta)              # scaled by e^{-beta}; ratios unaffected
    dIk = 0.5 * (special.ive(ks - 1, beta) + special.ive(ks + 1, beta))
    num = (Ik ** (N - 1) * dIk).sum()
    den = (Ik ** N).sum()
    return -N * num / den


def count_cycles_3_4(n, row_ptr, col):
    """Triangles and 4-cycles of a simple graph given as CSR (brute force)."""
    nb = [set(col[row_ptr[v]:row_ptr[v + 1]].tolist()) for v in range(n)]
    n3 = 0
    for v in range(n):
        for a in nb[v]:
            if a > v:
                n3 += len([b for b in nb[v] & nb[a] if b > a])
    n4 = 0
    for i in range(n):
        for k in range(i + 1, n):
            c = len(nb[i] & nb[k])
            n4 += c * (c - 1) // 2
    return n3, n4 // 2


def min_image_r2_counts(L: int):
    """Brute-force multiset of minimum-image squared distances from one site."""
    xs = np.arange(L)
    d = np.minimum(xs, L - xs)
    r2 = (d[:, None] ** 2 + d[None, :] ** 2).reshape(-1)
    r2 = r2[r2 > 0]
    vals, counts = np.unique(r2, return_counts=True)
    return dict(zip(vals.tolist(), counts.tolist()))


def edges_ring(n):
    return [(i, (i + 1) % n) for i in range(n)]


def edges_chain(n):
    return [(i, i + 1) for i in range(n - 1)]


def edges_complete(n):
    return list(itertools.combinations(range(n), 2))


def paper_critical_temperatures():
    """The paper's Table criticalexponents (T_c from T_f and from U crosses, by
    rho) and the analytic Erdos-Renyi T_c of Sec. IV, from
    tests/golden/critical_temperatures.txt."""
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "critical_temperatures.txt")
    rows, analytic = {}, None
    for line in open(path):
        line = line.split("#")[0].strip()
        if not line:
            continue
        w = line.split()
        if w[0] == "analytic_er":
            analytic = float(w[1])
            continue
        rows[float(w[0])] = tuple(float(x) for x in w[1:5])
    return rows, analytic
