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


# ----------------------------------------------------------------- FP32 parity from a shared state
FP32_TIE_EPS = 3e-5      # > 5x the worst FP32 error of exp(-beta dE) or of a PT exponent per decision
FP32_E_TOL = 1e-5        # energy per spin
FP32_DIR_TOL = 1e-4      # 99th percentile of the spin direction gaps (rad)
MAX_FLIPS = 3            # near-tie decisions forced together when tracing one replica-sweep


def direction_gap(a, b):
    """Angle between spin vectors a and b (..., d), d = 2 or 3, by atan2(|a x b|, a . b)."""
    dot = (a * b).sum(-1)
    if a.shape[-1] == 2:
        cross = np.abs(a[..., 0] * b[..., 1] - a[..., 1] * b[..., 0])
    else:
        cross = np.linalg.norm(np.cross(a, b), axis=-1)
    return np.arctan2(cross, dot)


def _replica_ok(gpu_vec, sim_vec, gpu_E, sim_E, N):
    gap = np.percentile(direction_gap(gpu_vec, sim_vec), 99)
    return abs(gpu_E - sim_E) / N < FP32_E_TOL and gap < FP32_DIR_TOL, abs(gpu_E - sim_E) / N


def fp32_parity_sweeps(plan, sims, samples, n_sweeps, ops, N_of, rep_slice):
    """FP32 kernel against the oracle in its 24-bit mode, one sweep at a time.

    Overrelaxation is chaotic (FP32 and FP64 trajectories decorrelate within
    about eight sweeps), so every sweep starts the oracle from the GPU's own
    spins, labels and sweep index, then both run one sweep.  Each replica must
    then agree: energy per spin within 1e-5 and 99% of spin directions within
    1e-4 rad (a site whose local field nearly cancels has an ill-conditioned
    reflection).  A replica that misses must be traced to decisions FP32
    rounding can flip: the oracle logs every Metropolis test within 3e-5 of
    flipping, and some set of at most three of that replica-sweep's logged
    decisions, forced the other way, must make the re-run oracle agree.  The
    slot labels must then agree too, with logged PT near-ties forced the same
    way where needed.  No other miss is allowed.

    Returns (replica-sweeps compared, misses traced, decisions flipped, worst
    |dE|/N among the agreeing ones)."""
    import itertools
    MET_OR = ops & 3
    compared = traced = flipped = 0
    worst = 0.0
    for _ in range(n_sweeps):
        t_gpu = plan.status()[1]
        labels = plan.labels()
        start = {}
        for s in samples:
            sim = sims[s]
            vec = np.stack([plan.spins(s, r) for r in range(sim.R)])
            start[s] = (vec, labels[rep_slice(s)].copy())
            sim.set_vectors(vec)
            sim.set_labels(start[s][1], t_gpu)
            sim.set_tie_eps(FP32_TIE_EPS)
            sim.clear_ties()
            sim.force([])
            sim.force_pt([])
            sim.set_active(None)
        plan.sweep(1, ops)
        E = plan.energies()
        labels_after = plan.labels()

        def restart(sim, s):
            sim.set_vectors(start[s][0])
            sim.set_labels(start[s][1], t_gpu)

        for s in samples:
            sim = sims[s]
            N = N_of(s)
            gvec = np.stack([plan.spins(s, r) for r in range(sim.R)])
            gE = E[rep_slice(s)]
            glab = labels_after[rep_slice(s)]
            sim.sweeps(1, ops)
            svec, sE = sim.vectors(), sim.energies()
            misses = []
            for r in range(sim.R):
                compared += 1
                ok, dE = _replica_ok(gvec[r], svec[r], gE[r], sE[r], N)
                if ok:
                    worst = max(worst, dE)
                else:
                    misses.append(r)
            if not misses and np.array_equal(glab, sim.labels()):
                continue
            log = sim.tie_log()
            pt_log = sim.tie_log(pt=True)
            forced = []
            for r in misses:
                cands = [(v, a) for rr, v, _, a in log if rr == r]
                found = None
                for size in range(1, min(len(cands), MAX_FLIPS) + 1):
                    for combo in itertools.combinations(cands, size):
                        restart(sim, s)
                        sim.set_active([r])
                        sim.force([(r, v, 1 - a) for v, a in combo])
                        sim.sweeps(1, MET_OR)
                        if _replica_ok(gvec[r], sim.vectors()[r], gE[r], sim.energies()[r], N)[0]:
                            found = combo
                            break
                    if found:
                        break
                assert found, f"sample {s} replica {r} sweep {t_gpu}: a miss not traced to near-tie decisions " \
                              f"({len(cands)} logged)"
                forced += [(r, v, 1 - a) for v, a in found]
                traced += 1
                flipped += len(found)
            # the whole sweep again with the traced decisions forced: every
            # replica agrees, and so do the labels (PT near-ties forced if needed)
            sim.set_active(None)
            pt_cands = [(k, a) for _, k, _, a in pt_log]
            ok_all = False
            for size in range(0, min(len(pt_cands), MAX_FLIPS) + 1):
                for combo in itertools.combinations(pt_cands, size):
                    restart(sim, s)
                    sim.force(forced)
                    sim.force_pt([(k, 1 - a) for k, a in combo])
                    sim.sweeps(1, ops)
                    same = all(_replica_ok(gvec[r], sim.vectors()[r], gE[r], sim.energies()[r], N)[0]
                               for r in range(sim.R))
                    if same and np.array_equal(glab, sim.labels()):
                        ok_all = True
                        flipped += size
                        break
                if ok_all:
                    break
            assert ok_all, f"sample {s} sweep {t_gpu}: labels or energies not traced to near-tie decisions"
            sim.force([])
            sim.force_pt([])
    return compared, traced, flipped, worst
