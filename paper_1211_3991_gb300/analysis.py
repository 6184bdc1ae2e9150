"""Host analysis of the sampler's accumulators (numpy, no GPU).

The library returns, per (sample, temperature slot), FP64 sums over the
measurements of e = E/N, e^2, |m|, m_x, m_y, m^2, m^4, chi(k_min) and m_z
(O(3) spins; zero for XY) (xyl_read_observables, field order ``FIELDS``).  This module turns them into the
observables of Sec. III and the finite-size tools of Sec. IV and App. C:

* ``observables``: specific heat (Eq. specificheat), susceptibility (Eq. chi,
  connected, and N<m^2>), the per-sample cumulant, chi(k_min) and the
  second-moment correlation length xi_2 with psi = min(rho - d, 2);
* ``disorder_u4``: U4 = [<m^4>] / [<m^2>^2] - 1, [.] the average over graphs;
* ``jackknife``: leave-one-out errors over graphs (or bins);
* ``crossing``: where two curves sampled on a temperature grid cross;
* ``fit_tf``: T_f(N) = T_c + A N^-x through crossing temperatures (Eq. Tfsscaling);
* ``fit_nu_bar``: ln dU4/dT = c + (1/nu_bar) ln N at fixed U4 (Eq. scaling_lndotU4);
* ``exponential_windows`` / ``window_means``: time averages over windows
  [2^k, 2^(k+1)) of the measurement series, the paper's equilibration check;
* ``window_histogram_check``: the distributions of an observable over the last
  two exponential windows against each other (two-sample Kolmogorov-Smirnov);
* ``heat_capacity_check``: the specific heat from fluctuations against the
  temperature derivative of the energy, the paper's second equilibration check.
"""
from __future__ import annotations

import numpy as np

FIELDS = ("n", "e", "e2", "absm", "mx", "my", "m2", "m4", "chik", "mz")
_IX = {f: k for k, f in enumerate(FIELDS)}


def thermal_means(acc: np.ndarray) -> np.ndarray:
    """Accumulator sums (..., F) -> thermal averages (..., F); field 0 keeps the count."""
    acc = np.asarray(acc, np.float64)
    out = acc.copy()
    out[..., 1:] = acc[..., 1:] / acc[..., :1]
    return out


def observables(means: np.ndarray, N: int, T, L: int, rho: float | None = None, d: int = 2) -> dict:
    """Sec. III observables from thermal averages (..., F) of one graph size
    (F = 10 as the library returns them, or 9 without the m_z field).

    T broadcasts against the leading axes (e.g. one value per slot).  xi_2 takes
    psi = rho - d in the long-range regime and 2 in the short-range one, read as
    psi = min(rho - d, 2) (psi = 2 when rho is None)."""
    m = np.asarray(means, np.float64)
    g = lambda f: m[..., _IX[f]]
    T = np.asarray(T, np.float64)
    chi0 = N * g("m2")
    mz = g("mz") if m.shape[-1] > _IX["mz"] else 0.0
    chik = g("chik")
    psi = 2.0 if rho is None else min(rho - d, 2.0)
    ratio = np.maximum(chi0 / chik - 1.0, 0.0)
    return {
        "e": g("e"),
        "c": N * (g("e2") - g("e") ** 2) / T ** 2,
        "absm": g("absm"),
        "chi": N * (g("m2") - g("mx") ** 2 - g("my") ** 2 - mz ** 2),
        "chi0": chi0,
        "chik": chik,
        "u4_sample": g("m4") / g("m2") ** 2 - 1.0,
        "xi2": ratio ** (1.0 / psi) / (2.0 * np.sin(np.pi / L)),
    }


def disorder_u4(means: np.ndarray) -> np.ndarray:
    """U4 = [<m^4>] / [<m^2>^2] - 1 with [.] the average over axis 0 (graphs)."""
    m = np.asarray(means, np.float64)
    m2, m4 = m[..., _IX["m2"]], m[..., _IX["m4"]]
    return m4.mean(0) / (m2 ** 2).mean(0) - 1.0


def jackknife(data: np.ndarray, fn):
    """Leave-one-out over axis 0: returns (fn(all), error, leave-one-out values)."""
    data = np.asarray(data)
    n = data.shape[0]
    full = np.asarray(fn(data))
    loo = np.array([fn(np.delete(data, k, axis=0)) for k in range(n)])
    err = np.sqrt((n - 1) / n * ((loo - loo.mean(0)) ** 2).sum(0))
    return full, err, loo


def crossing(T, a, b) -> float:
    """First temperature where a - b changes sign, by linear interpolation (nan if none)."""
    T = np.asarray(T, np.float64)
    d = np.asarray(a, np.float64) - np.asarray(b, np.float64)
    for k in range(len(T) - 1):
        if d[k] == 0.0:
            return float(T[k])
        if d[k] * d[k + 1] < 0:
            return float(T[k] + (T[k + 1] - T[k]) * d[k] / (d[k] - d[k + 1]))
    return float("nan")


def fit_tf(N, t_cross, err=None):
    """Eq. Tfsscaling: T_f(N) = T_c + A N^-x, least squares over (T_c, A, x) on a
    grid of x with (T_c, A) linear at each x.  Returns (T_c, A, x)."""
    N = np.asarray(N, np.float64)
    t = np.asarray(t_cross, np.float64)
    w = np.ones_like(t) if err is None else 1.0 / np.asarray(err, np.float64) ** 2
    best = None
    for x in np.linspace(0.05, 2.0, 3901):
        X = np.stack([np.ones_like(N), N ** -x], 1)
        WX = X * w[:, None]
        coef = np.linalg.solve(X.T @ WX, WX.T @ t)
        r = float((w * (t - X @ coef) ** 2).sum())
        if best is None or r < best[0]:
            best = (r, coef[0], coef[1], x)
    return best[1], best[2], best[3]


def fit_nu_bar(N, dudt):
    """Eq. scaling_lndotU4: slope of ln dU4/dT against ln N is 1/nu_bar."""
    slope = np.polyfit(np.log(np.asarray(N, np.float64)), np.log(np.abs(np.asarray(dudt, np.float64))), 1)[0]
    return 1.0 / slope


def exponential_windows(n_meas: int):
    """Windows [2^k, 2^(k+1)) of measurement indices (k = 0, 1, ...) inside n_meas."""
    out, k = [], 0
    while 2 ** (k + 1) <= n_meas:
        out.append((2 ** k, 2 ** (k + 1)))
        k += 1
    return out


def window_means(series: np.ndarray, windows=None):
    """Means of a measurement series (axis 0 = time) over exponential windows, and
    whether the last two windows agree within three combined standard errors
    (the paper's equilibration check on time averages)."""
    s = np.asarray(series, np.float64)
    windows = windows or exponential_windows(len(s))
    means = np.array([s[a:b].mean(0) for a, b in windows])
    sems = np.array([s[a:b].std(0, ddof=1) / np.sqrt(b - a) if b - a > 1 else np.full(s.shape[1:], np.inf)
                     for a, b in windows])
    ok = bool(np.all(np.abs(means[-1] - means[-2]) < 3 * np.hypot(sems[-1], sems[-2]))) if len(windows) >= 2 else False
    return means, ok


def window_histogram_check(series, windows=None):
    """The equilibration check on distributions: the values of one observable
    in the last two exponential windows are compared by a two-sample
    Kolmogorov-Smirnov test (measurements far enough apart to be nearly
    independent, e.g. every 32 sweeps).  Returns (statistic, p-value)."""
    from scipy import stats
    s = np.asarray(series, np.float64)
    windows = windows or exponential_windows(len(s))
    if len(windows) < 2:
        raise ValueError("need at least two exponential windows")
    (a0, a1), (b0, b1) = windows[-2], windows[-1]
    res = stats.ks_2samp(s[a0:a1], s[b0:b1])
    return float(res.statistic), float(res.pvalue)


def heat_capacity_check(T, e, c):
    """Specific heat per spin from fluctuations, c = N var(e) / T^2, against
    d<e>/dT from the energy curve (second-order finite differences on the
    possibly non-uniform temperature grid).  In equilibrium the two agree, as
    d<E>/dT = var(E) / T^2.  Returns (d<e>/dT, relative difference)."""
    T = np.asarray(T, np.float64)
    dedT = np.gradient(np.asarray(e, np.float64), T)
    c = np.asarray(c, np.float64)
    return dedT, np.abs(dedT - c) / np.maximum(np.abs(c), 1e-300)
