"""Critical temperature of the paper's Erdos-Renyi limit through the GPU engine.

At rho = 0 the paper's ensemble (2N bonds, Sec. II) is the uniform random graph
with mean degree 4, and the paper locates its transition (Sec. IV, Erdos-Renyi
limit; Table criticalexponents) at T_c = 1.93(1) from the crossing of
U4(T, N) with U4(T, N/4), in agreement with the analytic 1.9361.  For Poisson
degrees of mean c the mean excess degree is also c, and the tree (cavity)
instability of the XY model sits where c I1(beta)/I0(beta) = 1; that closed
form is pinned here against the printed value, then the crossing of the
disorder-averaged cumulant (Sec. III: U4 = [<m^4>] / [<m^2>^2] - 1, [.] the
average over graphs of the thermal averages) between L = 32 and L = 64 from the
FP32 batched engine is compared with it.
"""
import numpy as np
import pytest
from scipy.optimize import brentq
from scipy.special import iv

from helpers import paper_critical_temperatures


def cavity_tc(c=4.0):
    beta = brentq(lambda b: c * iv(1, b) / iv(0, b) - 1.0, 1e-3, 10.0)
    return 1.0 / beta


def test_cavity_temperature_is_the_papers_analytic_value():
    table, analytic = paper_critical_temperatures()
    assert abs(cavity_tc(4.0) - analytic) < 5e-5
    # and the paper's own crossing estimate at rho = 0 agrees with it
    tc_u, err_u = table[0.0][2], table[0.0][3]
    assert abs(tc_u - analytic) < err_u
    # large c: I1/I0 ~ beta/2, so T_c -> c/2 (the Gaussian mean-field value 2 at c = 4 is above it)
    assert abs(cavity_tc(400.0) - 200.0) / 200.0 < 1e-2


def _u4_curves(xyl, wl, L, n_samples, temps, warm, meas):
    cfg = wl.Config(f"ER{L}", [(L, 0.0, s) for s in range(n_samples)], temps, ensemble="bonds")
    plan, graphs = wl.make_plan(cfg, xyl.FP32_BATCHED)
    assert max(g.max_deg for g in graphs) > 8
    plan.bind()
    plan.init_spins()
    plan.sweep(warm, 15, 8)
    plan.reset_observables()
    plan.sweep(meas, 15, 8)
    assert plan.status() == (0, warm + meas)
    acc = plan.read_observables()["acc"].reshape(n_samples, len(temps), -1)
    m2 = acc[..., 6] / acc[..., 0]
    m4 = acc[..., 7] / acc[..., 0]
    idx = np.arange(n_samples)

    def u4(keep):
        return m4[keep].mean(0) / (m2[keep] ** 2).mean(0) - 1.0

    return u4(idx), np.array([u4(np.delete(idx, k)) for k in idx])


def _crossing(temps, d):
    for k in range(len(temps) - 1):
        if d[k] * d[k + 1] < 0:
            return temps[k] + (temps[k + 1] - temps[k]) * d[k] / (d[k] - d[k + 1])
    return np.nan


@pytest.mark.gpu
def test_u4_crossing_at_rho_zero_matches_analytic_tc():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need CUDA")
    from paper_1211_3991_gb300 import build
    build.build()
    from paper_1211_3991_gb300 import workloads as wl, xyl
    xyl.load()
    S = 64
    temps = wl.geometric_temperatures(1.7, 2.2, 12)
    u_a, loo_a = _u4_curves(xyl, wl, 32, S, temps, 2000, 8000)
    u_b, loo_b = _u4_curves(xyl, wl, 64, S, temps, 2000, 8000)
    # cumulant rises from 0 (ordered) towards 1 (two-component paramagnet)
    assert u_b[0] < 0.1 and u_b[-1] > 0.9 and np.all(np.diff(u_b) > -0.02)
    t_x = _crossing(temps, u_a - u_b)
    loo = np.array([_crossing(temps, a - b) for a, b in zip(loo_a, loo_b)])
    err = np.sqrt((S - 1) / S * np.nansum((loo - np.nanmean(loo)) ** 2))
    tc = cavity_tc(4.0)
    table, _ = paper_critical_temperatures()
    print(f"U4 crossing L=32/64: {t_x:.4f} +- {err:.4f} (analytic {tc:.4f}, paper {table[0.0][2]}({table[0.0][3]}))")
    assert np.isfinite(t_x) and err < 0.02
    # 3 sigma plus 0.01 for the finite-size shift of the crossing (O(N^-1/2) with nu_bar = 2)
    assert abs(t_x - tc) < 3 * err + 0.01, (t_x, err, tc)
    assert abs(t_x - table[0.0][2]) < 3 * err + table[0.0][3] + 0.01
