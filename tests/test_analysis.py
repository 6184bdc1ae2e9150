"""Host analysis layer (paper_1211_3991_gb300.analysis) against exact cases.

Sec. III observables from accumulator sums: a Gaussian two-component
magnetisation has <m^4> = 2 <m^2>^2 (U4 = 1), an ordered one U4 = 0 and chi = 0;
an Ornstein-Zernike chi(k) gives back its xi_2 exactly for any psi; the
specific heat is N var(e) / T^2.  FSS tools: known crossings, the power laws of
Eqs. Tfsscaling and scaling_lndotU4, jackknife = standard error for a mean,
exponential windows.
"""
import numpy as np
import pytest

from paper_1211_3991_gb300 import analysis as an


def _acc_from_samples(e, mx, my, chik):
    m2 = mx ** 2 + my ** 2
    rows = [len(e), e.sum(), (e ** 2).sum(), np.sqrt(m2).sum(), mx.sum(), my.sum(), m2.sum(), (m2 ** 2).sum(),
            chik.sum()]
    return np.array(rows, np.float64)


def test_gaussian_and_ordered_cumulants():
    rng = np.random.default_rng(0)
    n = 1_000_000
    N, T, L = 1024, 1.5, 32
    e = rng.normal(-1.2, 0.03, n)
    mx, my = rng.normal(0, 0.1, n), rng.normal(0, 0.1, n)
    obs = an.observables(an.thermal_means(_acc_from_samples(e, mx, my, np.full(n, 2.0))), N, T, L)
    assert abs(obs["u4_sample"] - 1.0) < 0.01
    assert abs(obs["c"] - N * 0.03 ** 2 / T ** 2) / (N * 0.03 ** 2 / T ** 2) < 0.01
    assert abs(obs["chi0"] - N * 0.02) / (N * 0.02) < 0.01
    # ordered: |m| fixed, direction fixed -> U4 = 0, connected chi = 0
    k = np.ones(1000)
    obs = an.observables(an.thermal_means(_acc_from_samples(-2.0 * k, 0.6 * k, 0.8 * k, k)), N, T, L)
    assert abs(obs["u4_sample"]) < 1e-12 and abs(obs["chi"]) < 1e-9 and abs(obs["chi0"] - N) < 1e-9
    assert obs["c"] == pytest.approx(0.0, abs=1e-9)


@pytest.mark.parametrize("rho,psi", [(None, 2.0), (3.5, 1.5), (5.0, 2.0)])
def test_xi2_of_ornstein_zernike(rho, psi):
    L, N, xi = 64, 4096, 7.3
    kh = 2 * np.sin(np.pi / L)
    chi0 = 250.0
    chik = chi0 / (1.0 + (kh * xi) ** psi)
    means = np.zeros(9)
    means[0] = 1
    means[6] = chi0 / N
    means[8] = chik
    assert an.observables(means, N, 1.0, L, rho=rho)["xi2"] == pytest.approx(xi, rel=1e-12)


def test_disorder_u4_is_a_ratio_of_graph_averages():
    means = np.zeros((2, 3, 9))
    a, b = np.array([0.2, 0.3, 0.4]), np.array([0.1, 0.5, 0.2])
    means[0, :, 6], means[1, :, 6] = a, b
    means[0, :, 7], means[1, :, 7] = 2 * a ** 2, 2 * b ** 2
    np.testing.assert_allclose(an.disorder_u4(means), 1.0, rtol=1e-14)
    means[1, :, 7] = b ** 2
    np.testing.assert_allclose(an.disorder_u4(means), (2 * a ** 2 + b ** 2) / (a ** 2 + b ** 2) - 1, rtol=1e-14)


def test_jackknife_of_a_mean_is_the_standard_error():
    x = np.random.default_rng(1).normal(size=(50, 3))
    full, err, loo = an.jackknife(x, lambda d: d.mean(0))
    np.testing.assert_allclose(full, x.mean(0))
    np.testing.assert_allclose(err, x.std(0, ddof=1) / np.sqrt(50), rtol=1e-12)
    assert loo.shape == (50, 3)


def test_crossing_and_fss_fits():
    T = np.linspace(1.0, 2.0, 11)
    assert an.crossing(T, T - 1.55, 2 * (T - 1.55)) == pytest.approx(1.55, abs=1e-12)
    assert np.isnan(an.crossing(T, T, T + 1))
    N = np.array([16, 32, 64, 128, 256]) ** 2.0
    tc, A, x = an.fit_tf(N, 1.9 + 0.5 * N ** -0.5)
    assert tc == pytest.approx(1.9, abs=1e-4) and x == pytest.approx(0.5, abs=1e-3) and A == pytest.approx(0.5, rel=1e-2)
    assert an.fit_nu_bar(N, 3.0 * N ** 0.5) == pytest.approx(2.0, rel=1e-12)


def test_exponential_windows_and_equilibration_check():
    assert an.exponential_windows(100) == [(1, 2), (2, 4), (4, 8), (8, 16), (16, 32), (32, 64)]
    rng = np.random.default_rng(2)
    _, ok = an.window_means(rng.normal(size=4096))
    assert ok
    _, ok = an.window_means(rng.normal(size=4096) + np.linspace(0, 5, 4096))
    assert not ok


def test_heat_capacity_check_on_the_xy_dimer():
    """Two XY spins, one bond: e = -I1(b)/I0(b) / 2 per spin, and
    var(E) = <cos^2> - <cos>^2 with <cos^2> = (1 + I2/I0) / 2 (Bessel), so
    c = N var(e) / T^2 = var(E) / (2 T^2) must equal de/dT."""
    from scipy.special import iv
    T = np.geomspace(0.5, 3.0, 400)
    b = 1.0 / T
    m1 = iv(1, b) / iv(0, b)
    m2 = 0.5 * (1.0 + iv(2, b) / iv(0, b))
    e = -0.5 * m1
    c = (m2 - m1 ** 2) / (2.0 * T ** 2)
    dedT, rel = an.heat_capacity_check(T, e, c)
    assert rel[2:-2].max() < 1e-3
    # an energy curve off by a temperature-dependent factor fails it
    _, rel_bad = an.heat_capacity_check(T, e * (1 + 0.2 * T), c)
    assert rel_bad[2:-2].max() > 0.05


def test_window_histograms_of_a_stationary_and_a_drifting_series():
    rng = np.random.default_rng(5)
    x = rng.standard_cauchy(4096)  # heavy tails: a distribution check, not a moment check
    _, p = an.window_histogram_check(x)
    assert p > 1e-3
    # same mean, wider spread in the last window: the means agree, the histograms do not
    y = x.copy()
    y[2048:] *= 3.0
    _, p = an.window_histogram_check(y)
    assert p < 1e-6
    with pytest.raises(ValueError):
        an.window_histogram_check(np.ones(3))


def test_connected_susceptibility_takes_m_z_for_o3():
    # an ordered O(3) state along z: m = (0, 0, 1), so chi = N(<m^2> - |<m>|^2) = 0
    means = np.zeros(10)
    means[0] = 1
    means[6] = 1.0   # m^2
    means[9] = 1.0   # m_z
    means[8] = 1.0   # chi(k_min)
    assert an.observables(means, 64, 1.0, 8)["chi"] == pytest.approx(0.0, abs=1e-12)
    # without the m_z field (XY accumulators) the same m^2 is all fluctuation
    assert an.observables(means[:9], 64, 1.0, 8)["chi"] == pytest.approx(64.0)
