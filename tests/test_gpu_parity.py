"""GPU parity of libxyl's engines against the oracle and against exact results.

All calls go through the C ABI (ctypes binding).  Bars:
* FP64 engine vs oracle (53-bit uniforms): every angle within 1e-9 rad, labels
  identical, over the first 10 sweeps (C1, C2).
* FP32 engines vs oracle (24-bit uniforms): per-sweep energy per spin within
  1e-5 for every (replica, sweep) before that replica's trajectory separates;
  the first separation must follow a decision the oracle flags as a near tie
  (|u - exp(-beta dE)| < 1e-4), and at least half of all pairs are compared.
* long runs: <e>, chi, U4, <|m|>, chi(k_min) within 3 sigma (binned jackknife)
  of the oracle.
* kernels alone against the chain / ring / quadrature / beta = 0 exact results.
"""
import numpy as np
import pytest

from helpers import (ACC, bin_means, chain_closed_form, edges_chain, edges_complete, edges_ring, jackknife,
                     quadrature_moments, ring_mean_energy, run_bins)

pytestmark = pytest.mark.gpu

ALL = 1 | 2 | 4 | 8
NO_PT = 1 | 2 | 8
TIE_EPS = 1e-4


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need CUDA")
    from paper_1211_3991_gb300 import build
    build.build()
    from paper_1211_3991_gb300 import workloads, xyl
    xyl.load()
    return xyl, workloads


def _oracle_for(orc, wl, cfg, k, u24):
    L, rho, _ = cfg.graphs[k]
    ei, ej, _, _ = orc.levy_graph(L, 6, rho, wl.GRAPH_SEED, wl.graph_stream_id(cfg, k))
    color, _ = orc.slo_color(L * L, ei, ej)
    sim = orc.Sim(L * L, ei, ej, color, cfg.betas(), cfg.deltas(), wl.SPIN_SEED, sample=wl.sample_id(k),
                  xy=orc.lattice_xy(L), L=L, u24=u24)
    sim.set_tie_eps(TIE_EPS)
    sim.init()
    return sim


def _gpu_angles(plan, sample, R):
    return np.stack([np.arctan2(*plan.spins(sample, r)[:, ::-1].T) for r in range(R)])


def _angle_gap(a, b):
    return np.abs(np.angle(np.exp(1j * (a - b))))


def _rep_slice(plan, sample):
    off = sum(plan.n_temps[:sample])
    return slice(off, off + plan.n_temps[sample])


# --------------------------------------------------------------- FP64 engine
@pytest.mark.parametrize("name", ["C1", "C2"])
def test_fp64_trajectory_matches_oracle(env, orc, name):
    xyl, wl = env
    cfg = wl.config(name)
    plan, _ = wl.make_plan(cfg, xyl.FP64_PLAIN)
    plan.bind()
    plan.init_spins()
    sim = _oracle_for(orc, wl, cfg, 0, u24=False)
    R = cfg.n_temps
    assert _angle_gap(_gpu_angles(plan, 0, R), sim.angles()).max() < 1e-12
    for t in range(10):
        plan.sweep(1, ALL)
        sim.sweeps(1, ALL)
        gap = _angle_gap(_gpu_angles(plan, 0, R), sim.angles()).max()
        assert gap < 1e-9, (t, gap)
        assert np.array_equal(plan.labels(), sim.labels())
        np.testing.assert_allclose(plan.energies(), sim.energies(), rtol=1e-10, atol=1e-9)
    g, o = plan.read_observables(), sim.accumulators()
    np.testing.assert_allclose(g["acc"], o["acc"], rtol=1e-9, atol=1e-12)
    for key in ("met_acc", "met_try", "pt_acc", "pt_try"):
        assert np.array_equal(g[key], o[key]), key
    assert plan.status() == (0, 10)


# --------------------------------------------------------------- FP32 engines
def _fp32_compare(plan, sims, samples, n_sweeps, ops, N_of):
    """Per (sample, replica, sweep): energies agree before the trajectories part."""
    compared = total = 0
    first_split = {}
    for t in range(n_sweeps):
        plan.sweep(1, ops)
        E = plan.energies()
        for s in samples:
            sim = sims[s]
            sim.sweeps(1, ops)
            R = sim.R
            ang = _gpu_angles(plan, s, R)
            gap = _angle_gap(ang, sim.angles()).max(axis=1)
            Eg = E[_rep_slice(plan, s)]
            Eo = sim.energies()
            for r in range(R):
                total += 1
                key = (s, r)
                if key in first_split:
                    continue
                if gap[r] > 1e-3:
                    first_split[key] = t
                    continue
                compared += 1
                assert abs(Eg[r] - Eo[r]) / N_of(s) < 1e-5, (s, r, t, Eg[r], Eo[r])
    # the earliest separation of each sample follows a flagged near tie
    for s in samples:
        ties, pt_tie, _ = sims[s].ties()
        splits = [first_split[k] for k in first_split if k[0] == s]
        if splits:
            flagged = [x for x in list(ties) + [pt_tie] if x >= 0]
            assert flagged and min(flagged) <= min(splits), (s, min(splits), flagged)
    return compared, total


@pytest.mark.parametrize("engine_name", ["FP32_BATCHED", "FP32_PLAIN"])
@pytest.mark.parametrize("name", ["C1", "C2"])
def test_fp32_energy_matches_oracle(env, orc, name, engine_name):
    xyl, wl = env
    cfg = wl.config(name)
    plan, _ = wl.make_plan(cfg, getattr(xyl, engine_name))
    plan.bind()
    plan.init_spins()
    sims = {0: _oracle_for(orc, wl, cfg, 0, u24=True)}
    assert _angle_gap(_gpu_angles(plan, 0, cfg.n_temps), sims[0].angles()).max() < 1e-6
    compared, total = _fp32_compare(plan, sims, [0], 10, ALL, lambda s: cfg.graphs[s][0] ** 2)
    assert compared >= 0.5 * total, (compared, total)
    assert plan.status()[0] == 0


# --------------------------------------------------------------- long runs
@pytest.mark.parametrize("engine_name", ["FP32_BATCHED", "FP64_PLAIN"])
def test_long_run_statistics_c1(env, orc, engine_name):
    xyl, wl = env
    cfg = wl.config("C1")
    # Delta tuned on the oracle to about 50% acceptance, then frozen
    sim = _oracle_for(orc, wl, cfg, 0, u24=False)
    delta = np.array(cfg.deltas())
    for _ in range(6):
        sim.sweeps(200, NO_PT)
        st = sim.accumulators()
        rate = st["met_acc"][0] / st["met_try"][0]
        delta = np.clip(delta * rate / 0.5, 0.05, np.pi)
        sim.set_delta(delta)
        sim.reset_acc()
    cfg.delta = list(delta)
    sim = _oracle_for(orc, wl, cfg, 0, u24=False)
    plan, _ = wl.make_plan(cfg, getattr(xyl, engine_name))
    plan.bind()
    plan.init_spins()
    for s in (sim, plan):
        s.sweeps(500, NO_PT)
        s.reset_acc()
    ob = bin_means(run_bins(sim, 100, 100, NO_PT))[:, 0, :]
    gb = bin_means(run_bins(plan, 100, 100, NO_PT))[:, 0, :]
    N = 256
    fns = {
        "e": lambda m: m[ACC["e"]],
        "chi": lambda m: N * (m[ACC["m2"]] - m[ACC["mx"]] ** 2 - m[ACC["my"]] ** 2),
        "U4": lambda m: m[ACC["m4"]] / m[ACC["m2"]] ** 2 - 1,
        "absm": lambda m: m[ACC["absm"]],
        "chik": lambda m: m[ACC["chik"]],
    }
    for key, fn in fns.items():
        a, da = jackknife(ob, fn)
        b, db = jackknife(gb, fn)
        assert abs(a - b) < 3 * np.hypot(da, db), (key, a, da, b, db)
    st = plan.read_observables()
    rate = st["met_acc"][0] / st["met_try"][0]
    assert 0.35 < rate < 0.65


# --------------------------------------------------------------- exact results through the kernels
def _edge_plan(xyl, edges, n, betas, deltas, engine, xy=None, L=0, seed=5):
    g = xyl.graph_from_edges(n, edges, xy=xy, L=L)
    p = xyl.Plan([(g, 0, betas, deltas)], engine=engine, seed=seed)
    p.bind()
    p.init_spins()
    return p


ENGINES = ["FP32_BATCHED", "FP64_PLAIN", "FP32_PLAIN"]


@pytest.mark.parametrize("engine_name", ENGINES)
def test_chain_and_ring_closed_forms(env, engine_name):
    xyl, _ = env
    eng = getattr(xyl, engine_name)
    n, beta = 12, 1.0
    p = _edge_plan(xyl, edges_chain(n), n, [beta], [2.0], eng)
    p.sweeps(200, NO_PT)
    p.reset_acc()
    bins = bin_means(run_bins(p, 200, 200, NO_PT))[:, 0, :]
    _, mean_E, var_E = chain_closed_form(n, beta)
    e, de = jackknife(bins, lambda m: m[ACC["e"]])
    assert abs(e * n - mean_E) < 4 * de * n
    v, dv = jackknife(bins, lambda m: n * n * (m[ACC["e2"]] - m[ACC["e"]] ** 2))
    assert abs(v - var_E) < 4 * dv + 0.01 * var_E
    N, beta = 10, 1.5
    p = _edge_plan(xyl, edges_ring(N), N, [beta], [1.8], eng)
    p.sweeps(200, NO_PT)
    p.reset_acc()
    bins = bin_means(run_bins(p, 200, 200, NO_PT))[:, 0, :]
    e, de = jackknife(bins, lambda m: m[ACC["e"]])
    assert abs(e - ring_mean_energy(N, beta) / N) < 4 * de


XY4 = [0, 0, 1, 0, 0, 1, 1, 1]


@pytest.mark.parametrize("engine_name", ENGINES)
def test_small_graphs_and_pt_against_quadrature(env, engine_name):
    xyl, _ = env
    eng = getattr(xyl, engine_name)
    for n, edges in ((3, edges_ring(3)), (4, edges_complete(4))):
        beta = 1.3
        p = _edge_plan(xyl, edges, n, [beta], [2.5], eng, xy=XY4[: 2 * n], L=2)
        p.sweeps(100, NO_PT)
        p.reset_acc()
        bins = bin_means(run_bins(p, 100, 400, NO_PT))[:, 0, :]
        q = quadrature_moments(n, edges, beta, M=40 if n == 4 else 96, xy=XY4[: 2 * n], L=2)
        for key in ("e", "e2", "m2", "m4", "absm", "chik"):
            got, err = jackknife(bins, lambda m, k=key: m[ACC[k]])
            assert abs(got - q[key]) < 4.5 * err + 1e-6, (n, key, got, q[key], err)
    # three slots under parallel tempering: every slot samples its own beta
    betas = [0.5, 1.0, 1.6]
    p = _edge_plan(xyl, edges_ring(4), 4, betas, [3.0, 2.5, 2.0], eng, xy=XY4, L=2)
    p.sweeps(100, ALL)
    p.reset_acc()
    bins = bin_means(run_bins(p, 100, 400, ALL))
    for k, b in enumerate(betas):
        q = quadrature_moments(4, edges_ring(4), b, M=40)
        for key in ("e", "m2"):
            got, err = jackknife(bins[:, k, :], lambda m, kk=key: m[ACC[kk]])
            assert abs(got - q[key]) < 4.5 * err, (k, key, got, q[key])
    p.sweeps(20, ALL)
    st = p.read_observables()
    assert st["pt_try"][0] > 0 and 0 < st["pt_acc"][0] < st["pt_try"][0]
    assert sorted(p.labels().tolist()) == [0, 1, 2]


@pytest.mark.parametrize("engine_name", ENGINES)
def test_beta_zero_exact_moments(env, engine_name):
    xyl, _ = env
    L = 8
    N = L * L
    g = xyl.build_graph_csr(L, 6, 3.5, 1, 0)
    p = xyl.Plan([(g, 0, [0.0], [np.pi])], engine=getattr(xyl, engine_name), seed=9)
    p.bind()
    p.init_spins()
    bins = bin_means(run_bins(p, 100, 200, NO_PT))[:, 0, :]
    chi0, d0 = jackknife(bins, lambda m: N * m[ACC["m2"]])
    U4, dU = jackknife(bins, lambda m: m[ACC["m4"]] / m[ACC["m2"]] ** 2 - 1)
    chik, dk = jackknife(bins, lambda m: m[ACC["chik"]])
    e, de = jackknife(bins, lambda m: m[ACC["e"]])
    assert abs(chi0 - 1) < 4 * d0 and abs(U4 - (1 - 1 / N)) < 4 * dU
    assert abs(chik - 1) < 4 * dk and abs(e) < 4 * de
    p.sweeps(5, NO_PT)
    st = p.read_observables()
    assert st["met_acc"][0] == st["met_try"][0]


# --------------------------------------------------------------- full-size configurations
@pytest.mark.parametrize("name,sampled", [("C3", [0, 400, 767]), ("C4", [0, 47]), ("C5", [70])])
def test_full_size_batched_sampled_parity(env, orc, name, sampled):
    """Whole batch in the benchmark's launch configuration; sampled samples are
    re-run by the oracle from the same seeds; every sample obeys the invariants."""
    xyl, wl = env
    cfg = wl.config(name)
    plan, graphs = wl.make_plan(cfg, xyl.FP32_BATCHED)
    plan.bind()
    plan.init_spins()
    sims = {k: _oracle_for(orc, wl, cfg, k, u24=True) for k in sampled}
    n_sweeps = 2 if name == "C5" else 3
    compared, total = _fp32_compare(plan, sims, sampled, n_sweeps, ALL, lambda s: cfg.graphs[s][0] ** 2)
    assert compared >= 0.5 * total, (compared, total)
    status, t = plan.status()
    assert status == 0 and t == n_sweeps
    # invariants over the whole batch
    E = plan.energies()
    sizes = np.repeat([L * L for L, _, _ in cfg.graphs], cfg.n_temps)
    assert np.all(np.isfinite(E)) and np.all(np.abs(E) <= 3 * sizes)
    labels = plan.labels().reshape(cfg.n_samples, cfg.n_temps)
    assert all(sorted(row.tolist()) == list(range(cfg.n_temps)) for row in labels)
    st = plan.read_observables()
    rate = st["met_acc"] / np.maximum(st["met_try"], 1)
    assert np.all(st["met_try"] == n_sweeps * sizes) and np.all((rate > 0) & (rate < 1))
    assert np.all(st["acc"][:, ACC["n"]] == n_sweeps)
    plan.recompute()
    assert np.max(np.abs(plan.energies() - E) / sizes) < 1e-5


# --------------------------------------------------------------- determinism, checkpoint, recovery
def test_batched_runs_are_deterministic_and_resumable(env):
    xyl, wl = env
    cfg = wl.config("C2")
    graphs = wl.build_graphs(cfg)
    a, _ = wl.make_plan(cfg, xyl.FP32_BATCHED, graphs=graphs)
    b, _ = wl.make_plan(cfg, xyl.FP32_BATCHED, graphs=graphs)
    for p in (a, b):
        p.bind()
        p.init_spins()
        p.sweep(10, ALL)
    blob = a.export_state()
    a.sweep(15, ALL)
    b.import_state(blob)
    b.sweep(15, ALL)
    for r in range(cfg.n_temps):
        assert np.array_equal(a.spins(0, r), b.spins(0, r))
    assert np.array_equal(a.labels(), b.labels())
    ra, rb = a.read_observables(), b.read_observables()
    for k in ra:
        assert np.array_equal(ra[k], rb[k]), k
    assert a.status() == b.status() == (0, 25)


def test_recompute_bounds_fp32_drift(env):
    xyl, wl = env
    cfg = wl.config("C2")
    plan, _ = wl.make_plan(cfg, xyl.FP32_BATCHED, recompute_every=50)
    plan.bind()
    plan.init_spins()
    plan.sweep(200, ALL)
    E = plan.energies()
    plan.recompute()
    assert np.max(np.abs(plan.energies() - E)) / 16384 < 1e-5
    s = plan.spins(0, 3)
    assert np.max(np.abs(np.hypot(s[:, 0], s[:, 1]) - 1)) < 1e-6


def test_split_sample_wait_times_out_and_recovers(env):
    """Running one of a sample's replica groups alone makes its bounded wait for
    the other groups give up: status ETIMEOUT, context still usable."""
    xyl, wl = env
    cfg = wl.config("C2")
    plan, _ = wl.make_plan(cfg, xyl.FP32_BATCHED, group=4)
    plan.bind()
    plan.init_spins()
    assert plan.unit_count() == 4
    plan.sweep_units(0, 1, 3, ALL)
    status, _ = plan.status()
    assert status == xyl.ETIMEOUT
    with pytest.raises(xyl.XylError) as e:
        plan.energies()
    assert e.value.code == xyl.ETIMEOUT
    plan.init_spins()
    plan.sweep(5, ALL)
    assert plan.status() == (0, 5)
