"""GPU parity of libxyl's engines against the oracle and against exact results.

All calls go through the C ABI (ctypes binding).  Bars:
* FP64 engine vs oracle (53-bit uniforms): every angle within 1e-9 rad, labels
  identical, over the first 10 sweeps (C1, C2).
* FP32 engines vs oracle (24-bit uniforms): overrelaxation is chaotic (FP32 vs
  FP64 trajectories decorrelate within about eight sweeps), so every sweep
  starts the oracle from the GPU's own spins and labels; energy per spin then
  agrees within 1e-5 and 99% of angles within 1e-4 rad for every (replica,
  sweep).  A replica-sweep that misses must be traced to decisions FP32
  rounding can flip: forcing at most three of the oracle's logged near-tie
  decisions of that replica-sweep (|u - exp(-beta dE)| < 3e-5) the other way
  must reproduce the GPU's result; no untraced miss is allowed.
* long runs: <e>, chi, U4, <|m|>, chi(k_min) within 3 sigma (binned jackknife)
  of the oracle.
* kernels alone against the chain / ring / quadrature / beta = 0 exact results.
"""
import numpy as np
import pytest

from helpers import (ACC, bin_means, chain_closed_form, edges_chain, edges_complete, edges_ring, fp32_parity_sweeps,
                     jackknife, quadrature_moments, ring_mean_energy, run_bins)

pytestmark = pytest.mark.gpu

ALL = 1 | 2 | 4 | 8
NO_PT = 1 | 2 | 8


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


def _oracle_graph(orc, wl, cfg, k):
    L, rho, _ = cfg.graphs[k]
    if cfg.ensemble == "bonds":
        ei, ej, _ = orc.levy_bonds(L, rho, wl.GRAPH_SEED, wl.graph_stream_id(cfg, k), fbc=cfg.boundary == "fbc")
        return ei, ej
    ei, ej, _, _ = orc.levy_graph(L, 6, rho, wl.GRAPH_SEED, wl.graph_stream_id(cfg, k))
    return ei, ej


def _oracle_for(orc, wl, cfg, k, u24):
    L, rho, _ = cfg.graphs[k]
    ei, ej = _oracle_graph(orc, wl, cfg, k)
    color, _ = orc.slo_color(L * L, ei, ej)
    sim = orc.Sim(L * L, ei, ej, color, cfg.betas(), cfg.deltas(), wl.SPIN_SEED, sample=wl.graph_stream_id(cfg, k),
                  xy=orc.lattice_xy(L), L=L, u24=u24)
    sim.init()
    return sim


def _gpu_angles(plan, sample, R):
    return np.stack([np.arctan2(*plan.spins(sample, r)[:, ::-1].T) for r in range(R)])


def _angle_gap(a, b):
    return np.abs(np.angle(np.exp(1j * (a - b))))


def _rep_slice(plan, sample):
    off = sum(plan.n_temps[:sample])
    return slice(off, off + plan.n_temps[sample])


# engine name -> (engine constant, plan options); the FP32 batched engine runs in
# its resident shape (spins in shared memory) and its global-memory shape
VARIANTS = {
    "FP32_RESIDENT": ("FP32_BATCHED", {"resident": 1}),
    "FP32_SPLIT": ("FP32_BATCHED", {"resident": 1, "cluster": 4}),
    "FP32_GLOBAL": ("FP32_BATCHED", {"resident": -1}),
    "FP32_PLAIN": ("FP32_PLAIN", {}),
    # the launch shape the benchmark's autotuner picks at C2
    "FP32_BENCH": ("FP32_BATCHED", {"resident": 1, "group": 1, "cluster": 6, "block": 512}),
    "FP64_PLAIN": ("FP64_PLAIN", {}),
}


def _variant(xyl, name):
    eng, opts = VARIANTS[name]
    return getattr(xyl, eng), dict(opts)


# --------------------------------------------------------------- FP64 engine
@pytest.mark.parametrize("name", ["C1", "C2", "E1", "E2"])
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
def _fp32_per_sweep(plan, sims, samples, n_sweeps, ops, N_of):
    """Per-sweep FP32 parity from a shared state; every miss traced to flipped
    near-tie decisions (helpers.fp32_parity_sweeps)."""
    return fp32_parity_sweeps(plan, sims, samples, n_sweeps, ops, N_of, lambda s: _rep_slice(plan, s))


def _report(label, stats):
    compared, traced, flipped, worst = stats
    print(f"{label}: {compared} replica-sweeps, {traced} misses traced to {flipped} flipped near-tie decisions, "
          f"0 unexplained, worst |dE|/N {worst:.2e}")


@pytest.mark.parametrize("engine_name", ["FP32_RESIDENT", "FP32_SPLIT", "FP32_GLOBAL", "FP32_PLAIN"])
@pytest.mark.parametrize("name", ["C1", "C2"])
def test_fp32_energy_matches_oracle(env, orc, name, engine_name):
    xyl, wl = env
    cfg = wl.config(name)
    eng, opts = _variant(xyl, engine_name)
    plan, _ = wl.make_plan(cfg, eng, **opts)
    plan.bind()
    plan.init_spins()
    sims = {0: _oracle_for(orc, wl, cfg, 0, u24=True)}
    assert _angle_gap(_gpu_angles(plan, 0, cfg.n_temps), sims[0].angles()).max() < 1e-6
    _report(f"{name} {engine_name}", _fp32_per_sweep(plan, sims, [0], 10, ALL, lambda s: cfg.graphs[s][0] ** 2))
    assert plan.status() == (0, 10)


def test_fp32_energy_matches_oracle_in_the_benchmark_shape(env, orc):
    """C2 in the launch shape the benchmark times (spins in shared memory, one
    replica per group, six CTAs per replica, 512 threads)."""
    xyl, wl = env
    cfg = wl.config("C2")
    eng, opts = _variant(xyl, "FP32_BENCH")
    plan, _ = wl.make_plan(cfg, eng, **opts)
    t = plan.tuning()
    assert (t["resident"], t["group"], t["cluster"], t["block"]) == (1, 1, 6, 512)
    plan.bind()
    plan.init_spins()
    sims = {0: _oracle_for(orc, wl, cfg, 0, u24=True)}
    _report("C2 bench shape", _fp32_per_sweep(plan, sims, [0], 10, ALL, lambda s: cfg.graphs[s][0] ** 2))
    assert plan.status() == (0, 10)


@pytest.mark.parametrize("engine_name", ["FP32_RESIDENT", "FP32_SPLIT", "FP32_GLOBAL", "FP32_PLAIN"])
@pytest.mark.parametrize("name", ["E1", "E2"])
def test_fp32_energy_matches_oracle_bond_ensemble(env, orc, name, engine_name):
    """The paper's 2N-bond graphs (Sec. II): free degrees up to 11 here, so
    both batched shapes run their any-degree kernels (rows read from the
    global CSR entry by entry)."""
    xyl, wl = env
    cfg = wl.config(name)
    graphs = wl.build_graphs(cfg)
    assert graphs[0].max_deg > 8
    eng, opts = _variant(xyl, engine_name)
    plan, _ = wl.make_plan(cfg, eng, graphs=graphs, **opts)
    plan.bind()
    plan.init_spins()
    sims = {0: _oracle_for(orc, wl, cfg, 0, u24=True)}
    _report(f"{name} {engine_name}", _fp32_per_sweep(plan, sims, [0], 10, ALL, lambda s: cfg.graphs[s][0] ** 2))
    assert plan.status() == (0, 10)


# --------------------------------------------------------------- long runs
def _observables(N):
    """Sec. III observables from a slot's mean accumulator row: e, the
    connected chi, U4 in the paper's form, <|m|> and chi(k_min)."""
    return {
        "e": lambda m: m[ACC["e"]],
        "chi": lambda m: N * (m[ACC["m2"]] - m[ACC["mx"]] ** 2 - m[ACC["my"]] ** 2),
        "U4": lambda m: m[ACC["m4"]] / m[ACC["m2"]] ** 2 - 1,
        "absm": lambda m: m[ACC["absm"]],
        "chik": lambda m: m[ACC["chik"]],
    }


def _compare_long_run(label, ob, gb, fns, slots):
    """Per slot and observable: FP32 engine minus FP64 oracle within 3 sigma
    (binned jackknife of both); prints the difference and sigma."""
    for k in slots:
        for key, fn in fns.items():
            a, da = jackknife(ob[:, k, :], fn)
            b, db = jackknife(gb[:, k, :], fn)
            sigma = np.hypot(da, db)
            print(f"ERRTAB {label} slot {k} {key}: oracle {a:.6g} +- {da:.2g}, FP32 {b:.6g} +- {db:.2g}, "
                  f"diff {b - a:+.3g} = {(b - a) / sigma:+.2f} sigma")
            assert abs(a - b) < 3 * sigma, (label, k, key, a, da, b, db)


def _tuned_deltas(orc, wl, cfg, ops):
    """Metropolis half-widths tuned on the oracle to about 50% acceptance, then frozen."""
    sim = _oracle_for(orc, wl, cfg, 0, u24=False)
    delta = np.array(cfg.deltas())
    for _ in range(6):
        sim.sweeps(200, ops)
        st = sim.accumulators()
        rate = st["met_acc"] / st["met_try"]
        delta = np.clip(delta * rate / 0.5, 0.05, np.pi)
        sim.set_delta(delta)
        sim.reset_acc()
    return list(delta)


def test_long_run_statistics_bond_ensemble(env, orc):
    """E1 (L=16, 2N bonds, rho=0, four temperatures around the critical point
    with parallel tempering): per slot <e>, chi, U4 and <|m|> of the FP32
    batched engine agree with the FP64 oracle within 3 sigma (binned jackknife)."""
    xyl, wl = env
    cfg = wl.config("E1")
    cfg.delta = _tuned_deltas(orc, wl, cfg, ALL)
    sim = _oracle_for(orc, wl, cfg, 0, u24=False)
    plan, _ = wl.make_plan(cfg, xyl.FP32_BATCHED)
    plan.bind()
    plan.init_spins()
    for s in (sim, plan):
        s.sweeps(500, ALL)
        s.reset_acc()
    ob = bin_means(run_bins(sim, 100, 100, ALL))
    gb = bin_means(run_bins(plan, 100, 100, ALL))
    N = 256
    _compare_long_run("E1", ob, gb, _observables(N), range(cfg.n_temps))
    assert plan.status()[0] == 0


@pytest.mark.parametrize("engine_name", ["FP32_RESIDENT", "FP32_GLOBAL", "FP64_PLAIN"])
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
    eng, opts = _variant(xyl, engine_name)
    plan, _ = wl.make_plan(cfg, eng, **opts)
    plan.bind()
    plan.init_spins()
    for s in (sim, plan):
        s.sweeps(500, NO_PT)
        s.reset_acc()
    ob = bin_means(run_bins(sim, 100, 100, NO_PT))
    gb = bin_means(run_bins(plan, 100, 100, NO_PT))
    _compare_long_run(f"C1 {engine_name}", ob, gb, _observables(256), [0])
    plan.sweeps(200, NO_PT)
    st = plan.read_observables()
    rate = st["met_acc"][0] / st["met_try"][0]
    assert 0.35 < rate < 0.65


# --------------------------------------------------------------- exact results through the kernels
def _edge_plan(xyl, edges, n, betas, deltas, variant, xy=None, L=0, seed=5):
    g = xyl.graph_from_edges(n, edges, xy=xy, L=L)
    eng, opts = _variant(xyl, variant)
    p = xyl.Plan([(g, 0, betas, deltas)], engine=eng, seed=seed, **opts)
    p.bind()
    p.init_spins()
    return p


ENGINES = ["FP32_RESIDENT", "FP32_SPLIT", "FP32_GLOBAL", "FP64_PLAIN", "FP32_PLAIN"]


@pytest.mark.parametrize("engine_name", ENGINES)
def test_chain_and_ring_closed_forms(env, engine_name):
    xyl, _ = env
    eng = engine_name
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
    eng = engine_name
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
    eng, opts = _variant(xyl, engine_name)
    p = xyl.Plan([(g, 0, [0.0], [np.pi])], engine=eng, seed=9, **opts)
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
@pytest.mark.parametrize("name,sampled,resident", [("C3", [0, 400, 767], 1), ("C3", [1, 511], -1),
                                                    ("C4", [0, 47], 0), ("C5", [70], 0),
                                                    ("C3", [2, 700], "bench"), ("C4", [5, 44], "bench"),
                                                    ("C5", [3, 127], "bench")])
def test_full_size_batched_sampled_parity(env, orc, name, sampled, resident):
    """Whole batch in a given launch configuration (resident "bench": the shapes
    the benchmark takes from the committed autotune cache, e.g. C5 spread over
    the whole GPU); sampled samples are re-run by the oracle from the same
    seeds; every sample obeys the invariants."""
    import os
    xyl, wl = env
    cfg = wl.config(name)
    bench_shape = resident == "bench"
    plan, graphs = wl.make_plan(cfg, xyl.FP32_BATCHED, resident=0 if bench_shape else resident)
    assert bench_shape or plan.tuning()["resident"] == (1 if resident == 1 else -1) or resident == 0
    plan.bind()
    if bench_shape:
        cache = os.path.join(os.path.dirname(xyl.__file__), "autotune_cache.json")
        _, hit = plan.autotune_cached(cache)
        assert hit, "the committed cache holds this batch's shapes"
        if name == "C3":
            # one group per sample, never waiting on another: all 768 in one launch, as many resident as fit
            assert plan.wave_units() == 768 and 0 < plan.live_units() < 768
    plan.init_spins()
    sims = {k: _oracle_for(orc, wl, cfg, k, u24=True) for k in sampled}
    n_sweeps = 2 if name == "C5" else 3
    _report(name, _fp32_per_sweep(plan, sims, sampled, n_sweeps, ALL, lambda s: cfg.graphs[s][0] ** 2))
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
@pytest.mark.parametrize("shape", [dict(resident=1), dict(resident=1, cluster=4), dict(resident=-1)])
def test_batched_runs_are_deterministic_and_resumable(env, shape):
    xyl, wl = env
    cfg = wl.config("C2")
    graphs = wl.build_graphs(cfg)
    a, _ = wl.make_plan(cfg, xyl.FP32_BATCHED, graphs=graphs, **shape)
    b, _ = wl.make_plan(cfg, xyl.FP32_BATCHED, graphs=graphs, **shape)
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
    for k in ("met_acc", "met_try", "pt_acc", "pt_try"):
        assert np.array_equal(ra[k], rb[k]), k
    # sums across CTAs are FP64 atomics in no fixed order: last bits only
    np.testing.assert_allclose(ra["acc"], rb["acc"], rtol=1e-12, atol=0)
    assert a.status() == b.status() == (0, 25)


@pytest.mark.parametrize("shape", [dict(resident=-1), dict(resident=1), dict(resident=1, cluster=4)])
def test_standalone_pt_and_measure_between_sweeps(env, shape):
    """xyl_pt_swap and xyl_measure between batched sweeps: the next sweep's
    fused energies still equal a fresh FP64 recomputation."""
    xyl, wl = env
    cfg = wl.config("C2")
    plan, _ = wl.make_plan(cfg, xyl.FP32_BATCHED, **shape)
    plan.bind()
    plan.init_spins()
    plan.sweep(3, ALL)
    plan.measure()
    plan.pt_swap()
    plan.sweep(2, ALL)
    E = plan.energies()
    plan.recompute()
    assert np.max(np.abs(plan.energies() - E)) / 16384 < 1e-5
    assert np.all(plan.read_observables()["acc"][:, ACC["n"]] == 6)  # five sweeps and one xyl_measure


def test_c4_drift_at_its_recompute_interval(env):
    """C4 (uneven sizes, FP64 recompute every 100 sweeps): the largest
    |E_fused - E_fp64| the recomputes see stays far below the 1e-5-per-spin
    bar of the smallest sample (N = 1024)."""
    xyl, wl = env
    cfg = wl.config("C4")
    plan, _ = wl.make_plan(cfg, xyl.FP32_BATCHED)
    plan.bind()
    plan.init_spins()
    plan.sweep(300, ALL, 32)
    d = plan.drift()
    print(f"ERRTAB C4 drift after 300 sweeps (recompute every 100): max |E_fused - E_fp64| = {d:.3g} "
          f"({d / 1024:.2g} per spin at N = 1024, {d / 36864:.2g} at N = 36864)")
    assert plan.status() == (0, 300)
    assert 0.0 < d < 1e-5 * 1024


def test_device_check_of_the_colour_classes(env):
    """xyl_check_plan finds no fault in sound plans (fixed-degree graphs, the
    paper's 2N-bond graphs, a mixed-size batch run as parts) and counts the
    faults of a CSR corrupted in the workspace: a link inside a colour class."""
    import torch
    xyl, wl = env
    for name in ("C2", "E1", "B64"):
        cfg = wl.config(name)
        plan, _ = wl.make_plan(cfg, xyl.FP32_BATCHED)
        plan.bind()
        assert plan.check() == 0, name
    cfg = _c4_two_per_size(wl)
    plan, _ = wl.make_plan(cfg, xyl.FP32_BATCHED)
    plan.bind()
    assert plan.check() == 0
    # corrupt sample 0 of C2: the first id of row 0 becomes a site of row 0's own class
    cfg = wl.config("C2")
    graphs = wl.build_graphs(cfg)
    plan, _ = wl.make_plan(cfg, xyl.FP32_BATCHED, graphs=graphs)
    plan.bind()
    _, row_ptr, col, cptr = graphs[0].csr()
    ws = plan.workspace.cpu().numpy().view(np.int32).copy()
    hits = np.flatnonzero(ws[: len(ws) - len(col)] == col[0])
    at = next(k for k in hits if np.array_equal(ws[k:k + len(col)], col))
    ws[at] = 1 if cptr[1] > 1 else 0  # site 1 shares site 0's colour class
    plan.workspace.copy_(torch.from_numpy(ws.view(np.uint8)).to(plan.workspace.device))
    assert plan.check() >= 2  # the link is inside a class and is missing from row 1


def test_recompute_bounds_fp32_drift(env):
    xyl, wl = env
    cfg = wl.config("C2")
    plan, _ = wl.make_plan(cfg, xyl.FP32_BATCHED, recompute_every=50)
    plan.bind()
    plan.init_spins()
    assert plan.drift() == 0.0
    plan.sweep(200, ALL)
    # four periodic recomputes ran: their largest |E_fused - E_fp64| is recorded
    d200 = plan.drift()
    assert 0.0 < d200 / 16384 < 1e-5
    E = plan.energies()
    plan.recompute()
    gap = np.max(np.abs(plan.energies() - E))
    assert gap / 16384 < 1e-5
    assert plan.drift() == max(d200, gap)
    s = plan.spins(0, 3)
    assert np.max(np.abs(np.hypot(s[:, 0], s[:, 1]) - 1)) < 1e-6
    # writing spins changes the energies but is not a drift; a reset clears it
    plan.write_spins(0, 3, -s)
    assert plan.drift(reset=True) == max(d200, gap)
    assert plan.drift() == 0.0


@pytest.mark.parametrize("shape", [dict(resident=1), dict(resident=-1)])
def test_delta_tuning_reaches_half_acceptance(env, shape):
    """xyl_tune_delta: after the warm-up every C2 slot (T in [0.8, 1.6], where
    Delta < pi suffices) accepts 40-60% of its proposals with the frozen
    half-widths, and the accumulators start from zero."""
    xyl, wl = env
    cfg = wl.config("C2")
    plan, _ = wl.make_plan(cfg, xyl.FP32_BATCHED, **shape)
    plan.bind()
    plan.init_spins()
    d0 = plan.get_delta(0)
    rate = plan.tune_delta(rounds=8, n_sweeps=50)
    d = plan.get_delta(0)
    assert np.all((rate > 0.4) & (rate < 0.6)), rate
    assert np.all((d > 0) & (d <= np.pi)) and not np.allclose(d, d0)
    assert np.all(np.diff(d) > 0)  # hotter slots take wider steps
    st = plan.read_observables()
    assert not st["acc"].any() and not st["met_try"].any()
    # the frozen widths hold: a further block accepts about half as well
    plan.sweep(100, 1 | 2 | 4)
    st = plan.read_observables()
    r = st["met_acc"] / st["met_try"]
    assert np.all((r > 0.35) & (r < 0.65)), r


@pytest.mark.parametrize("shape", [dict(group=4, resident=-1), dict(group=1, cluster=4, resident=1)])
def test_split_sample_wait_times_out_and_recovers(env, shape):
    """Running one of a sample's replica groups alone makes its bounded wait for
    the other groups give up: status ETIMEOUT, context still usable."""
    xyl, wl = env
    cfg = wl.config("C2")
    plan, _ = wl.make_plan(cfg, xyl.FP32_BATCHED, **shape)
    plan.bind()
    plan.init_spins()
    assert plan.unit_count() == cfg.n_temps // shape["group"]
    plan.sweep_units(0, 1, 3, ALL)
    status, _ = plan.status()
    assert status == xyl.ETIMEOUT
    with pytest.raises(xyl.XylError) as e:
        plan.energies()
    assert e.value.code == xyl.ETIMEOUT
    plan.init_spins()
    plan.sweep(5, ALL)
    assert plan.status() == (0, 5)


def test_launch_shape_does_not_change_the_trajectory(env):
    """Per-site arithmetic does not depend on the launch shape: replica groups,
    cluster width, block size and CSR staging give bit-identical spins.  (PT
    decisions read FP32 energy sums whose order follows the shape, so this
    runs Metropolis + overrelaxation.)"""
    xyl, wl = env
    cfg = wl.config("C2")
    graphs = wl.build_graphs(cfg)
    shapes = [dict(group=16, cluster=16, block=512, resident=-1), dict(group=1, cluster=8, block=256, resident=-1),
              dict(group=4, cluster=4, block=128, stage=-1, resident=-1),
              dict(group=4, cluster=16, block=640, resident=-1),
              dict(group=1, block=640, resident=1), dict(group=1, block=256, stage=-1, resident=1),
              dict(group=1, cluster=4, block=640, resident=1), dict(group=1, cluster=2, block=384, stage=-1, resident=1),
              dict(group=1, block=1024, resident=1), dict(group=1, cluster=6, block=768, resident=1)]
    ref = None
    for shp in shapes:
        p, _ = wl.make_plan(cfg, xyl.FP32_BATCHED, graphs=graphs, **shp)
        p.bind()
        p.init_spins()
        p.sweep(6, NO_PT)
        got = (np.stack([p.spins(0, r) for r in range(cfg.n_temps)]), p.labels())
        if ref is None:
            ref = got
        else:
            assert np.array_equal(got[0], ref[0]), shp
            assert np.array_equal(got[1], ref[1]), shp
    # the per-colour-launch FP32 engine performs the same per-site arithmetic
    p, _ = wl.make_plan(cfg, xyl.FP32_PLAIN, graphs=graphs)
    p.bind()
    p.init_spins()
    p.sweep(6, NO_PT)
    assert np.array_equal(np.stack([p.spins(0, r) for r in range(cfg.n_temps)]), ref[0])


def test_any_degree_shapes_give_the_same_spins(env):
    """On the paper's 2N-bond graphs (degrees above 8): the resident shape (one
    CTA, two, or four per group), the global-memory shape and the FP32 plain
    engine perform the same per-site arithmetic, bit for bit."""
    xyl, wl = env
    cfg = wl.Config("B8", [(64, 10.0 / 3.0, s) for s in range(8)], wl.geometric_temperatures(1.4, 2.0, 12),
                    ensemble="bonds")
    graphs = wl.build_graphs(cfg)
    assert max(g.max_deg for g in graphs) > 8
    ref = None
    for eng, shp in ((xyl.FP32_BATCHED, dict(group=4, resident=1)), (xyl.FP32_BATCHED, dict(group=2, resident=1)),
                     (xyl.FP32_BATCHED, dict(group=1, cluster=4, resident=1)),
                     (xyl.FP32_BATCHED, dict(group=4, cluster=2, block=1024, resident=1)),
                     (xyl.FP32_BATCHED, dict(group=4, cluster=2, resident=-1)), (xyl.FP32_PLAIN, {})):
        p, _ = wl.make_plan(cfg, eng, graphs=graphs, **shp)
        if eng == xyl.FP32_BATCHED:
            assert p.tuning()["resident"] == shp["resident"], shp
        p.bind()
        p.init_spins()
        p.sweep(5, NO_PT)
        got = np.stack([p.spins(k, r) for k in range(cfg.n_samples) for r in range(cfg.n_temps)])
        if ref is None:
            ref = got
        else:
            assert np.array_equal(got, ref), shp
        assert p.status() == (0, 5)


def _c4_two_per_size(wl):
    """C4's six sizes (L = 32..192, rho = 3, 20 temperatures), two samples each."""
    cfg = wl.config("C4")
    idx = [k for k, g in enumerate(cfg.graphs) if g[2] < 2]
    cfg.stream_ids = [wl.graph_stream_id(cfg, k) for k in idx]
    cfg.graphs = [cfg.graphs[k] for k in idx]
    return cfg


def test_mixed_sizes_as_parts_give_the_same_spins(env):
    """A mixed-size batch run as parts (each size its own launch shape, spins in
    shared memory where a group fits, the parts without a cross-cluster barrier
    side by side on forked streams) gives spins bit-identical to the whole
    batch in one global-memory shape; with parallel tempering and measurement
    it runs cleanly and every sample keeps a permutation of its slots."""
    xyl, wl = env
    cfg = _c4_two_per_size(wl)
    graphs = wl.build_graphs(cfg)
    parts, _ = wl.make_plan(cfg, xyl.FP32_BATCHED, graphs=graphs)
    whole, _ = wl.make_plan(cfg, xyl.FP32_BATCHED, graphs=graphs, resident=-1)
    assert parts.part_count() == 6 and whole.part_count() == 1
    assert [parts.part_tuning(k)["resident"] for k in range(6)][-3:] == [1, 1, 1]
    for p in (parts, whole):
        p.bind()
        p.init_spins()
        p.sweep(4, NO_PT)
        p.sweep(3, NO_PT)
    for k in range(cfg.n_samples):
        for r in range(cfg.n_temps):
            assert np.array_equal(parts.spins(k, r), whole.spins(k, r)), (k, r)
    assert parts.status() == (0, 7)
    parts.sweep(40, ALL, 4)
    assert parts.status() == (0, 47)
    labels = parts.labels().reshape(cfg.n_samples, cfg.n_temps)
    assert all(sorted(row.tolist()) == list(range(cfg.n_temps)) for row in labels)
    st = parts.read_observables()
    assert np.all(st["acc"][:, ACC["n"]] == 7 + 10)  # every one of the first 7 sweeps measured, then every 4th
    assert np.all(st["pt_try"].reshape(cfg.n_samples, cfg.n_temps)[:, :-1] > 0)


def test_replica_pairs_same_spins_in_every_shape(env):
    """Four L=64 samples x 24 temperatures (replicas updated in pairs, RV = 2):
    the resident shape at 512 and 1024 threads, split over three CTAs, and the
    global-memory shape give bit-identical spins (Metropolis + overrelaxation)."""
    xyl, wl = env
    cfg = wl.config("C3")
    cfg.graphs = cfg.graphs[:2] + cfg.graphs[256:257] + cfg.graphs[767:768]
    cfg.stream_ids = [0, 1, 256, 767]
    graphs = wl.build_graphs(cfg)
    ref = None
    for shp in (dict(group=4, block=512, resident=1), dict(group=4, block=1024, resident=1),
                dict(group=2, cluster=3, block=768, resident=1), dict(group=8, cluster=2, block=640, resident=-1)):
        p, _ = wl.make_plan(cfg, xyl.FP32_BATCHED, graphs=graphs, **shp)
        p.bind()
        p.init_spins()
        p.sweep(5, NO_PT)
        got = np.stack([p.spins(s, r) for s in range(4) for r in range(cfg.n_temps)])
        if ref is None:
            ref = got
        else:
            assert np.array_equal(got, ref), shp


def _twenty_slots(wl, L=48):
    """Two L x L samples of C4's family (rho = 3) with C4's 20 temperatures."""
    return wl.Config("T20", [(L, 3.0, 0), (L, 3.0, 1)], wl.geometric_temperatures(1.5, 3.5, 20))


# global-memory shapes whose lanes per site (group / 2 replicas per thread)
# are not a power of two: one group per sample (20), two (10), a block that
# leaves threads without a lane (1024 = 102 x 10 + 4), rows staged
NON_POW2 = [dict(group=20, cluster=2, block=640, resident=-1), dict(group=10, cluster=3, block=640, resident=-1),
            dict(group=20, cluster=4, block=1024, resident=-1), dict(group=10, cluster=1, block=512, resident=-1),
            dict(group=10, cluster=2, block=640, resident=-1, stage=0)]


def test_groups_of_any_size_give_the_same_spins(env):
    """Replica groups whose lanes per site are not a power of two (20 slots:
    groups of 20 or 10) perform the same per-site arithmetic as the
    power-of-two groups and the FP32 plain engine, bit for bit; their CTA
    sums (thread order instead of warp shuffles) agree with the power-of-two
    shape's to FP32 rounding, the Metropolis counts exactly."""
    xyl, wl = env
    cfg = _twenty_slots(wl)
    graphs = wl.build_graphs(cfg)
    ref = None
    for eng, shp in [(xyl.FP32_BATCHED, dict(group=4, cluster=2, block=640, resident=-1))] + \
            [(xyl.FP32_BATCHED, shp) for shp in NON_POW2] + [(xyl.FP32_PLAIN, {})]:
        p, _ = wl.make_plan(cfg, eng, graphs=graphs, **shp)
        if eng == xyl.FP32_BATCHED:
            t = p.tuning()
            assert (t["group"], t["resident"]) == (shp["group"], -1), shp
        p.bind()
        p.init_spins()
        p.sweep(6, NO_PT, 2)
        spins = np.stack([p.spins(k, r) for k in range(2) for r in range(20)])
        st = p.read_observables()
        if ref is None:
            ref = (spins, st)
            continue
        assert np.array_equal(spins, ref[0]), shp
        assert np.array_equal(st["met_acc"], ref[1]["met_acc"]) and np.array_equal(st["met_try"], ref[1]["met_try"])
        np.testing.assert_allclose(st["acc"], ref[1]["acc"], rtol=2e-5, atol=2e-5, err_msg=str(shp))
        assert p.status() == (0, 6)


@pytest.mark.parametrize("shape", NON_POW2[:3], ids=["g20", "g10", "g20-1024"])
def test_fp32_parity_groups_of_any_size(env, orc, shape):
    """With parallel tempering and measurement: every replica-sweep of both
    samples against the oracle (24-bit draws) under the traced parity rule."""
    xyl, wl = env
    cfg = _twenty_slots(wl, L=32)
    plan, _ = wl.make_plan(cfg, xyl.FP32_BATCHED, **shape)
    plan.bind()
    plan.init_spins()
    sims = {k: _oracle_for(orc, wl, cfg, k, u24=True) for k in range(2)}
    _report(f"T20 {shape}", _fp32_per_sweep(plan, sims, [0, 1], 6, ALL, lambda s: 32 * 32))
    assert plan.status() == (0, 6)


# global-memory shapes whose replica group spans several clusters (span): the
# span clusters of a group share its colour chunks and meet at a bounded
# global barrier after every colour phase
SPREAD = [dict(group=16, cluster=2, block=512, resident=-1, span=4),
          dict(group=16, cluster=1, block=1024, resident=-1, span=12),
          dict(group=8, cluster=4, block=640, resident=-1, span=3)]


def test_groups_spread_over_clusters_give_the_same_spins(env):
    """A group spread over several clusters performs the same per-site
    arithmetic as one cluster per group, bit for bit (Metropolis +
    overrelaxation); its sums agree to FP32 rounding, its Metropolis counts
    exactly."""
    xyl, wl = env
    cfg = wl.config("C2")
    graphs = wl.build_graphs(cfg)
    ref = None
    for shp in [dict(group=16, cluster=2, block=512, resident=-1)] + SPREAD:
        p, _ = wl.make_plan(cfg, xyl.FP32_BATCHED, graphs=graphs, **shp)
        assert p.tuning()["span"] == shp.get("span", 1), shp
        p.bind()
        p.init_spins()
        p.sweep(6, NO_PT, 2)
        spins = np.stack([p.spins(0, r) for r in range(cfg.n_temps)])
        st = p.read_observables()
        assert p.status() == (0, 6), shp
        if ref is None:
            ref = (spins, st)
            continue
        assert np.array_equal(spins, ref[0]), shp
        assert np.array_equal(st["met_acc"], ref[1]["met_acc"]), shp
        np.testing.assert_allclose(st["acc"], ref[1]["acc"], rtol=2e-5, atol=2e-5, err_msg=str(shp))


@pytest.mark.parametrize("shape", SPREAD[:2], ids=["span4", "span12"])
def test_fp32_parity_groups_spread_over_clusters(env, orc, shape):
    """With parallel tempering and measurement, against the oracle (24-bit
    draws) under the traced parity rule."""
    xyl, wl = env
    cfg = wl.config("C2")
    plan, _ = wl.make_plan(cfg, xyl.FP32_BATCHED, **shape)
    plan.bind()
    plan.init_spins()
    sims = {0: _oracle_for(orc, wl, cfg, 0, u24=True)}
    _report(f"C2 {shape}", _fp32_per_sweep(plan, sims, [0], 6, ALL, lambda s: 128 * 128))
    assert plan.status() == (0, 6)


def test_spread_shape_at_full_size(env, orc):
    """Two C5 samples (L=512, 32 temperatures), each spread over eight
    8-CTA clusters of 1024 threads: both against the oracle for two sweeps."""
    xyl, wl = env
    cfg = wl.first_samples(wl.config("C5"), 2)
    plan, _ = wl.make_plan(cfg, xyl.FP32_BATCHED, group=32, cluster=8, block=1024, resident=-1, span=8)
    plan.bind()
    # the 8 clusters of a sample wait on one another: a wave is whole samples, all resident
    assert plan.unit_count() == 2 and plan.wave_units() == plan.live_units() >= 1
    plan.init_spins()
    sims = {k: _oracle_for(orc, wl, cfg, k, u24=True) for k in range(2)}
    _report("C5x2 span 8", _fp32_per_sweep(plan, sims, [0, 1], 2, ALL, lambda s: 512 * 512))
    assert plan.status() == (0, 2)


def test_cache_entry_that_does_not_fit_is_retuned(env, tmp_path):
    """A cached launch shape that cannot run on this GPU (more clusters per
    group than can be resident) is replaced by a fresh autotune, not raised."""
    import json
    xyl, wl = env
    cfg = wl.config("G1")
    plan, _ = wl.make_plan(cfg, xyl.FP32_BATCHED)
    plan.bind()
    plan.init_spins()
    path = tmp_path / "cache.json"
    bad = {"block": 256, "cluster": 1, "group": 4, "stage": -1, "resident": -1, "waves": -1, "span": 100000}
    path.write_text(json.dumps({plan.signature(): {"parts": [bad], "sizes": [256], "slots": [4]}}))
    parts, hit = plan.autotune_cached(str(path), 2)
    assert not hit and parts[0]["span"] < 100000
    assert json.loads(path.read_text())[plan.signature()]["parts"] == parts
    plan.sweep(3)
    assert plan.status() == (0, 3)


def test_autotune_restores_state(env):
    xyl, wl = env
    cfg = wl.config("C2")
    graphs = wl.build_graphs(cfg)
    a, _ = wl.make_plan(cfg, xyl.FP32_BATCHED, graphs=graphs)
    b, _ = wl.make_plan(cfg, xyl.FP32_BATCHED, graphs=graphs)
    for p in (a, b):
        p.bind()
        p.init_spins()
        p.sweep(3, ALL)
    best = a.autotune(10)
    assert best == {k: a.tuning()[k] for k in best}
    assert a.status() == b.status() == (0, 3)
    for p in (a, b):
        p.sweep(4, ALL)
    for r in range(cfg.n_temps):
        assert np.array_equal(a.spins(0, r), b.spins(0, r))


def test_long_run_statistics_reduced_c3(env, orc):
    """One C3 graph (L=64, rho=3.5) with four temperatures of C3's range under
    parallel tempering: per slot <e>, chi, U4 and <|m|> of the FP32 batched
    engine agree with the FP64 oracle within 3 sigma (binned jackknife)."""
    xyl, wl = env
    cfg = wl.config("C3")
    cfg.graphs = cfg.graphs[256:257]
    cfg.stream_ids = [256]
    cfg.temperatures = wl.geometric_temperatures(1.5, 3.5, 4)
    sim = _oracle_for(orc, wl, cfg, 0, u24=False)
    plan, _ = wl.make_plan(cfg, xyl.FP32_BATCHED)
    plan.bind()
    plan.init_spins()
    for s in (sim, plan):
        s.sweeps(500, ALL)
        s.reset_acc()
    ob = bin_means(run_bins(sim, 60, 100, ALL))
    gb = bin_means(run_bins(plan, 60, 100, ALL))
    _compare_long_run("reduced C3", ob, gb, _observables(64 * 64), range(4))


@pytest.mark.parametrize("engine_name", ENGINES)
def test_degenerate_inputs(env, engine_name):
    """No links, a single site, a zero Metropolis step, an odd number of slots."""
    xyl, _ = env
    eng = engine_name
    # isolated spins: zero field, zero energy; overrelaxation leaves them alone and
    # every Metropolis move is accepted (dE = 0)
    p = _edge_plan(xyl, [], 5, [1.0, 0.5, 2.0], [1.0, 1.0, 1.0], eng)
    s0 = np.stack([p.spins(0, r) for r in range(3)])
    p.sweep(3, 2 | 4 | 8)
    assert np.array_equal(np.stack([p.spins(0, r) for r in range(3)]), s0)
    assert np.all(p.energies() == 0.0)
    p.sweep(3, ALL)
    st = p.read_observables()
    assert np.array_equal(st["met_acc"], st["met_try"])
    assert np.all(st["pt_acc"][:2] == st["pt_try"][:2])  # equal energies: every swap accepted
    assert np.allclose(np.hypot(*np.stack([p.spins(0, r) for r in range(3)]).reshape(-1, 2).T), 1, atol=1e-6)
    # one site, one slot
    p = _edge_plan(xyl, [], 1, [1.0], [0.5], eng)
    p.sweep(4, ALL)
    st = p.read_observables()
    assert st["acc"][0, ACC["n"]] == 4 and abs(st["acc"][0, ACC["m2"]] - 4.0) < 1e-5
    # Delta = 0: proposals equal the current spin, so Metropolis changes nothing
    g = xyl.build_graph_csr(8, 6, 3.5, 1, 0)
    e, opts = _variant(xyl, eng)
    p = xyl.Plan([(g, 0, [1.0, 0.7, 0.4], [0.0, 0.0, 0.0])], engine=e, seed=4, **opts)
    p.bind()
    p.init_spins()
    s0 = np.stack([p.spins(0, r) for r in range(3)])
    p.sweep(5, 1 | 4 | 8)
    assert np.max(np.abs(np.stack([p.spins(0, r) for r in range(3)]) - s0)) < 1e-6
    assert p.status() == (0, 5)
