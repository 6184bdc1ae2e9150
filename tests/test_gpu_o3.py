"""O(3) spins on the GPU plain engines (App. B's other continuous models)
against the oracle.

* FP64: initial spins identical to the oracle's, then 10 sweeps of Metropolis,
  overrelaxation, PT and measurement with every spin within 1e-12, identical
  slot labels and FP64 accumulators (including m_z and chi(k)) to 1e-9; with
  and without random +-1 couplings.
* FP32: every sweep starts the oracle (24-bit draws) from the GPU's spins and
  labels; energies per spin within 1e-5 and directions within 1e-4 rad, every
  miss traced to near-tie decisions that, forced the other way, reproduce it.
* Gauge invariance: couplings tau_i tau_j J_ij (and fields tau_i h_i) with
  spins tau_i S_i give the negated run bit for bit on every engine.
* Random 3-vector fields (OH1, OH2): the same FP64, FP32 and shape checks.
* A random tree measured by the FP32 engine against the exact tree energy
  -(n-1) L(beta) / n, L the Langevin function.
"""
import numpy as np
import pytest

from helpers import fp32_parity_sweeps

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


def _oracle(orc, wl, cfg, k, u24):
    L, rho, _ = cfg.graphs[k]
    ei, ej, _, _ = orc.levy_graph(L, 6, rho, wl.GRAPH_SEED, wl.graph_stream_id(cfg, k))
    color, _ = orc.slo_color(L * L, ei, ej)
    sim = orc.Sim(L * L, ei, ej, color, cfg.betas(), cfg.deltas(), wl.SPIN_SEED, sample=wl.graph_stream_id(cfg, k),
                  xy=orc.lattice_xy(L), L=L, u24=u24, dim=3)
    J = wl.couplings_for(cfg, k, len(ei))
    if J is not None:
        sim.set_couplings(J.astype(np.float64))
    h = wl.fields_for(cfg, k, L * L)
    if h is not None:
        sim.set_fields(h)
    sim.init()
    return sim


def _gpu_vectors(plan, sample, R):
    return np.stack([plan.spins(sample, r) for r in range(R)])


@pytest.mark.parametrize("name", ["O1", "O2", "O2G", "OH1", "OH2"])
def test_fp64_trajectory_matches_oracle(env, orc, name):
    xyl, wl = env
    cfg = wl.config(name)
    plan, _ = wl.make_plan(cfg, xyl.FP64_PLAIN)
    plan.bind()
    plan.init_spins()
    sim = _oracle(orc, wl, cfg, 0, u24=False)
    R = cfg.n_temps
    assert np.array_equal(_gpu_vectors(plan, 0, R), sim.vectors())
    for t in range(10):
        plan.sweep(1, ALL)
        sim.sweeps(1, ALL)
        gap = np.abs(_gpu_vectors(plan, 0, R) - sim.vectors()).max()
        assert gap < 1e-12, (t, gap)
        assert np.array_equal(plan.labels(), sim.labels())
        np.testing.assert_allclose(plan.energies(), sim.energies(), rtol=1e-10, atol=1e-9)
    g, o = plan.read_observables(), sim.accumulators()
    np.testing.assert_allclose(g["acc"], o["acc"], rtol=1e-9, atol=1e-12)
    assert np.array_equal(g["met_acc"], o["met_acc"]) and np.array_equal(g["pt_acc"], o["pt_acc"])
    assert np.abs(o["acc"][:, 9]).max() > 0  # m_z is measured
    assert plan.status() == (0, 10)


# the FP32 engines for O(3) spins: the per-colour-launch plain engine and the
# batched engine's resident shape (three component arrays in shared memory)
FP32_O3 = {"FP32_PLAIN": ("FP32_PLAIN", {}), "FP32_RESIDENT": ("FP32_BATCHED", {"resident": 1}),
           "FP32_RESIDENT_1": ("FP32_BATCHED", {"resident": 1, "group": 1, "block": 1024})}


@pytest.mark.parametrize("engine_name", ["FP32_PLAIN", "FP32_RESIDENT"])
@pytest.mark.parametrize("name", ["O1", "O2", "O2G", "OH1", "OH2"])
def test_fp32_energy_matches_oracle(env, orc, name, engine_name):
    xyl, wl = env
    cfg = wl.config(name)
    eng, opts = FP32_O3[engine_name]
    plan, _ = wl.make_plan(cfg, getattr(xyl, eng), **opts)
    plan.bind()
    plan.init_spins()
    sim = _oracle(orc, wl, cfg, 0, u24=True)
    R, N = cfg.n_temps, cfg.graphs[0][0] ** 2
    assert np.abs(_gpu_vectors(plan, 0, R) - sim.vectors()).max() < 1e-7
    compared, traced, flipped, worst = fp32_parity_sweeps(plan, {0: sim}, [0], 10, ALL, lambda s: N,
                                                          lambda s: slice(0, R))
    print(f"{name} {engine_name}: {compared} replica-sweeps, {traced} misses traced to {flipped} flipped near-tie "
          f"decisions, 0 unexplained, worst |dE|/N {worst:.2e}")
    assert plan.status() == (0, 10)


@pytest.mark.parametrize("name", ["O2", "O2G", "OH2", "O3"])
def test_resident_shape_gives_the_plain_engines_spins(env, name):
    """The resident O(3) shape performs the plain FP32 engine's per-spin
    arithmetic (same Philox block per replica, neighbour sums in row order,
    the single-precision steps of o3_f32.cuh), so Metropolis + overrelaxation
    sweeps give bit-identical spins; several groups per CTA, one replica per
    CTA at 1024 threads, and a batch of samples (O3: four L=64 graphs)."""
    xyl, wl = env
    cfg = wl.config(name)
    if name == "O3":
        cfg.graphs = cfg.graphs[:4]
    graphs = wl.build_graphs(cfg)
    ref = None
    for eng_name in ("FP32_PLAIN", "FP32_RESIDENT", "FP32_RESIDENT_1"):
        eng, opts = FP32_O3[eng_name]
        p, _ = wl.make_plan(cfg, getattr(xyl, eng), graphs=graphs, **opts)
        if eng == "FP32_BATCHED":
            t = p.tuning()
            assert t["resident"] == 1 and t["spin_dim"] == 3
        p.bind()
        p.init_spins()
        p.sweep(5, NO_PT)
        got = np.stack([p.spins(k, r) for k in range(cfg.n_samples) for r in range(cfg.n_temps)])
        if ref is None:
            ref = got
        else:
            assert np.array_equal(got, ref), eng_name
        assert p.status() == (0, 5)


@pytest.mark.parametrize("engine_name", ["FP32_PLAIN", "FP64_PLAIN", "FP32_RESIDENT"])
@pytest.mark.parametrize("name", ["O2G", "OH2"])
def test_gauge_invariance_is_exact(env, engine_name, name):
    """tau_i S_i with couplings tau_i tau_j J_ij and fields tau_i h_i is the same
    physics: the run follows the original one sign for sign, bit for bit."""
    xyl, wl = env
    cfg = wl.config(name)
    eng_name, opts = FP32_O3.get(engine_name, (engine_name, {}))
    eng = getattr(xyl, eng_name)
    g = wl.build_graphs(cfg)[0]
    ei, ej = g.edges()
    J = wl.couplings_for(cfg, 0, g.n_edges)
    tau = np.random.default_rng(8).choice(np.array([-1, 1], np.int8), g.n)
    gauged = xyl.build_graph_csr(128, 6, 3.5, wl.GRAPH_SEED, wl.graph_stream_id(cfg, 0))
    gauged.set_couplings((tau[ei] * tau[ej] * J).astype(np.int8))
    h = wl.fields_for(cfg, 0, g.n)
    if h is not None:
        gauged.set_fields(h * tau[:, None])
    a, _ = wl.make_plan(cfg, eng, graphs=[g], **opts)
    b, _ = wl.make_plan(cfg, eng, graphs=[gauged], **opts)
    for p in (a, b):
        p.bind()
        p.init_spins()
    for r in range(cfg.n_temps):
        b.write_spins(0, r, a.spins(0, r) * tau[:, None].astype(np.float64))
    # both renormalised the same way (xyl_recompute rescales every spin to |S| = 1)
    b.recompute()
    a.recompute()
    for _ in range(3):
        a.sweep(4, ALL)
        b.sweep(4, ALL)
        for r in range(cfg.n_temps):
            assert np.array_equal(b.spins(0, r), a.spins(0, r) * tau[:, None]), r
        assert np.array_equal(a.labels(), b.labels())
        np.testing.assert_allclose(a.energies(), b.energies(), rtol=1e-12, atol=0)
    assert a.status() == b.status() == (0, 12)


@pytest.mark.parametrize("engine_name", ["FP32_PLAIN", "FP32_RESIDENT"])
def test_random_tree_energy_is_the_langevin_law(env, engine_name):
    xyl, _ = env
    rng = np.random.default_rng(21)
    n, beta = 4096, 1.3
    edges = np.array([(int(rng.integers(0, i)), i) for i in range(1, n)], np.int32)
    g = xyl.graph_from_edges(n, edges)
    eng, opts = FP32_O3[engine_name]
    plan = xyl.Plan([(g, 0, [beta] * 8, [2.0] * 8)], engine=getattr(xyl, eng), seed=3, spin_dim=3, **opts)
    plan.bind()
    plan.init_spins()
    plan.sweep(200, NO_PT)
    plan.reset_observables()
    plan.sweep(2000, NO_PT, 4)
    acc = plan.read_observables()["acc"]
    e = acc[:, 1] / acc[:, 0]
    want = -(n - 1) * (1.0 / np.tanh(beta) - 1.0 / beta) / n
    # 8 independent replicas: their spread bounds the statistical error
    err = e.std(ddof=1) / np.sqrt(len(e))
    assert abs(e.mean() - want) < 5 * err + 2e-5, (e.mean(), want, err)
    assert plan.status() == (0, 2200)


@pytest.mark.parametrize("engine_name", ["FP32_PLAIN", "FP64_PLAIN", "FP32_RESIDENT"])
def test_degenerate_inputs(env, engine_name):
    """No links, a single site, a zero Metropolis step, an odd number of slots."""
    xyl, _ = env
    eng_name, opts = FP32_O3.get(engine_name, (engine_name, {}))
    eng = getattr(xyl, eng_name)

    def plan_of(g, betas, deltas):
        p = xyl.Plan([(g, 0, betas, deltas)], engine=eng, seed=4, spin_dim=3, **opts)
        p.bind()
        p.init_spins()
        return p

    # isolated spins: overrelaxation leaves them alone, every Metropolis move is accepted
    p = plan_of(xyl.graph_from_edges(5, []), [1.0, 0.5, 2.0], [1.0, 1.0, 1.0])
    s0 = np.stack([p.spins(0, r) for r in range(3)])
    p.sweep(3, 2 | 4 | 8)
    assert np.array_equal(np.stack([p.spins(0, r) for r in range(3)]), s0)
    assert np.all(p.energies() == 0.0)
    p.sweep(3, ALL)
    st = p.read_observables()
    assert np.array_equal(st["met_acc"], st["met_try"])
    assert np.all(st["pt_acc"][:2] == st["pt_try"][:2])
    v = np.stack([p.spins(0, r) for r in range(3)]).reshape(-1, 3)
    assert np.allclose(np.linalg.norm(v, axis=1), 1, atol=1e-6) and np.abs(v[:, 2]).max() > 0
    # one site, one slot: m^2 = 1 exactly at every measurement
    p = plan_of(xyl.graph_from_edges(1, []), [1.0], [0.5])
    p.sweep(4, ALL)
    st = p.read_observables()
    assert st["acc"][0, 0] == 4 and abs(st["acc"][0, 6] - 4.0) < 1e-5
    # Delta = 0: the cap is the spin itself, Metropolis changes nothing
    p = plan_of(xyl.build_graph_csr(8, 6, 3.5, 1, 0), [1.0, 0.7, 0.4], [0.0, 0.0, 0.0])
    s0 = np.stack([p.spins(0, r) for r in range(3)])
    p.sweep(5, 1 | 4 | 8)
    assert np.max(np.abs(np.stack([p.spins(0, r) for r in range(3)]) - s0)) < 1e-6
    assert p.status() == (0, 5)


def test_uneven_batch_each_sample_matches_its_oracle(env, orc):
    """Two samples of different sizes (L = 16 and 24) and slot counts in one FP64
    plan: each follows its own oracle run (streams keyed by its sample id)."""
    xyl, wl = env
    sizes, temps = [16, 24], [[0.9, 1.3, 1.8], [1.0, 1.5]]
    graphs = [xyl.build_graph_csr(L, 6, 3.5, wl.GRAPH_SEED, k) for k, L in enumerate(sizes)]
    samples = [(g, 10 + k, [1 / T for T in ts], [1.5] * len(ts)) for k, (g, ts) in enumerate(zip(graphs, temps))]
    plan = xyl.Plan(samples, engine=xyl.FP64_PLAIN, seed=wl.SPIN_SEED, spin_dim=3)
    plan.bind()
    plan.init_spins()
    sims = []
    for k, (L, ts) in enumerate(zip(sizes, temps)):
        ei, ej, _, _ = orc.levy_graph(L, 6, 3.5, wl.GRAPH_SEED, k)
        color, _ = orc.slo_color(L * L, ei, ej)
        sim = orc.Sim(L * L, ei, ej, color, [1 / T for T in ts], [1.5] * len(ts), wl.SPIN_SEED, sample=10 + k,
                      xy=orc.lattice_xy(L), L=L, dim=3)
        sim.init()
        sims.append(sim)
    plan.sweep(6, ALL)
    for sim in sims:
        sim.sweeps(6, ALL)
    labels = plan.labels()
    off = 0
    for k, sim in enumerate(sims):
        R = len(temps[k])
        assert np.abs(_gpu_vectors(plan, k, R) - sim.vectors()).max() < 1e-12, k
        assert np.array_equal(labels[off:off + R], sim.labels()), k
        off += R


@pytest.mark.parametrize("engine_name", ["FP32_PLAIN", "FP32_RESIDENT"])
def test_checkpoint_resumes_bit_for_bit(env, engine_name):
    xyl, wl = env
    cfg = wl.config("O1")
    eng, opts = FP32_O3[engine_name]
    a, _ = wl.make_plan(cfg, getattr(xyl, eng), **opts)
    a.bind()
    a.init_spins()
    a.sweep(5, ALL)
    blob = a.export_state()
    a.sweep(7, ALL)
    want = (_gpu_vectors(a, 0, cfg.n_temps), a.labels(), a.read_observables()["acc"])
    b, _ = wl.make_plan(cfg, getattr(xyl, eng), **opts)
    b.bind()
    b.import_state(blob)
    b.sweep(7, ALL)
    got = (_gpu_vectors(b, 0, cfg.n_temps), b.labels(), b.read_observables()["acc"])
    assert np.array_equal(got[0], want[0]) and np.array_equal(got[1], want[1])
    np.testing.assert_allclose(got[2], want[2], rtol=1e-12)
    assert b.status() == (0, 12)
