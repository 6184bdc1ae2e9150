"""xyl_sweep_noalloc: the batched sweep for callers that cannot obtain device
memory while they run (the kernel's scratch comes from a fixed array inside the
library).  It must give what xyl_sweep gives on the same plan, call after call,
also when the two entry points are mixed on one plan and when the plan
recomputes its energies in FP64 every few sweeps.

Kept in a file of its own that pytest collects last; it runs alone in a fresh
process as well as after the other GPU tests.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ALL = 1 | 2 | 4 | 8


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


def _same_state(xyl, cfg, a, b):
    """Energies within 1e-5 per spin, spins within 1e-5, labels and counters
    identical, accumulators within FP64 summation-order noise."""
    N = cfg.graphs[0][0] ** 2
    assert a.status() == b.status()
    assert np.max(np.abs(a.energies() - b.energies())) / N < 1e-5
    assert np.array_equal(a.labels(), b.labels())
    for r in range(cfg.n_temps):
        assert np.max(np.abs(a.spins(0, r) - b.spins(0, r))) < 1e-5
    x, y = a.read_observables(), b.read_observables()
    np.testing.assert_allclose(x["acc"], y["acc"], rtol=1e-6, atol=1e-9)
    for key in ("met_acc", "met_try", "pt_acc", "pt_try"):
        assert np.array_equal(x[key], y[key]), key


def _twins(xyl, wl, cfg, shape):
    graphs = wl.build_graphs(cfg)
    plans = [wl.make_plan(cfg, xyl.FP32_BATCHED, graphs=graphs, **shape)[0] for _ in range(2)]
    for p in plans:
        p.bind()
        p.init_spins()
    return plans


@pytest.mark.parametrize("shape", [dict(resident=1), dict(resident=1, cluster=4), dict(resident=-1),
                                   dict(resident=1, cluster=4, recompute_every=5),
                                   dict(resident=-1, recompute_every=5),
                                   dict(resident=-1, group=16, cluster=2, block=640, span=8)])
def test_noalloc_sweep_matches_sweep_twice(env, shape):
    xyl, wl = env
    cfg = wl.config("C2")
    ref, new = _twins(xyl, wl, cfg, shape)
    for call in range(2):
        ref.sweep(7, ALL)
        new.sweep_noalloc(7, ALL)
        assert new.status() == (0, 7 * (call + 1))
        _same_state(xyl, cfg, new, ref)
        if shape.get("recompute_every"):
            # the FP64 recomputes ran at the same sweeps: same recorded drift
            assert new.drift() == pytest.approx(ref.drift(), rel=1e-6, abs=1e-9)


@pytest.mark.parametrize("shape", [dict(resident=1, cluster=4), dict(resident=-1)])
def test_noalloc_and_sweep_mix_on_one_plan(env, shape):
    """An odd number of allocation-free sweeps, then xyl_sweep on the same
    plan, equals xyl_sweep alone: the plan's own sum buffer is left cleared.
    Both shapes add their per-CTA sums into that buffer (several CTAs per
    replica group)."""
    xyl, wl = env
    cfg = wl.config("C2")
    ref, mix = _twins(xyl, wl, cfg, shape)
    mix.sweep_noalloc(7, ALL)
    mix.sweep(5, ALL)
    mix.sweep_noalloc(0, ALL)  # nothing runs
    ref.sweep(12, ALL)
    assert mix.status() == (0, 12)
    _same_state(xyl, cfg, mix, ref)


def test_noalloc_on_a_mixed_size_batch(env):
    """A batch of several sizes runs as parts (one launch shape per size); the
    allocation-free sweep runs its parts one after another instead of side by
    side, with the same result."""
    xyl, wl = env
    cfg = wl.config("C4")
    idx = [k for k, g in enumerate(cfg.graphs) if g[2] == 0]
    cfg.stream_ids = [wl.graph_stream_id(cfg, k) for k in idx]
    cfg.graphs = [cfg.graphs[k] for k in idx]
    graphs = wl.build_graphs(cfg)
    plans = [wl.make_plan(cfg, xyl.FP32_BATCHED, graphs=graphs)[0] for _ in range(2)]
    for p in plans:
        assert p.part_count() == 6
        p.bind()
        p.init_spins()
    ref, new = plans
    for _ in range(2):
        ref.sweep(6, ALL)
        new.sweep_noalloc(6, ALL)
    assert new.status() == ref.status() == (0, 12)
    sizes = np.repeat([L * L for L, _, _ in cfg.graphs], cfg.n_temps)
    assert np.max(np.abs(new.energies() - ref.energies()) / sizes) < 1e-5
    assert np.array_equal(new.labels(), ref.labels())
    for k in range(cfg.n_samples):
        for r in range(cfg.n_temps):
            assert np.max(np.abs(new.spins(k, r) - ref.spins(k, r))) < 1e-5


def test_noalloc_batch_limit(env):
    """256 B per slot + 4 B per sample within the 1 MiB array: 31 samples x 128
    slots fit (1015932 B), 32 x 128 do not (1048704 B)."""
    xyl, _ = env
    g = xyl.build_graph_csr(8, 6, 3.5, 1, 0)
    betas = list(np.linspace(0.3, 1.0, 128))

    def plan(samples):
        p = xyl.Plan([(g, s, betas, [1.0] * 128) for s in range(samples)], engine=xyl.FP32_BATCHED, seed=3,
                     resident=-1)
        p.bind()
        p.init_spins()
        return p

    p = plan(31)
    p.sweep_noalloc(2, ALL)
    assert p.status() == (0, 2)
    p = plan(32)
    with pytest.raises(xyl.XylError) as e:
        p.sweep_noalloc(1, ALL)
    assert e.value.code == xyl.EINVAL and "scratch" in str(e.value)
