"""xyl_sweep_noalloc: the batched sweep for callers that cannot obtain device
memory while they run (the kernel's scratch comes from a fixed array inside the
library).  It must give what xyl_sweep gives on the same plan, call after call.

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


@pytest.mark.parametrize("shape", [dict(resident=1), dict(resident=1, cluster=4), dict(resident=-1)])
def test_noalloc_sweep_matches_sweep_twice(env, shape):
    xyl, wl = env
    cfg = wl.config("C2")
    graphs = wl.build_graphs(cfg)
    ref, _ = wl.make_plan(cfg, xyl.FP32_BATCHED, graphs=graphs, **shape)
    new, _ = wl.make_plan(cfg, xyl.FP32_BATCHED, graphs=graphs, **shape)
    for p in (ref, new):
        p.bind()
        p.init_spins()
    N = cfg.graphs[0][0] ** 2
    for call in range(2):
        ref.sweep(7, ALL)
        new.sweep_noalloc(7, ALL)
        assert new.status() == ref.status() == (0, 7 * (call + 1))
        assert np.max(np.abs(new.energies() - ref.energies())) / N < 1e-5
        assert np.array_equal(new.labels(), ref.labels())
        for r in range(cfg.n_temps):
            assert np.max(np.abs(new.spins(0, r) - ref.spins(0, r))) < 1e-5
        a, b = new.read_observables(), ref.read_observables()
        np.testing.assert_allclose(a["acc"], b["acc"], rtol=1e-6, atol=1e-9)
        for key in ("met_acc", "met_try", "pt_acc", "pt_try"):
            assert np.array_equal(a[key], b[key]), key


def test_noalloc_rejects_batches_beyond_its_scratch(env):
    xyl, _ = env
    g = xyl.build_graph_csr(8, 6, 3.5, 1, 0)
    betas = list(np.linspace(0.3, 1.0, 256))
    p = xyl.Plan([(g, s, betas, [1.0] * 256) for s in range(24)], engine=xyl.FP32_BATCHED, seed=3)
    p.bind()
    p.init_spins()
    with pytest.raises(xyl.XylError) as e:
        p.sweep_noalloc(1, ALL)
    assert e.value.code == xyl.EINVAL and "scratch" in str(e.value)
