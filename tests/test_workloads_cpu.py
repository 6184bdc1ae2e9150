"""Every named workload is well formed, and the small ones build their graphs
and plans on the host (no GPU): the inputs the tests and the benchmark use."""
import numpy as np
import pytest

from paper_1211_3991_gb300 import workloads as wl

NAMES = ["C1", "C2", "C3", "C4", "C5", "E1", "E2", "B64", "G1", "G2", "H1", "H2", "O1", "O2", "O2G", "O3"]


@pytest.mark.parametrize("name", NAMES)
def test_config_is_well_formed(name):
    cfg = wl.config(name)
    assert cfg.name == name and cfg.n_samples >= 1 and cfg.n_temps >= 1
    assert all(t > 0 for t in cfg.temperatures)
    assert np.allclose(cfg.betas(), 1.0 / np.asarray(cfg.temperatures))
    assert all(0 < d <= np.pi for d in cfg.deltas())
    assert cfg.spin_dim in (2, 3) and not (cfg.spin_dim == 3 and cfg.field)
    assert cfg.description


def test_unknown_name():
    with pytest.raises(KeyError):
        wl.config("C9")


@pytest.mark.parametrize("name", ["C1", "E1", "E2", "G1", "H1", "O1"])
def test_small_workloads_build_on_the_host(name):
    from paper_1211_3991_gb300 import xyl
    cfg = wl.config(name)
    graphs = wl.build_graphs(cfg)
    assert len(graphs) == cfg.n_samples
    L = cfg.graphs[0][0]
    assert graphs[0].n == L * L
    if cfg.ensemble == "bonds":
        assert graphs[0].n_edges == 2 * L * L
    if cfg.couplings == "pm":
        j = graphs[0].couplings()
        assert set(np.unique(j)) <= {-1, 1} and (j == -1).any()
    engine = xyl.FP32_PLAIN if cfg.spin_dim == 3 else xyl.FP32_BATCHED
    plan, _ = wl.make_plan(cfg, engine, graphs=graphs, device="cpu")
    assert plan.workspace_bytes > 0 and plan.tuning()["spin_dim"] == cfg.spin_dim


def test_fields_and_couplings_are_seeded():
    cfg = wl.config("H1")
    a, b = wl.fields_for(cfg, 0, 256), wl.fields_for(cfg, 0, 256)
    assert np.array_equal(a, b) and np.allclose(np.hypot(*a.T), 0.5)
    assert wl.fields_for(wl.config("G1"), 0, 256) is None
    j = wl.couplings_for(cfg, 0, 768)
    assert np.array_equal(j, wl.couplings_for(cfg, 0, 768)) and abs((j == 1).mean() - 0.5) < 0.1
