"""Host-side checks of libxyl (no GPU needed).

* the shared library loads and exports every entry point include/xyl.h declares;
* the library's graph builder and the oracle's build edge-for-edge identical
  graphs and bit-identical colour-sorted CSR at every configuration size;
* argument validation and call-order errors.
"""
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="session")
def xyl():
    from paper_1211_3991_gb300 import build
    build.build()
    from paper_1211_3991_gb300 import xyl as mod
    mod.load()
    return mod


def _header_functions():
    text = open(os.path.join(ROOT, "include", "xyl.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(xyl_[a-z_0-9]+)\s*\(", text)))


def test_exports_every_declared_symbol(xyl):
    names = _header_functions()
    assert len(names) >= 25
    lib = xyl.load()
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    assert set(names) == set(xyl.EXPORTED)


def _oracle_csr(orc, L, rho, seed, sid):
    ei, ej, restarts, _ = orc.levy_graph(L, 6, rho, seed, sid)
    col, q = orc.slo_color(L * L, ei, ej)
    return (ei, ej), orc.csr(L * L, ei, ej, col, q), restarts


CASES = [(16, 3.5, 1, 0), (128, 3.5, 1, 0)] + [(64, rho, 1, s) for rho in (2.5, 3.5, 4.5) for s in (0, 1, 255)] + \
        [(L, 3.0, 1, 3) for L in (32, 48, 64, 96, 128, 192)] + [(512, 2.5, 1, 0), (512, 4.5, 1, 64)] + \
        [(4, 3.5, 9, 0), (6, 2.0, 9, 1), (8, 7.0, 9, 2)]


@pytest.mark.parametrize("L,rho,seed,sid", CASES)
def test_graph_and_csr_bit_exact_vs_oracle(xyl, orc, L, rho, seed, sid):
    g = xyl.build_graph_csr(L, 6, rho, seed, sid)
    (oi, oj), ocsr, restarts = _oracle_csr(orc, L, rho, seed, sid)
    ei, ej = g.edges()
    assert np.array_equal(ei, oi) and np.array_equal(ej, oj)
    for mine, theirs in zip(g.csr(), ocsr):
        assert mine.dtype == theirs.dtype and np.array_equal(mine, theirs)
    assert g.restarts == restarts
    assert g.max_deg == 6 and g.n_edges == L * L * 3


BOND_CASES = [(L, rho, fbc, sid) for fbc in (False, True) for (L, rho, sid) in
              [(16, 0.0, 0), (16, 3.5, 1), (64, 0.0, 2), (64, 7.0 / 3.0, 3), (64, 14.0 / 3.0, 4), (128, 10.0 / 3.0, 5),
               (256, 0.5, 6)]] + [(7, 2.0, True, 7), (4, 1.0, False, 8)]


@pytest.mark.parametrize("L,rho,fbc,sid", BOND_CASES)
def test_levy_bonds_bit_exact_vs_oracle(xyl, orc, L, rho, fbc, sid):
    """The paper's M-bond ensemble (Sec. II): the library's builder and the
    oracle's give the same bonds in the same order and the same CSR."""
    g = xyl.build_levy_bonds(L, rho, 3, sid, fbc=fbc)
    oi, oj, _ = orc.levy_bonds(L, rho, 3, sid, fbc=fbc)
    ei, ej = g.edges()
    assert np.array_equal(ei, oi) and np.array_equal(ej, oj)
    col, q = orc.slo_color(L * L, oi, oj)
    for mine, theirs in zip(g.csr(), orc.csr(L * L, oi, oj, col, q)):
        assert mine.dtype == theirs.dtype and np.array_equal(mine, theirs)


def test_levy_bonds_rejects_bad_input(xyl):
    for args in [(5, 1.0, 0, 0, False), (4, float("nan"), 0, 0, False), (1, 1.0, 0, 0, True)]:
        with pytest.raises(xyl.XylError) as e:
            xyl.build_levy_bonds(args[0], args[1], args[2], args[3], fbc=args[4])
        assert e.value.code == xyl.EINVAL
    with pytest.raises(xyl.XylError) as e:
        xyl.build_levy_bonds(4, 1.0, 0, n_bonds=121)
    assert e.value.code == xyl.EINVAL
    g = xyl.build_levy_bonds(4, 1.0, 0, n_bonds=0)
    assert g.n_edges == 0 and g.n_colors == 1


def test_graph_from_edges_matches_oracle_colouring(xyl, orc):
    rng = np.random.default_rng(4)
    n = 40
    pairs = set()
    while len(pairs) < 90:
        a, b = rng.integers(0, n, 2)
        if a != b:
            pairs.add((int(min(a, b)), int(max(a, b))))
    edges = np.array(sorted(pairs), np.int32)
    g = xyl.graph_from_edges(n, edges)
    col, q = orc.slo_color(n, edges[:, 0], edges[:, 1])
    for mine, theirs in zip(g.csr(), orc.csr(n, edges[:, 0], edges[:, 1], col, q)):
        assert np.array_equal(mine, theirs)


def test_graph_from_edges_rejects_bad_input(xyl):
    with pytest.raises(xyl.XylError) as e:
        xyl.graph_from_edges(3, [[0, 0]])
    assert e.value.code == xyl.EINVAL
    with pytest.raises(xyl.XylError):
        xyl.graph_from_edges(3, [[0, 1], [1, 0]])
    with pytest.raises(xyl.XylError):
        xyl.graph_from_edges(3, [[0, 3]])


@pytest.mark.parametrize("args", [(5, 6, 3.5), (2, 1, 3.5), (16, 0, 3.5), (4, 16, 3.5), (16, 6, float("nan"))])
def test_build_graph_rejects_bad_sizes(xyl, args):
    with pytest.raises(xyl.XylError) as e:
        xyl.build_graph_csr(*args, 1)
    assert e.value.code == xyl.EINVAL


def test_dead_end_limit_reports_egraph(xyl, orc):
    """13-regular graphs on 16 sites: most seeds need restarts and a few exhaust
    all 100 (host-side failure, no GPU involved); both builders agree on every
    outcome and on the number of restarts."""
    fails = 0
    for seed in range(40):
        try:
            g = xyl.build_graph_csr(4, 13, 3.5, seed, 0)
            lib = g.restarts
        except xyl.XylError as e:
            assert e.code == xyl.EGRAPH
            lib = None
        try:
            theirs = orc.levy_graph(4, 13, 3.5, seed, 0)[2]
        except RuntimeError:
            theirs = None
        assert lib == theirs
        fails += lib is None
    assert fails >= 1


def test_plan_validation_without_gpu(xyl):
    g = xyl.build_graph_csr(16, 6, 3.5, 1, 0)
    with pytest.raises(xyl.XylError) as e:
        xyl.Plan([(g, 0, [1.0, 0.5], [1.0])], engine=xyl.FP32_BATCHED, device="cpu")
    with pytest.raises(xyl.XylError):
        xyl.Plan([(g, 0, [1.0], [1.0])], engine=7, device="cpu")
    with pytest.raises(xyl.XylError):
        xyl.Plan([(g, 0, [1.0, 2.0, 3.0], [1.0] * 3)], engine=xyl.FP32_BATCHED, group=2, device="cpu")
    p = xyl.Plan([(g, 0, [1.0, 0.9], [1.0, 1.0])], engine=xyl.FP32_BATCHED, device="cpu")
    assert p.workspace_bytes > 256 * 2 * 8
    with pytest.raises(xyl.XylError) as e:
        p.sweep(1, stream=0)
    assert e.value.code == xyl.ESTATE


def test_resident_shape_selection_without_gpu(xyl):
    """The batched engine's resident shape (spins in shared memory) is the
    default where a CTA can hold whole replicas, with the largest group that
    fits and at most 16 groups per sample; otherwise the global-memory shape."""
    def tuning(L, R, **kw):
        g = xyl.build_graph_csr(L, 6, 3.5, 1, 0)
        return xyl.Plan([(g, 0, [1.0] * R, [1.0] * R)], engine=xyl.FP32_BATCHED, device="cpu", **kw).tuning()

    t = tuning(128, 16)  # 16384 sites: one replica per CTA (128 KB), the 16 groups in one cluster
    assert (t["resident"], t["group"], t["cluster"]) == (1, 1, 1)
    t = tuning(64, 24)   # 4096 sites: four replicas per CTA, six groups per cluster, CSR staged
    assert (t["resident"], t["group"], t["cluster"], t["stage"]) == (1, 4, 1, 1)
    t = tuning(128, 16, cluster=8)  # each replica's sites split over 8 CTAs
    assert (t["resident"], t["group"], t["cluster"], t["stage"]) == (1, 1, 8, 1)
    t = tuning(64, 24, stage=-1)
    assert (t["resident"], t["stage"]) == (1, -1)
    t = tuning(256, 8)   # 65536 sites: 512 KB per replica, does not fit
    assert t["resident"] == -1
    t = tuning(128, 32)  # 32 groups of one replica: no cluster holds them all
    assert t["resident"] == -1
    assert tuning(128, 32, resident=1)["resident"] == 1  # asked for: groups meet at a global barrier
    assert tuning(64, 24, resident=-1)["resident"] == -1
    with pytest.raises(xyl.XylError) as e:
        tuning(256, 8, resident=1)
    assert e.value.code == xyl.EINVAL
    # samples with different slot counts cannot share a resident cluster shape
    g1, g2 = xyl.build_graph_csr(16, 6, 3.5, 1, 0), xyl.build_graph_csr(16, 6, 3.5, 1, 1)
    p = xyl.Plan([(g1, 0, [1.0] * 2, [1.0] * 2), (g2, 1, [1.0] * 4, [1.0] * 4)], engine=xyl.FP32_BATCHED,
                 device="cpu")
    assert p.tuning()["resident"] == -1


def test_couplings_are_validated_and_aligned_with_the_csr(xyl):
    g = xyl.build_graph_csr(16, 6, 3.5, 1, 0)
    ei, ej = g.edges()
    rng = np.random.default_rng(5)
    J = rng.choice(np.array([-1, 1], np.int8), g.n_edges)
    g.set_couplings(J)
    perm, rp, col, _ = g.csr()
    jc = g.couplings()
    inv = np.empty_like(perm)
    inv[perm] = np.arange(len(perm))
    for e in range(g.n_edges):
        for a, b in ((inv[ei[e]], inv[ej[e]]), (inv[ej[e]], inv[ei[e]])):
            k = rp[a] + np.searchsorted(col[rp[a]:rp[a + 1]], b)
            assert col[k] == b and jc[k] == J[e]
    bad = J.copy()
    bad[7] = 0
    with pytest.raises(xyl.XylError) as e:
        g.set_couplings(bad)
    assert e.value.code == xyl.EINVAL
    assert np.array_equal(g.couplings(), jc)     # a rejected call leaves the couplings as they were
    g.set_couplings(None)
    assert np.all(g.couplings() == 1)


def test_fields_are_validated(xyl):
    g = xyl.build_graph_csr(8, 6, 3.5, 1, 0)
    h = np.zeros((64, 2))
    h[5, 1] = np.nan
    with pytest.raises(xyl.XylError) as e:
        g.set_fields(h)
    assert e.value.code == xyl.EINVAL
    g.set_fields(np.ones((64, 2)))
    p = xyl.Plan([(g, 0, [1.0, 0.5], [1.0, 1.0])], engine=xyl.FP32_BATCHED, device="cpu")
    q = xyl.Plan([(g.set_fields(None), 0, [1.0, 0.5], [1.0, 1.0])], engine=xyl.FP32_BATCHED, device="cpu")
    # one float2 per site for the fields (an empty region still takes one 256-byte slot)
    assert p.workspace_bytes == q.workspace_bytes + 64 * 8 - 256


def test_group_sizes_are_validated(xyl):
    """The global-memory shape takes a power of two or an even group dividing
    every n_temps (up to 32); the resident shape only powers of two."""
    g = xyl.build_graph_csr(16, 6, 3.5, 1, 0)
    temps = [1.0] * 20
    for group in (20, 10, 4, 2, 1):
        t = xyl.Plan([(g, 0, temps, temps)], engine=xyl.FP32_BATCHED, device="cpu", group=group, cluster=2,
                     resident=-1).tuning()
        assert (t["group"], t["resident"]) == (group, -1)
    for group, resident in ((3, -1), (5, -1), (40, -1), (10, 1), (20, 1)):
        with pytest.raises(xyl.XylError) as e:
            xyl.Plan([(g, 0, temps, temps)], engine=xyl.FP32_BATCHED, device="cpu", group=group, resident=resident)
        assert e.value.code == xyl.EINVAL, (group, resident)


def test_span_is_validated(xyl):
    """Clusters per replica group above one: global-memory shape only."""
    g = xyl.build_graph_csr(16, 6, 3.5, 1, 0)
    temps = [1.0] * 16
    t = xyl.Plan([(g, 0, temps, temps)], engine=xyl.FP32_BATCHED, device="cpu", group=16, cluster=2, resident=-1,
                 span=4).tuning()
    assert (t["span"], t["cluster"], t["resident"]) == (4, 2, -1)
    assert xyl.Plan([(g, 0, temps, temps)], engine=xyl.FP32_BATCHED, device="cpu", group=16,
                    resident=-1).tuning()["span"] == 1
    for kw in (dict(resident=1, span=2), dict(resident=-1, span=-1)):
        with pytest.raises(xyl.XylError) as e:
            xyl.Plan([(g, 0, temps, temps)], engine=xyl.FP32_BATCHED, device="cpu", group=16, **kw)
        assert e.value.code == xyl.EINVAL, kw


def test_o3_plans_are_validated(xyl):
    g = xyl.build_graph_csr(8, 6, 3.5, 1, 0)
    for engine, kw in ((xyl.FP32_BATCHED, {"spin_dim": 3, "resident": -1}), (xyl.FP32_PLAIN, {"spin_dim": 4})):
        with pytest.raises(xyl.XylError) as e:
            xyl.Plan([(g, 0, [1.0, 0.5], [1.0, 1.0])], engine=engine, device="cpu", **kw)
        assert e.value.code == xyl.EINVAL
    # O(3) on the batched engine: the resident shape, one CTA per group of
    # replicas, the largest group whose three component arrays fit
    big = xyl.build_graph_csr(128, 6, 3.5, 1, 0)
    t = xyl.Plan([(big, 0, [1.0] * 16, [1.0] * 16)], engine=xyl.FP32_BATCHED, device="cpu", spin_dim=3).tuning()
    assert (t["resident"], t["group"], t["cluster"], t["spin_dim"]) == (1, 1, 1, 3)
    mid = xyl.build_graph_csr(64, 6, 3.5, 1, 0)
    t = xyl.Plan([(mid, 0, [1.0] * 24, [1.0] * 24)], engine=xyl.FP32_BATCHED, device="cpu", spin_dim=3).tuning()
    assert (t["resident"], t["group"]) == (1, 4)
    huge = xyl.build_graph_csr(192, 6, 3.5, 1, 0)  # 12 B x 36865 sites > 220 KB even for one replica
    with pytest.raises(xyl.XylError) as e:
        xyl.Plan([(huge, 0, [1.0] * 2, [1.0] * 2)], engine=xyl.FP32_BATCHED, device="cpu", spin_dim=3)
    assert e.value.code == xyl.EINVAL
    q = xyl.Plan([(g, 0, [1.0, 0.5], [1.0, 1.0])], engine=xyl.FP32_PLAIN, device="cpu")
    p = xyl.Plan([(g, 0, [1.0, 0.5], [1.0, 1.0])], engine=xyl.FP32_PLAIN, device="cpu", spin_dim=3)
    # spins are padded 4-vectors: 16 B instead of 8 B per (site, replica)
    assert p.workspace_bytes == q.workspace_bytes + 2 * 64 * 8
    # fields keep the spins' component count: XY fields refuse O(3) spins and the reverse
    g.set_fields(np.ones((64, 2)))
    with pytest.raises(xyl.XylError) as e:
        xyl.Plan([(g, 0, [1.0, 0.5], [1.0, 1.0])], engine=xyl.FP64_PLAIN, device="cpu", spin_dim=3)
    assert e.value.code == xyl.EINVAL
    g.set_fields(np.ones((64, 3)))
    with pytest.raises(xyl.XylError) as e:
        xyl.Plan([(g, 0, [1.0, 0.5], [1.0, 1.0])], engine=xyl.FP64_PLAIN, device="cpu")
    assert e.value.code == xyl.EINVAL
    # O(3) fields: one padded 4-vector per site (16 B FP32, 32 B FP64), every engine
    for engine, kw, b in ((xyl.FP32_PLAIN, {}, 16), (xyl.FP64_PLAIN, {}, 32), (xyl.FP32_BATCHED, {"resident": 1}, 16)):
        with_f = xyl.Plan([(g, 0, [1.0, 0.5], [1.0, 1.0])], engine=engine, device="cpu", spin_dim=3, **kw)
        g.set_fields(None)
        no_f = xyl.Plan([(g, 0, [1.0, 0.5], [1.0, 1.0])], engine=engine, device="cpu", spin_dim=3, **kw)
        g.set_fields(np.ones((64, 3)))
        assert with_f.workspace_bytes == no_f.workspace_bytes + 64 * b - 256
    h = np.ones((64, 3))
    h[7, 2] = np.inf
    with pytest.raises(xyl.XylError) as e:
        g.set_fields(h)
    assert e.value.code == xyl.EINVAL


def test_philox_entry_rejects_bad_arguments(xyl):
    import ctypes as C
    lib = xyl.load()
    assert lib.xyl_philox(None, None, -1, None, None) == xyl.EINVAL
    assert lib.xyl_philox(None, None, 4, None, None) == xyl.EINVAL
    assert lib.xyl_philox(None, None, 0, None, None) == 0
    assert lib.xyl_philox(C.c_void_p(16), C.c_void_p(12), 1, C.c_void_p(32), None) == xyl.EINVAL  # key misaligned


def test_launch_shape_choice_on_the_host(xyl):
    """Shape selection is host logic: the resident shape takes graphs of any
    degree (the 2N-bond ensemble reaches 11 and more) with rows read from the
    global CSR, stages 16-bit rows only up to degree 8, and O(3) plans report
    their spin dimension."""
    bonds = xyl.build_levy_bonds(32, 0.0, 1, 0)
    assert bonds.max_deg > 8
    p = xyl.Plan([(bonds, 0, [1.0] * 8, [1.0] * 8)], engine=xyl.FP32_BATCHED, device="cpu")
    t = p.tuning()
    assert t["resident"] == 1 and t["stage"] == -1 and t["group"] == 8
    fixed = xyl.build_graph_csr(32, 6, 3.5, 1, 0)
    t = xyl.Plan([(fixed, 0, [1.0] * 8, [1.0] * 8)], engine=xyl.FP32_BATCHED, device="cpu").tuning()
    assert t["resident"] == 1 and t["stage"] == 1
    t = xyl.Plan([(bonds, 0, [1.0] * 8, [1.0] * 8)], engine=xyl.FP32_BATCHED, device="cpu", resident=-1).tuning()
    assert t["resident"] == -1
    t = xyl.Plan([(fixed, 0, [1.0] * 2, [1.0] * 2)], engine=xyl.FP32_PLAIN, device="cpu", spin_dim=3).tuning()
    assert t["spin_dim"] == 3


def test_calls_before_bind_report_the_call_order(xyl):
    """Every device-side entry point checks its plan first: a NULL plan is
    XYL_EINVAL, a plan without a workspace XYL_ESTATE; nothing reaches CUDA."""
    import ctypes as C
    lib = xyl.load()
    g = xyl.build_graph_csr(8, 6, 3.5, 1, 0)
    p = xyl.Plan([(g, 0, [1.0, 0.5], [1.0, 1.0])], engine=xyl.FP32_BATCHED, device="cpu")
    h = p.handle
    buf = (C.c_double * 64)()
    calls = {
        "xyl_init_spins": lambda q: lib.xyl_init_spins(q, 0, None),
        "xyl_sweep": lambda q: lib.xyl_sweep(q, 1, 15, 1, None),
        "xyl_sweep_units": lambda q: lib.xyl_sweep_units(q, 0, 1, 1, 15, 1, None),
        "xyl_sweep_noalloc": lambda q: lib.xyl_sweep_noalloc(q, 1, 15, 1, None),
        "xyl_pt_swap": lambda q: lib.xyl_pt_swap(q, None),
        "xyl_measure": lambda q: lib.xyl_measure(q, None),
        "xyl_recompute": lambda q: lib.xyl_recompute(q, None),
        "xyl_set_delta": lambda q: lib.xyl_set_delta(q, 0, buf, None),
        "xyl_read_energies": lambda q: lib.xyl_read_energies(q, buf, None),
        "xyl_read_spins": lambda q: lib.xyl_read_spins(q, 0, 0, buf, None),
        "xyl_export_state": lambda q: lib.xyl_export_state(q, buf, 64 * 8, None),
        "xyl_read_drift": lambda q: lib.xyl_read_drift(q, buf, 0, None),
        "xyl_tune_delta": lambda q: lib.xyl_tune_delta(q, 2, 10, 3, 0.5, buf, None),
        "xyl_check_plan": lambda q: lib.xyl_check_plan(q, C.cast(buf, C.POINTER(C.c_int64)), None),
    }
    for name, call in calls.items():
        assert call(h) == xyl.ESTATE, name
        assert call(None) == xyl.EINVAL, name
    # counts of a plan not yet bound (or no plan) are 0
    for name in ("xyl_wave_units", "xyl_live_units"):
        assert getattr(lib, name)(h) == 0 and getattr(lib, name)(None) == 0, name


def test_mixed_sizes_run_as_parts(xyl):
    """A batch of several sizes with the library choosing the shapes runs one
    part per size, largest first: spins in shared memory where a replica group
    fits (all groups of a sample in one cluster), else in global memory; a
    caller-given shape keeps one part.  Units are numbered part by part."""
    graphs = {L: xyl.build_graph_csr(L, 6, 3.0, 1, k) for k, L in enumerate((32, 64, 96, 128, 192))}
    betas = [1.0 / t for t in np.geomspace(1.5, 3.5, 20)]
    samples = [(graphs[L], k, betas, [1.0] * 20) for k, L in enumerate((64, 192, 32, 96, 128, 64))]
    p = xyl.Plan(samples, engine=xyl.FP32_BATCHED, device="cpu")
    assert p.part_count() == 5
    parts = [p.part_tuning(k) for k in range(5)]
    assert [t["samples"] for t in parts] == [1, 1, 1, 2, 1]          # N = 192^2, 128^2, 96^2, 64^2, 32^2
    assert [t["resident"] for t in parts] == [-1, -1, 1, 1, 1]
    assert [t["group"] for t in parts[2:]] == [2, 4, 4]               # largest group whose spins fit
    assert p.tuning() == {**p.tuning(), **{k: v for k, v in parts[0].items() if k != "samples"}}
    assert p.unit_count() == sum(20 // t["group"] for t in parts[:2]) * 1 + 10 + 2 * 5 + 5
    q = xyl.Plan(samples, engine=xyl.FP32_BATCHED, device="cpu", resident=-1)
    assert q.part_count() == 1 and q.part_tuning(0)["samples"] == 6
    r = xyl.Plan(samples[:1] + samples[5:], engine=xyl.FP32_BATCHED, device="cpu")
    assert r.part_count() == 1
