"""Pins of the oracle's checking aids used by the single-precision parity tests:
the near-tie log, forced outcomes and the replica mask.

None of them may change the sampler when left unset; set, each does exactly
what the parity tests rely on: a forced outcome replaces only the accept/reject
decision of that one (replica, site) test, and a masked run updates only the
chosen replicas.
"""
import numpy as np

OPS_MET_OR = 1 | 2
ALL = 1 | 2 | 4 | 8


def _sim(orc, u24=True, R=4):
    L = 8
    ei, ej, _, _ = orc.levy_graph(L, 6, 3.5, 1, 0)
    color, _ = orc.slo_color(L * L, ei, ej)
    betas = [1.6, 1.2, 0.9, 0.7][:R]
    sim = orc.Sim(L * L, ei, ej, color, betas, [1.5] * R, 7, sample=3, xy=orc.lattice_xy(L), L=L, u24=u24)
    sim.init()
    return sim


def _state(sim):
    return sim.vectors().copy(), sim.labels().copy(), sim.sweep_index


def _restore(sim, st):
    v, lab, t = st
    sim.set_vectors(v)
    sim.set_labels(lab, t)


def test_log_lists_every_counted_tie_with_its_outcome(orc):
    sim = _sim(orc)
    sim.sweeps(3, ALL)
    sim.set_tie_eps(0.05)  # wide band: many logged tests
    sim.clear_ties()
    sim.sweeps(2, ALL)
    log = sim.tie_log()
    counts = sim.tie_counts()
    assert len(log) == counts.sum() > 20
    for r in range(sim.R):
        assert sum(1 for e in log if e[0] == r) == counts[r]
    assert {e[2] for e in log} <= {3, 4}
    assert {e[3] for e in log} == {0, 1}
    sim.clear_ties()
    assert sim.tie_log() == [] and sim.tie_counts().sum() == 0


def test_forcing_the_logged_outcomes_changes_nothing(orc):
    sim = _sim(orc)
    sim.sweeps(2, ALL)
    st = _state(sim)
    sim.set_tie_eps(0.5)
    sim.clear_ties()
    sim.sweeps(1, ALL)
    ref = sim.vectors().copy(), sim.labels().copy(), sim.energies().copy()
    log = sim.tie_log()
    assert len(log) > 50
    _restore(sim, st)
    sim.force([(r, v, a) for r, v, _, a in log])
    sim.sweeps(1, ALL)
    assert np.array_equal(sim.vectors(), ref[0])
    assert np.array_equal(sim.labels(), ref[1]) and np.array_equal(sim.energies(), ref[2])


def test_forced_reject_keeps_the_spin_and_forced_accept_takes_the_proposal(orc):
    sim = _sim(orc, u24=False)
    sim.sweeps(2, ALL)
    st = _state(sim)
    sim.set_tie_eps(1e9)  # every test is logged
    sim.clear_ties()
    sim.sweeps(1, 1)  # Metropolis only: each site is tested once
    unforced = sim.vectors().copy()
    log = sim.tie_log()
    assert len(log) == sim.R * sim.n
    accepted = [(r, v) for r, v, _, a in log if a == 1]
    rejected = [(r, v) for r, v, _, a in log if a == 0]
    assert accepted and rejected
    before = st[0]
    # an accepted move forced to reject: that spin keeps its value
    r, v = accepted[0]
    _restore(sim, st)
    sim.force([(r, v, 0)])
    sim.sweeps(1, 1)
    assert np.array_equal(sim.vectors()[r, v], before[r, v])
    assert not np.array_equal(unforced[r, v], before[r, v])
    # a rejected move forced to accept: the spin turns by the step the MET
    # stream gives, delta = Delta (2u - 1), u = u53(w0, w1) of block
    # (site, sweep, MET << 24 | replica, sample); Delta = 1.5 in every slot
    r, v = rejected[0]
    _restore(sim, st)
    sim.force([(r, v, 1)])
    sim.sweeps(1, 1)
    after = sim.vectors()[r, v]
    w = orc.philox([v, st[2], (2 << 24) | r, 3], [7, 0]).astype(np.uint64)
    u = float(((w[0] << np.uint64(32)) | w[1]) >> np.uint64(11)) / 2.0 ** 53
    delta = 1.5 * (2.0 * u - 1.0)
    turn = np.arctan2(after[1], after[0]) - np.arctan2(before[r, v, 1], before[r, v, 0])
    assert abs(np.angle(np.exp(1j * (turn - delta)))) < 1e-12
    assert np.array_equal(unforced[r, v], before[r, v])
    # forcing removed: the unforced run again, bit for bit
    _restore(sim, st)
    sim.force([])
    sim.sweeps(1, 1)
    assert np.array_equal(sim.vectors(), unforced)


def test_masked_run_updates_only_the_chosen_replicas(orc):
    sim = _sim(orc)
    sim.sweeps(2, ALL)
    st = _state(sim)
    sim.sweeps(1, OPS_MET_OR)
    full = sim.vectors().copy()
    _restore(sim, st)
    sim.set_active([1, 3])
    sim.sweeps(1, OPS_MET_OR)
    got = sim.vectors()
    assert np.array_equal(got[[1, 3]], full[[1, 3]])
    assert np.array_equal(got[[0, 2]], st[0][[0, 2]])
    sim.set_active(None)
    _restore(sim, st)
    sim.sweeps(1, OPS_MET_OR)
    assert np.array_equal(sim.vectors(), full)


def test_forced_pt_outcome_replaces_the_swap_decision(orc):
    sim = _sim(orc)
    sim.sweeps(5, ALL)
    # find a sweep whose PT step accepts some pair, then force that pair to reject
    for _ in range(40):
        st = _state(sim)
        before = sim.accumulators()["pt_acc"].copy()
        sim.sweeps(1, ALL)
        gained = np.flatnonzero(sim.accumulators()["pt_acc"] - before)
        if len(gained):
            break
    k = int(gained[0])
    labels_swapped = sim.labels().copy()
    _restore(sim, st)
    acc0 = sim.accumulators()["pt_acc"].copy()
    sim.force_pt([(k, 0)])
    sim.sweeps(1, ALL)
    lab = sim.labels()
    assert lab[k] == st[1][k] and lab[k + 1] == st[1][k + 1]
    assert lab[k] == labels_swapped[k + 1]
    assert sim.accumulators()["pt_acc"][k] == acc0[k]
    sim.force_pt([])
    # PT near-ties are logged with their pair
    sim.set_tie_eps(1.0)
    sim.clear_ties()
    sim.sweeps(2, ALL)
    log = sim.tie_log(pt=True)
    assert log and all(e[0] == -1 and 0 <= e[1] < sim.R - 1 for e in log)
