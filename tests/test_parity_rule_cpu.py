"""The single-precision parity rule itself, checked on the CPU.

A stand-in for a GPU plan runs a second copy of the oracle (24-bit mode) with
one Metropolis decision planted the other way.  The rule of
``helpers.fp32_parity_sweeps`` must accept the run when the planted decision
is one the oracle logged as a near-tie (it traces the miss to that decision),
and must reject it when the planted decision was far from flipping.
"""
import numpy as np
import pytest

from helpers import FP32_TIE_EPS, fp32_parity_sweeps

ALL = 1 | 2 | 4 | 8
L = 32


class _OracleAsPlan:
    """The calls fp32_parity_sweeps makes on a plan, served by an oracle copy;
    `plant[t]` lists (replica, site, accept) decisions forced at sweep t."""

    def __init__(self, sim):
        self.sim = sim
        self.plant = {}

    def status(self):
        return 0, self.sim.sweep_index

    def labels(self):
        return self.sim.labels()

    def spins(self, s, r):
        return self.sim.vectors()[r]

    def energies(self):
        return self.sim.energies()

    def sweep(self, n, ops):
        for _ in range(n):
            self.sim.force(self.plant.get(self.sim.sweep_index, []))
            self.sim.sweeps(1, ops)
            self.sim.force([])


def _sim(orc):
    ei, ej, _, _ = orc.levy_graph(L, 6, 3.5, 1, 0)
    color, _ = orc.slo_color(L * L, ei, ej)
    betas = list(1.0 / np.geomspace(0.8, 1.6, 8))
    sim = orc.Sim(L * L, ei, ej, color, betas, [1.5] * 8, 2, sample=0, xy=orc.lattice_xy(L), L=L, u24=True)
    sim.init()
    return sim


def _first_tie(orc):
    """(sweep, replica, site, outcome) of the first logged near-tie decision."""
    sim = _sim(orc)
    sim.set_tie_eps(FP32_TIE_EPS)
    for _ in range(200):
        sim.clear_ties()
        sim.sweeps(1, ALL)
        log = sim.tie_log()
        if log:
            r, v, t, a = log[0]
            return t, r, v, a
    pytest.skip("no near-tie decision in 200 sweeps")


def _run_rule(orc, t, plant):
    gpu = _OracleAsPlan(_sim(orc))
    gpu.sim.sweeps(t, ALL)
    gpu.plant = {t: plant}
    ref = _sim(orc)
    return fp32_parity_sweeps(gpu, {0: ref}, [0], 2, ALL, lambda s: L * L, lambda s: slice(0, 8))


def test_unplanted_copy_agrees_without_tracing(orc):
    t, _, _, _ = _first_tie(orc)
    compared, traced, flipped, worst = _run_rule(orc, t, [])
    assert compared == 16 and traced == 0 and flipped == 0 and worst == 0.0


def test_flip_at_a_logged_near_tie_is_traced(orc):
    t, r, v, a = _first_tie(orc)
    compared, traced, flipped, _ = _run_rule(orc, t, [(r, v, 1 - a)])
    # the flip is visible in that replica and traced to exactly that decision
    assert compared == 16 and traced == 1 and flipped == 1


def test_flip_far_from_any_tie_is_rejected(orc):
    t, _, _, _ = _first_tie(orc)
    # a decision of sweep t that the log does not list, whose flip is visible
    probe = _sim(orc)
    probe.sweeps(t, ALL)
    st = (probe.vectors().copy(), probe.labels().copy())
    probe.set_tie_eps(1e9)
    probe.clear_ties()
    probe.sweeps(1, ALL)
    ref_E = probe.energies().copy()
    every = probe.tie_log()
    probe.set_tie_eps(FP32_TIE_EPS)
    probe.clear_ties()
    probe.set_vectors(st[0])
    probe.set_labels(st[1], t)
    probe.sweeps(1, ALL)
    ties = {(r, v) for r, v, _, _ in probe.tie_log()}
    chosen = None
    for r, v, _, a in every:
        if (r, v) in ties:
            continue
        probe.set_vectors(st[0])
        probe.set_labels(st[1], t)
        probe.force([(r, v, 1 - a)])
        probe.sweeps(1, ALL)
        probe.force([])
        if abs(probe.energies()[r] - ref_E[r]) / (L * L) > 1e-4:
            chosen = (r, v, 1 - a)
            break
    assert chosen is not None
    with pytest.raises(AssertionError):
        _run_rule(orc, t, [chosen])
