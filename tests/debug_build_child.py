"""Runs a list of small sweeps through whichever libxyl the environment selects
(XYL_DEBUG=1: the debug build) and saves their final states.  Imported by
tests/test_gpu_debug_build.py for the release run and executed by it as a
child process for the debug run, so both sides run the same code.

A case is (config name, engine name, tuning).  Each runs two samples of the
configuration's graph family (stream ids 0 and 1) for six sweeps of
Metropolis + overrelaxation + PT with a measurement every second sweep and an
FP64 recompute every third.  With corrupt=True the first neighbour id in
sample 0's CSR is set, in the bound workspace, to N + 1: one past the
last valid index of every engine (the resident shapes keep a zero row at N).
Every access that id could reach without the debug checks stays inside its
allocation (the next sample's spins or the regions that follow the spins; in
shared memory the arrays that follow the spin rows).
"""
from __future__ import annotations

import dataclasses
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

CASES = [
    ("C1", "FP64_PLAIN", {}),
    ("C1", "FP32_PLAIN", {}),
    ("C1", "FP32_BATCHED", {}),
    ("C1", "FP32_BATCHED", {"resident": -1}),
    ("C1", "FP32_BATCHED", {"resident": -1, "stage": -1, "block": 1024}),
    ("E1", "FP64_PLAIN", {}),
    ("E1", "FP32_BATCHED", {}),
    ("E1", "FP32_BATCHED", {"resident": -1, "stage": -1}),
    ("G1", "FP32_BATCHED", {}),
    ("H1", "FP32_PLAIN", {}),
    ("O1", "FP64_PLAIN", {}),
    ("O1", "FP32_PLAIN", {}),
    ("O1", "FP32_BATCHED", {"resident": 1}),
]


def two_samples(wl, name):
    cfg = wl.config(name)
    L, rho, _ = cfg.graphs[0]
    return dataclasses.replace(cfg, graphs=[(L, rho, 0), (L, rho, 1)])


def _corrupt_first_id(plan, graph):
    import torch
    _, _, col, _ = graph.csr()
    ws = plan.workspace.cpu().numpy().view(np.int32).copy()
    ids = ws & np.int32(0x7fffffff)  # the device CSR keeps a link's J = -1 in the top bit
    hits = np.flatnonzero(ids[: len(ws) - len(col)] == col[0])
    at = next(k for k in hits if np.array_equal(ids[k:k + len(col)], col))
    sign = ws[at] & np.int32(-2 ** 31)  # keep a random bond's sign bit
    ws[at] = sign | np.int32(graph.n + 1)
    plan.workspace.copy_(torch.from_numpy(ws.view(np.uint8)).to(plan.workspace.device))


def run_case(case, corrupt=False):
    """Final state bytes and status word of one case."""
    from paper_1211_3991_gb300 import workloads as wl, xyl
    name, engine, tune = case
    cfg = two_samples(wl, name)
    graphs = wl.build_graphs(cfg)
    plan, _ = wl.make_plan(cfg, getattr(xyl, engine), graphs=graphs, recompute_every=3, **tune)
    plan.bind()
    plan.init_spins()
    if corrupt:
        _corrupt_first_id(plan, graphs[0])
    plan.sweep(6, xyl.OP_MET | xyl.OP_OR | xyl.OP_PT | xyl.OP_MEASURE, 2)
    status, _ = plan.status()
    state = plan.export_state() if status == 0 else b""
    return state, status


def main(out_path, corrupt):
    from paper_1211_3991_gb300 import xyl
    assert xyl.LIB_PATH.endswith("libxyl_debug.so") == (os.environ.get("XYL_DEBUG") == "1")
    states, statuses = {}, []
    for k, case in enumerate(CASES):
        state, status = run_case(case, corrupt)
        states[f"case{k}"] = np.frombuffer(state, np.uint8)
        statuses.append(status)
    np.savez(out_path, statuses=np.array(statuses), lib=np.array(xyl.LIB_PATH), **states)


if __name__ == "__main__":
    main(sys.argv[1], json.loads(sys.argv[2]) if len(sys.argv) > 2 else False)
