"""The multi-GPU path on CPU ranks (gloo, world size 2).

Disorder samples are independent, so ranks share no data during a run: each
rank takes its own samples (disjoint random streams, together covering the
batch) and only the timing is reduced (slowest rank, total units)."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, queue):
    import torch
    import torch.distributed as dist
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    from paper_1211_3991_gb300 import workloads as wl
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world, init_method=f"tcp://127.0.0.1:{port}")
    out = {}
    for name in ("C2", "C3", "C4"):
        sh = wl.shard(wl.config(name), rank, world)
        ids = [wl.graph_stream_id(sh, k) for k in range(sh.n_samples)]
        sizes = [L for L, _, _ in sh.graphs]
        gathered = [None] * world
        dist.all_gather_object(gathered, (ids, sizes))
        out[name] = gathered
    t, u = bench.reduce_over_ranks(1.0 + rank, 10 * (rank + 1), world, torch.device("cpu"))
    out["reduce"] = (t, u)
    queue.put((rank, out))
    dist.destroy_process_group()


def test_two_ranks_shard_samples_without_collectives():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    from paper_1211_3991_gb300 import workloads as wl
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    results = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for name in ("C2", "C3", "C4"):
        (ids0, sz0), (ids1, sz1) = results[0][name]
        assert not set(ids0) & set(ids1)
        full = wl.config(name)
        if full.n_samples >= 2:
            assert sorted(ids0 + ids1) == list(range(full.n_samples))
            assert sorted(sz0 + sz1) == sorted(L for L, _, _ in full.graphs)
        else:
            assert len(ids0) == len(ids1) == full.n_samples
    assert results[0]["reduce"] == results[1]["reduce"] == (2.0, 30.0)
