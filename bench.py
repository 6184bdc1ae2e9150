"""Benchmark: site-updates/s of the FP32 batched sampler vs the FP64 plain kernel.

One step = `sweeps_per_step` whole sweeps (Metropolis pass + overrelaxation pass
over every colour class, parallel-tempering swap attempt after every sweep, an
FP64 measurement every `measure_every` sweeps) of the workload's full batch.
Default workload C5: 128 Levy graphs, L=512 (262144 sites each), z=6, rho in
{2.5, 4.5}, 32 temperatures geometric in [1.5, 3.5]; C2 (one graph, L=128, 16
temperatures), C3 (768 graphs, L=64, 24 temperatures) and C4 (48 graphs of six
sizes L=32..192, 20 temperatures) are measured in the same run.  A
site-update is one Metropolis or one overrelaxation update of one spin of one
replica.

Prints ONE JSON line (rank 0).  `--impl reference` times the sequential CPU
oracle on the same workload instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "site-updates/s FP32-batched vs FP64-plain on one GB300; % of memory roofline"
UNIT = "site-updates/s"
OPS_ALL = 1 | 2 | 4 | 8
L2_FLUSH_BYTES = 256 << 20
# algorithmic bytes per site-update (FP32 float2 spins, z = 6, R replicas sharing one CSR):
# compulsory HBM model = own spin read 8 B + write 8 B + 6 x 4 B of indices / R
# L2-level gather model = (z + 1) spin reads + 1 write (8 B each) + 6 x 4 B of indices / R
def hbm_bytes_per_update(R, dim=2):
    """Compulsory bytes of one site-update: the spin read and written once
    (8 B FP32 XY, 16 B for an O(3) spin padded to a 4-vector), the site's
    tables (24 B) once per sweep shared by the R replicas."""
    return 2.0 * (8.0 if dim == 2 else 16.0) + 24.0 / R


def l2_bytes_per_update(R, dim=2):
    return 64.0 * (1.0 if dim == 2 else 2.0) + 24.0 / R


def _env_rank():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("LOCAL_RANK", "0"))


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi samples of SM clocks and throttle reasons during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.proc = None
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(device_index)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


KERNEL_SOURCES = {
    "batched_kernel": ["batched.cu"],
    "resident_kernel": ["resident.cu"],
    "o3_phase_kernel": ["o3.cu", "o3_f32.cuh"],
    "resident_o3_kernel": ["resident_o3.cu", "o3_f32.cuh"],
    "walk_kernel": ["walk.cu"],
    "plain_phase_kernel": ["plain.cu"],
}
SHARED_SOURCES = ["engines.h", "device.cuh", "philox.cuh", "sweep_tail.cuh"]


def kernel_source_digest(kernel):
    """SHA-256 over a kernel's source file and the headers it includes."""
    h = hashlib.sha256()
    for f in KERNEL_SOURCES[kernel] + SHARED_SOURCES:
        h.update(open(os.path.join(ROOT, "paper_1211_3991_gb300", "csrc", f), "rb").read())
    return h.hexdigest()


def _profile_values(kernel, config):
    """The machine-read lines ("- key: value") of the committed ncu summary of
    `kernel` on `config`, or None once the kernel's sources have changed since
    the capture."""
    path = os.path.join(ROOT, "profiles", f"{kernel}_{config}.md")
    if not os.path.exists(path) or kernel not in KERNEL_SOURCES:
        return None
    vals = {}
    for line in open(path):
        if ":" in line and line.startswith("- "):
            k, v = line[2:].split(":", 1)
            vals[k.strip()] = v.strip().strip("`")
    if vals.get("source_sha256") != kernel_source_digest(kernel):
        return None
    return vals


def _profile_traffic(kernel, config):
    """DRAM bytes per launch of `kernel` on `config` from the committed ncu
    summary, valid only while the kernel's sources are unchanged since the capture."""
    vals = _profile_values(kernel, config)
    if vals is None:
        return None
    try:
        out = {"bytes_per_launch": float(vals["dram_bytes_per_launch"]),
               "scales": not vals.get("traffic_scales_with_sweeps", "yes").startswith("no"),
               "sweeps_per_launch": float(vals["sweeps_per_launch"])}
        if "site_updates_per_launch" in vals:
            out["updates_per_launch"] = float(vals["site_updates_per_launch"])
        return out
    except (KeyError, ValueError):
        return None


def reduce_over_ranks(elapsed, units, world, device):
    """Whole-job figures: the slowest rank's time and the units all ranks did."""
    if world <= 1:
        return float(elapsed), float(units)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(elapsed)], dtype=torch.float64, device=device)
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def run_oracle_sample(cfg, sweeps=0, seconds=0.0, measure_every=32, chunk=25, max_seconds=30.0, sample_index=0):
    """The sequential FP64 oracle on one sample of the workload, one host thread:
    `sweeps` sweeps, or (sweeps = 0) chunks of `chunk` sweeps until at least
    `seconds` (at most `max_seconds`) have passed.  Graph construction is not
    timed.  Returns (site-updates, seconds, sweeps run)."""
    import oracle
    from paper_1211_3991_gb300 import workloads as wl
    L, rho, _ = cfg.graphs[sample_index]
    if cfg.ensemble == "bonds":
        ei, ej, _ = oracle.levy_bonds(L, rho, wl.GRAPH_SEED, wl.graph_stream_id(cfg, sample_index),
                                      fbc=cfg.boundary == "fbc")
    else:
        ei, ej, _, _ = oracle.levy_graph(L, wl.Z, rho, wl.GRAPH_SEED, wl.graph_stream_id(cfg, sample_index))
    color, _ = oracle.slo_color(L * L, ei, ej)
    sim = oracle.Sim(L * L, ei, ej, color, cfg.betas(), cfg.deltas(), wl.SPIN_SEED, sample=wl.graph_stream_id(cfg, sample_index),
                     xy=oracle.lattice_xy(L), L=L, dim=cfg.spin_dim)
    J = wl.couplings_for(cfg, sample_index, len(ei))
    if J is not None:
        sim.set_couplings(J.astype(float))
    h = wl.fields_for(cfg, sample_index, L * L)
    if h is not None:
        sim.set_fields(h)
    sim.init()
    done, dt = 0, 0.0
    while True:
        n = sweeps - done if sweeps > 0 else chunk
        t0 = time.perf_counter()
        sim.sweeps(n, OPS_ALL, measure_every)
        dt += time.perf_counter() - t0
        done += n
        if sweeps > 0 or dt >= seconds or dt >= max_seconds:
            break
    sim.close()
    return L * L * cfg.n_temps * 2 * done, dt, done


def _oracle_worker(job):
    name, k, sweeps, seconds, measure_every = job
    from paper_1211_3991_gb300 import workloads as wl
    return run_oracle_sample(wl.config(name), sweeps=sweeps, seconds=seconds, measure_every=measure_every,
                             sample_index=k)


def run_oracle_parallel(cfg, seconds, measure_every, procs, sweeps=0):
    """The oracle on samples 0..procs-1 of a multi-sample workload, one process
    per sample on the host cores (spawned, so safe after GPU work), all running
    at once: `sweeps` sweeps each, or (sweeps = 0) about `seconds` each.
    Returns (site-updates/s summed over processes, [(site-updates, seconds,
    sweeps)] per process)."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    with ctx.Pool(procs) as pool:
        res = pool.map(_oracle_worker, [(cfg.name, k, sweeps, seconds, measure_every) for k in range(procs)])
    return sum(u / dt for u, dt, _ in res), res


def _oracle_steps_worker(job):
    """One oracle process: build sample k once, then warm-up and timed chunks
    of `sweeps` sweeps; returns (site-updates per chunk, [seconds per timed chunk])."""
    name, max_samples, k, sweeps, warmup, steps, measure_every = job
    import oracle
    from paper_1211_3991_gb300 import workloads as wl
    cfg = wl.config(name)
    if max_samples > 0:
        cfg = wl.first_samples(cfg, max_samples)
    L, rho, _ = cfg.graphs[k]
    if cfg.ensemble == "bonds":
        ei, ej, _ = oracle.levy_bonds(L, rho, wl.GRAPH_SEED, wl.graph_stream_id(cfg, k), fbc=cfg.boundary == "fbc")
    else:
        ei, ej, _, _ = oracle.levy_graph(L, wl.Z, rho, wl.GRAPH_SEED, wl.graph_stream_id(cfg, k))
    color, _ = oracle.slo_color(L * L, ei, ej)
    sim = oracle.Sim(L * L, ei, ej, color, cfg.betas(), cfg.deltas(), wl.SPIN_SEED, sample=wl.graph_stream_id(cfg, k),
                     xy=oracle.lattice_xy(L), L=L, dim=cfg.spin_dim)
    J = wl.couplings_for(cfg, k, len(ei))
    if J is not None:
        sim.set_couplings(J.astype(float))
    h = wl.fields_for(cfg, k, L * L)
    if h is not None:
        sim.set_fields(h)
    sim.init()
    for _ in range(warmup):
        sim.sweeps(sweeps, OPS_ALL, measure_every)
    times = []
    for _ in range(steps):
        t0 = time.perf_counter()
        sim.sweeps(sweeps, OPS_ALL, measure_every)
        times.append(time.perf_counter() - t0)
    sim.close()
    return L * L * cfg.n_temps * 2 * sweeps, times


def reference_arm(args, cfg):
    """The oracle as it stands on the host cores: one process per independent
    sample (one sample: one core), each building its sample once, then
    `warmup` + `steps` chunks of sweeps (about a second each); the rate is the
    sum of the processes' rates."""
    rank, world, _ = _env_rank()
    if rank != 0:
        return
    import multiprocessing as mp
    import oracle
    oracle.build()
    procs = min(cfg.n_samples, os.cpu_count() or 1)
    per_sweep = 2 * cfg.spins_per_sweep() / cfg.n_samples
    per_step = args.ref_sweeps or int(max(1, round(2.5e7 / per_sweep)))
    jobs = [(cfg.name, args.max_samples, k, per_step, args.warmup, args.steps, args.measure_every) for k in range(procs)]
    with mp.get_context("spawn").Pool(procs) as pool:
        res = pool.map(_oracle_steps_worker, jobs)
    value = sum(u * len(t) / sum(t) for u, t in res)
    ms_step = 1e3 * max(sum(t) for _, t in res) / args.steps
    sample = (f"{per_step} sweeps of sample 0 of {cfg.name} ({cfg.description}) per step" if procs == 1 else
              f"{per_step} sweeps of each of samples 0..{procs - 1} of {cfg.name}, one process each, per step")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"{cfg.name}: {cfg.description}", "engine": "sequential FP64 CPU oracle"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": procs, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


WALK_METRIC = "walker-steps/s of simple random walks (spectral dimension, App. A)"


def walk_bench(args):
    """Random walks on one 2N-bond Levy graph (L=512, rho=10/3, periodic): each
    step of a walker reads its node's CSR row bounds and one neighbour id
    (12 B of algorithmic gathers, two dependent loads).  Walkers start on random
    nodes of degree > 2 (the paper's rule for rho <= 4)."""
    import numpy as np
    import torch
    import torch.distributed as dist
    from paper_1211_3991_gb300 import build as libbuild
    libbuild.build()
    from paper_1211_3991_gb300 import xyl
    rank, world, local = _env_rank()
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    L, rho, W, T = 512, 10.0 / 3.0, args.walkers, args.walk_steps
    g = xyl.build_levy_bonds(L, rho, 1, rank)
    _, row_ptr, col, _ = g.csr()
    start = np.random.default_rng(rank).choice(np.flatnonzero(np.diff(row_ptr) > 2), W).astype(np.int32)
    rp, cl = torch.from_numpy(row_ptr).to(dev), torch.from_numpy(col).to(dev)
    st = torch.from_numpy(start).to(dev)
    out = torch.empty(T + 1, dtype=torch.int64, device=dev)
    stream = torch.cuda.current_stream()
    for k in range(args.warmup):
        xyl.walk_returns(rp, cl, st, T, 1000 + k, out, stream=stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = ClockSampler(local)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for k in range(args.steps):
        xyl.walk_returns(rp, cl, st, T, 2000 + k, out, first_walker=0, stream=stream)
    b.record(stream)
    b.synchronize()
    clock_info = clocks.stop()
    ms = a.elapsed_time(b)
    max_ms, units = reduce_over_ranks(ms, float(W) * T * args.steps, world, dev)
    value = units / (max_ms / 1e3)
    # end to end: start nodes host -> device and the return histogram back, every step
    host_start = torch.from_numpy(start).pin_memory()
    host_out = torch.empty(T + 1, dtype=torch.int64).pin_memory()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(args.steps):
        st.copy_(host_start, non_blocking=True)
        xyl.walk_returns(rp, cl, st, T, 3000 + k, out, stream=stream)
        host_out.copy_(out, non_blocking=True)
        torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e_max, e2e_units = reduce_over_ranks(e2e_s, float(W) * T * args.steps, world, dev)
    peak, peak_kind = _peaks()
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        import oracle
        # chunks of 20000 walkers until about 10 s of oracle time
        n_cpu, dt, chunk = 0, 0.0, 20000
        while dt < 10.0 and n_cpu + chunk <= W:
            t1 = time.perf_counter()
            oracle.walk_returns(row_ptr, col, start[n_cpu:n_cpu + chunk], T, 5)
            dt += time.perf_counter() - t1
            n_cpu += chunk
        cpu = {"value": n_cpu * T / dt, "unit": "walker-steps/s", "cores": 1, "kind": "oracle",
               "sample": f"{n_cpu} of the walkers, {T} steps ({dt:.1f} s, one thread)"}
    # DRAM bytes of one launch from the committed ncu summary (one launch = one step of W walkers)
    prof = _profile_traffic("walk_kernel", "walk")
    walk_traffic = prof["bytes_per_launch"] if prof and W == 1 << 20 and T == 1000 else None
    if rank == 0:
        print(json.dumps({
            "metric": WALK_METRIC, "value": value, "unit": "walker-steps/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": max_ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": f"one 2N-bond Levy graph per rank, L={L}, rho=10/3, periodic; {W} walkers x {T} "
                       "steps per step, starts on nodes of degree > 2", "l2": "CSR (5 MB) L2-resident by design"},
            "roofline": {"bound": "hbm", "achieved": 12.0 * value / world / 1e9, "peak": peak, "unit": "GB/s",
                         "frac": 12.0 * value / world / 1e9 / peak, "traffic": walk_traffic, "peak_kind": peak_kind,
                         "bytes_per_update": 12.0, "kernel": "walk_kernel",
                         "note": "two dependent L2 gathers per step: latency-bound, not HBM-bound"},
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_units / e2e_max, "unit": "walker-steps/s", "h2d_bytes_per_step": int(start.nbytes),
                    "d2h_bytes_per_step": int(8 * (T + 1))},
            "gpu_launches": args.steps,
            "clocks": clock_info,
        }), flush=True)
    if world > 1:
        dist.destroy_process_group()


# Secondary ceilings measured on this GB300 by the project's own probes (CUDA
# events, 2.07 GHz): MEASURED_PEAKS.json holds only the HBM copy and BF16 GEMM.
# on-chip peaks, measured by `python bench.py --probe-peaks` (paper_1211_3991_gb300/peaks.py) on a GB300
SMEM_GATHER_PROBE_GBS = 15000.0  # random 8-byte gathers from shared memory, 128 KB per CTA, every SM
L2_STREAM_PROBE_GBS = 19300.0    # streaming reads of a 64 MiB L2-resident buffer
L2_BYTES = 126 << 20             # L2 capacity usable for a resident working set


def roofline_for(plan, cfg, per_launch_updates, avg_launch_s, name, spins_live_bytes):
    """Roofline of the kernel a plan runs, against the ceiling its schedule
    meets: spins held in shared memory for a whole launch -> on-chip gather
    model vs the shared-memory gather probe; spins in global memory with a
    launch wave's spins within L2 -> L2 gather model vs the L2 probe; else the
    compulsory HBM model vs the measured HBM copy bandwidth."""
    R, dim = cfg.n_temps, cfg.spin_dim
    kernel = kernel_name(plan)
    hbm_peak, hbm_kind = _peaks()
    models = {"hbm_compulsory": hbm_bytes_per_update(R, dim), "gather": l2_bytes_per_update(R, dim)}
    if kernel == "resident_o3_kernel":
        # three 4-byte components per spin in shared memory: 7 reads + 1 write of 12 B
        models["gather"] = 96.0 + 24.0 / R
    achieved = {k: b * per_launch_updates / avg_launch_s / 1e9 for k, b in models.items()}
    if kernel in ("resident_kernel", "resident_o3_kernel"):
        bound, b, peak, kind = "smem", models["gather"], SMEM_GATHER_PROBE_GBS, \
            "own probe: shared-memory random 8-byte gathers"
        spin_b = 12 if kernel == "resident_o3_kernel" else 8
        basis = (f"spins held in shared memory for the whole launch: (z+1) {spin_b}-B spin reads + one {spin_b}-B "
                 "write per update")
    elif spins_live_bytes <= L2_BYTES:
        bound, b, peak, kind = "l2", models["gather"], L2_STREAM_PROBE_GBS, "own probe: L2-resident stream read"
        basis = f"the spins resident at once ({spins_live_bytes / 2**20:.0f} MiB) stay in L2: gather model"
    else:
        bound, b, peak, kind = "hbm", models["hbm_compulsory"], hbm_peak, hbm_kind
        basis = (f"the spins resident at once ({spins_live_bytes / 2**30:.2f} GiB) exceed L2: compulsory model, each "
                 "spin read and written once per pass")
    a = b * per_launch_updates / avg_launch_s / 1e9
    prof = _profile_traffic(kernel, name)
    traffic = None
    if prof is not None:
        # DRAM bytes of the captured launch, scaled to this launch by its site-updates
        # (a capture of a subset of the workload) unless they do not grow with it
        if not prof["scales"]:
            traffic = prof["bytes_per_launch"]
        elif "updates_per_launch" in prof:
            traffic = prof["bytes_per_launch"] * per_launch_updates / prof["updates_per_launch"]
        else:
            traffic = prof["bytes_per_launch"] * per_launch_updates / (cfg.spins_per_sweep() * 2) / \
                prof["sweeps_per_launch"]
    out = {"bound": bound, "achieved": a, "peak": peak, "unit": "GB/s", "frac": a / peak, "traffic": traffic,
           "peak_kind": kind, "bytes_per_update": b, "kernel": kernel, "basis": basis,
           "other_models_GBps": {k: v for k, v in achieved.items()}}
    if traffic is not None:
        # the DRAM rate the measured traffic implies at this launch's duration
        out["dram_GBps_from_traffic"] = traffic / avg_launch_s / 1e9
        out["dram_frac_of_measured_hbm"] = out["dram_GBps_from_traffic"] / hbm_peak
        out["dram_bytes_per_update"] = traffic / per_launch_updates
    return out


def fp64_bound(name):
    """What bounds the FP64 plain engine on this workload, from the committed
    ncu summary of its phase kernel (while its sources are unchanged): the FP64
    pipe's active fraction, time-weighted over the launches of one sweep."""
    vals = _profile_values("plain_phase_kernel", name)
    if vals is None or "fp64_pipe_active_pct" not in vals:
        return {"fp64_pipe_active": None}
    return {"fp64_pipe_active": float(vals["fp64_pipe_active_pct"]) / 100.0,
            "bound": "FP64 pipe (ncu sm__pipe_fp64_cycles_active, time-weighted over one sweep)",
            "profile": f"profiles/plain_phase_kernel_{name}.md"}


def spins_live_bytes(plan, cfg):
    """Bytes of spins the units resident on the GPU at once keep live: a launch
    wave's units when they wait on one another, else as many clusters as fit
    (each runs all of a launch's sweeps while resident); the plain engines
    keep the whole batch live."""
    units = plan.unit_count()
    frac = 1.0
    if units and plan.part_count() == 1:
        frac = min(1.0, plan.live_units() / units)
    return frac * cfg.spins_per_sweep() * (8 if cfg.spin_dim == 2 else 16)


def measure_workload(args, name, xyl, wl, dev, stream, flush, rank, world, steps, warmup, full):
    """Time one workload: FP32 sampler (Delta tuned in the library, launch shape
    autotuned), the FP64 plain engine on the same batch, and, for the headline
    workload (full=True), the end-to-end loop and the clock record."""
    import numpy as np
    import torch
    cfg = wl.config(name)
    if args.max_samples > 0:
        cfg = wl.first_samples(cfg, args.max_samples)
    # every rank runs its own disorder realisations; no data-path collective
    cfg = wl.shard(cfg, rank, world)
    graphs = wl.build_graphs(cfg)
    engine_name = "FP32_BATCHED"
    tune = dict(block=args.block, cluster=args.cluster, group=args.group, resident=args.resident, waves=args.waves,
                span=args.span)
    if not full:
        tune = {}
    plan, _ = wl.make_plan(cfg, getattr(xyl, engine_name), graphs=graphs, **tune)
    plan.bind(stream)
    plan.init_spins(stream=stream)
    explicit = full and (args.block or args.cluster or args.group)
    autotune_s, shape_source = None, "library default"
    if explicit:
        shape_source = "command line"
    elif engine_name == "FP32_BATCHED" and not args.no_autotune:
        t0 = time.perf_counter()
        n_try = args.autotune_sweeps or int(min(64, max(4, round(2e9 / (2 * cfg.spins_per_sweep())))))
        if args.autotune_cache:
            _, hit = plan.autotune_cached(args.autotune_cache, n_try, OPS_ALL, args.measure_every, stream=stream)
            shape_source = "autotune cache (shapes xyl_autotune chose for this batch signature)" if hit else "autotuned"
        else:
            plan.autotune(n_try, OPS_ALL, args.measure_every, stream=stream)
            shape_source = "autotuned"
        autotune_s = time.perf_counter() - t0
    # Metropolis half-widths: warm-up to about 50% acceptance in the chosen shape, then frozen
    rates = None
    if not args.no_tune_delta:
        rates = plan.tune_delta(rounds=args.tune_rounds, n_sweeps=args.tune_sweeps, ops=1 | 2 | 4, stream=stream)
    updates_per_sweep = cfg.spins_per_sweep() * 2

    def timed_steps(p, n_steps, sweeps):
        total_ms, launches = 0.0, 0
        for _ in range(n_steps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            p.sweep(sweeps, OPS_ALL, args.measure_every, stream=stream)
            b.record(stream)
            b.synchronize()
            total_ms += a.elapsed_time(b)
            launches += p.last_launch_count()
        return total_ms, launches

    # calibrate the step length (about 50 ms, at least min_sweeps sweeps)
    sweeps = args.sweeps_per_step if full else 0
    if sweeps <= 0:
        probe = max(2, args.min_sweeps)
        ms, _ = timed_steps(plan, 1, probe)
        sweeps = int(min(20000, max(args.min_sweeps, round(50.0 / max(ms / probe, 1e-6)))))
    for _ in range(warmup):
        timed_steps(plan, 1, sweeps)

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    barrier()
    clocks = ClockSampler(torch.cuda.current_device()) if full else None
    total_ms, launches = timed_steps(plan, steps, sweeps)
    clock_info = clocks.stop() if clocks else None
    barrier()
    max_ms, units = reduce_over_ranks(total_ms, updates_per_sweep * sweeps * steps, world, dev)
    value = units / (max_ms / 1e3)

    e2e = None
    if full:
        # end to end through the public API with host buffers: per step the slot
        # half-widths go host->device, the step's measurements come back device->host
        deltas = [plan.get_delta(s) for s in range(cfg.n_samples)]
        h2d = d2h = 0
        barrier()
        t0 = time.perf_counter()
        for _ in range(steps):
            for s in range(cfg.n_samples):
                plan.set_delta(s, deltas[s], stream=stream)
            h2d = sum(d.nbytes for d in deltas)
            plan.sweep(sweeps, OPS_ALL, args.measure_every, stream=stream)
            obs = plan.read_observables(stream=stream)
            d2h = sum(v.nbytes for v in obs.values())
            plan.reset_observables(stream=stream)
        barrier()
        e2e_s = time.perf_counter() - t0
        e2e_max_s, e2e_units = reduce_over_ranks(e2e_s, updates_per_sweep * sweeps * steps, world, dev)
        e2e = {"value": e2e_units / e2e_max_s, "unit": UNIT,
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)}

    status, _ = plan.status(stream=stream)
    if status != 0:
        raise SystemExit(f"device status {status}")

    # FP64 plain kernel on the same workload and GPU, same half-widths
    fp64 = None
    if not args.no_fp64:
        p64, _ = wl.make_plan(cfg, xyl.FP64_PLAIN, graphs=graphs)
        p64.bind(stream)
        for s in range(cfg.n_samples):
            p64.set_delta(s, plan.get_delta(s), stream=stream)
        p64.init_spins(stream=stream)
        ms1, _ = timed_steps(p64, 1, 2)
        s64 = int(max(2, min(sweeps, round(100.0 / max(ms1 / 2, 1e-6)))))
        n64 = max(3, min(steps, 5))
        ms64, _ = timed_steps(p64, n64, s64)
        fp64 = updates_per_sweep * s64 * n64 / (ms64 / 1e3)
        del p64

    avg_launch_s = (total_ms / 1e3) / max(1, launches)
    per_launch_updates = updates_per_sweep * sweeps * steps / max(1, launches)
    roof = roofline_for(plan, cfg, per_launch_updates, avg_launch_s, name, spins_live_bytes(plan, cfg))
    out = {
        "value": value, "ms_per_step": max_ms / steps, "sweeps_per_step": sweeps, "launches": int(launches),
        "workload": f"{cfg.name}: {cfg.description}", "engine": engine_name, "cluster": plan_shape(plan),
        "samples": cfg.n_samples, "temperatures": cfg.n_temps,
        "fp64_plain": {"value": fp64, "unit": UNIT,
                       "ratio_fp32_batched_over_fp64_plain": (value / world / fp64) if fp64 else None,
                       **fp64_bound(name)},
        "roofline": roof, "e2e": e2e, "clocks": clock_info, "autotune_s": autotune_s, "shape_source": shape_source,
    }
    if rates is not None:
        out["metropolis_acceptance"] = {"tuned_to": 0.5, "min": float(np.min(rates)), "max": float(np.max(rates)),
                                        "per_slot_sample0": [round(float(x), 3) for x in rates[:cfg.n_temps]],
                                        "delta_sample0": [round(float(x), 4) for x in plan.get_delta(0)]}
    del plan
    return out, cfg


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="C5")
    ap.add_argument("--extra-configs", default="C2,C3,C4",
                    help="comma-separated workloads also measured (shorter) and reported in the same line; '' = none")
    ap.add_argument("--extra-steps", type=int, default=5)
    ap.add_argument("--sweeps-per-step", type=int, default=0, help="0 = calibrate to about 50 ms per step")
    ap.add_argument("--min-sweeps", type=int, default=8, help="least sweeps per step when calibrating")
    ap.add_argument("--block", type=int, default=0)
    ap.add_argument("--cluster", type=int, default=0)
    ap.add_argument("--group", type=int, default=0)
    ap.add_argument("--resident", type=int, default=0, choices=[-1, 0, 1],
                    help="1 = spins in shared memory for a launch, -1 = global-memory shape, 0 = library/autotuner")
    ap.add_argument("--waves", type=int, default=0, choices=[-1, 0, 1],
                    help="global-memory shape: 1 = launch waves sized to L2, -1 = never, 0 = library/autotuner")
    ap.add_argument("--span", type=int, default=0,
                    help="global-memory shape: clusters per replica group (0 = library/autotuner)")
    ap.add_argument("--ref-sweeps", type=int, default=0,
                    help="oracle sweeps per step of --impl reference (0 = about 1 s of the workload's sample)")
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="CPU-baseline sample: oracle time to run")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--autotune-sweeps", type=int, default=0,
                    help="sweeps per timed try of the autotuner (0 = about 2e9 site-updates, 4 to 64)")
    ap.add_argument("--autotune-cache", default=os.path.join(ROOT, "paper_1211_3991_gb300", "autotune_cache.json"),
                    help="JSON file of launch shapes by batch signature ('' = always autotune)")
    ap.add_argument("--no-tune-delta", action="store_true")
    ap.add_argument("--tune-rounds", type=int, default=6)
    ap.add_argument("--tune-sweeps", type=int, default=40)
    ap.add_argument("--measure-every", type=int, default=32, help="sweeps between measurements (the paper: 32)")
    ap.add_argument("--probe-peaks", action="store_true",
                    help="measure the on-chip peaks the roofline uses (paper_1211_3991_gb300/peaks.py) and exit")
    ap.add_argument("--workload", default="sweep", choices=["sweep", "walk"],
                    help="sweep: the Monte Carlo sampler (default); walk: random walks for the spectral dimension")
    ap.add_argument("--max-samples", type=int, default=0,
                    help="run only the first N samples of the workload (0 = all), e.g. for a profiler capture")
    ap.add_argument("--walkers", type=int, default=1 << 20)
    ap.add_argument("--walk-steps", type=int, default=1000)
    args = ap.parse_args()
    if args.probe_peaks:
        # the on-chip peaks of the roofline (L2 stream, shared-memory gathers), measured here
        from paper_1211_3991_gb300 import peaks
        print(json.dumps({"probe": "on-chip peaks", **peaks.measure(),
                          "used_by_roofline": {"l2_stream_read_GBps": L2_STREAM_PROBE_GBS,
                                               "smem_random_8B_gather_GBps": SMEM_GATHER_PROBE_GBS}}))
        return
    if args.workload == "walk":
        if args.impl == "reference":
            raise SystemExit("--impl reference times the sampler workload only")
        walk_bench(args)
        return

    from paper_1211_3991_gb300 import workloads as wl
    if args.impl == "reference":
        cfg = wl.config(args.config)
        if args.max_samples > 0:
            cfg = wl.first_samples(cfg, args.max_samples)
        reference_arm(args, cfg)
        return

    import torch
    import torch.distributed as dist
    from paper_1211_3991_gb300 import build as libbuild
    libbuild.build()
    from paper_1211_3991_gb300 import xyl

    rank, world, local = _env_rank()
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)

    head, cfg = measure_workload(args, args.config, xyl, wl, dev, stream, flush, rank, world, args.steps,
                                 args.warmup, True)
    extras = {}
    for name in [n for n in args.extra_configs.split(",") if n and n != args.config]:
        res, _ = measure_workload(args, name, xyl, wl, dev, stream, flush, rank, world, args.extra_steps,
                                  min(args.warmup, 3), False)
        extras[name] = {k: res[k] for k in ("value", "ms_per_step", "sweeps_per_step", "workload", "cluster",
                                            "fp64_plain", "roofline", "metropolis_acceptance", "shape_source")
                        if k in res}

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        if cfg.n_samples > 1:
            # independent samples: one oracle process per host core
            procs = min(cfg.n_samples, os.cpu_count() or 1)
            rate, res = run_oracle_parallel(cfg, args.cpu_seconds, args.measure_every, procs)
            n_sw = [n for _, _, n in res]
            cpu = {"value": rate, "unit": UNIT, "cores": procs, "kind": "oracle",
                   "sample": f"samples 0..{procs - 1} of {cfg.name}, one process each, about {args.cpu_seconds:.0f} s "
                             f"each ({min(n_sw)}-{max(n_sw)} sweeps), rates summed"}
        else:
            ups, secs, n_sw = run_oracle_sample(cfg, seconds=args.cpu_seconds, measure_every=args.measure_every)
            cpu = {"value": ups / secs, "unit": UNIT, "cores": 1, "kind": "oracle",
                   "sample": f"{n_sw} sweeps of sample 0 of {cfg.name} ({ups} site-updates, {secs:.1f} s, one thread)"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": head["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": head["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": head["workload"], "engine": head["engine"],
                       "sweeps_per_step": head["sweeps_per_step"], "samples_on_rank0": head["samples"],
                       "temperatures": head["temperatures"],
                       "l2": "flushed (256 MiB write) between timed steps",
                       "measure_every": args.measure_every,
                       "cluster": head["cluster"], "parallelism": f"dp{world} (independent samples per rank)"},
            "fp64_plain": head["fp64_plain"],
            "roofline": head["roofline"],
            "metropolis_acceptance": head.get("metropolis_acceptance"),
            "cpu_baseline": cpu,
            "e2e": head["e2e"],
            "gpu_launches": head["launches"],
            "clocks": head["clocks"],
            "autotune_s": head["autotune_s"],
            "shape_source": head["shape_source"],
            "extra_configs": extras,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def plan_shape(plan):
    from paper_1211_3991_gb300 import xyl
    if plan.engine != xyl.FP32_BATCHED:  # plain engines: one launch per colour phase, 256 threads per CTA
        return {"plain": True, "threads_per_cta": 256}
    t = plan.tuning()
    out = {"spins_in_shared_memory": t["resident"] > 0, "units": plan.unit_count(), "replicas_per_group": t["group"],
           "ctas_per_cluster": t["cluster"], "threads_per_cta": t["block"], "csr_in_shared_memory": t["stage"] > 0,
           "l2_sized_waves": t["waves"] > 0, "clusters_per_group": t["span"], "units_per_launch": plan.wave_units()}
    if plan.part_count() > 1:
        # a mixed-size batch: one launch shape per size, largest first (the keys above are part 0's)
        out["parts"] = [plan.part_tuning(k) for k in range(plan.part_count())]
    return out


def kernel_name(plan):
    from paper_1211_3991_gb300 import xyl
    if plan.engine != xyl.FP32_BATCHED:
        return "o3_phase_kernel" if plan.dim == 3 else "plain_phase_kernel"
    if plan.dim == 3:
        return "resident_o3_kernel"
    return "resident_kernel" if plan.tuning()["resident"] > 0 else "batched_kernel"


if __name__ == "__main__":
    main()
