"""Synthetic workloads: graph sizes, decay exponents, temperature grids, seeds.

Pure configuration (no method arithmetic), shared by the benchmark and the
tests.  The paper measures on synthetic Levy graphs of its own ensemble only
(Sec. IV: L = 16..384, 2^21 sweeps, measurements every 32 sweeps); these
configurations keep its structure at the sizes the benchmark names:

  C1  one graph, L=16, z=6, rho=3.5, one temperature T=1.0
  C2  one graph, L=128, z=6, rho=3.5, 16 temperatures geometric in [0.8, 1.6], PT every sweep
  C3  256 graphs per rho in {2.5, 3.5, 4.5}, L=64, 24 temperatures geometric in [1.5, 3.5]
  C4  8 graphs per L in {32, 48, 64, 96, 128, 192}, rho=3.0, 20 temperatures in [1.5, 3.5], FP64 recompute every 100 sweeps
  C5  64 graphs per rho in {2.5, 4.5}, L=512, 32 temperatures in [1.5, 3.5]

The paper's own graph ensemble (Sec. II: 2N bonds, free degrees, periodic or
free boundaries) at small sizes for parity checks:

  E1  one graph, L=16, rho=0 (Erdos-Renyi limit), periodic, 4 temperatures geometric in [1.6, 2.4]
  E2  one graph, L=16, rho=7/3, free boundaries, 4 temperatures geometric in [1.6, 2.4]
  B64 64 graphs, L=64, rho=10/3 (long-range regime), periodic, 12 temperatures geometric in [1.4, 2.0]

Random bonds (the method's random-bond variant, App. B): C1's and C2's graphs
with J = +-1 at random (probability 1/2 each, the XY spin glass):

  G1  L=16, rho=3.5, 4 temperatures geometric in [0.4, 1.0]
  G2  L=128, rho=3.5, 16 temperatures geometric in [0.3, 1.2]
  H1  G1 with random fields of magnitude 0.5 (uniform random directions)
  H2  G2 with random fields of magnitude 0.5
  O1  C1's graph with O(3) spins, 4 temperatures geometric in [0.9, 1.8]
  O2  C2's graph with O(3) spins, 16 temperatures geometric in [0.9, 1.8]
  O2G O2 with random +-1 couplings, 16 temperatures geometric in [0.4, 1.2]
  OH1 O1's graph with random +-1 couplings and random 3-vector fields of magnitude 0.5, 4 temperatures in [0.4, 1.2]
  OH2 O2G with random 3-vector fields of magnitude 0.5
  O3  256 graphs L=64 (rho=3.5) with O(3) spins, 24 temperatures geometric in [0.9, 1.8]
"""
from __future__ import annotations

import concurrent.futures as cf
import math
import os
from dataclasses import dataclass, field

Z = 6
GRAPH_SEED = 1
SPIN_SEED = 2


def geometric_temperatures(t_min: float, t_max: float, n: int):
    if n == 1:
        return [t_min]
    return [t_min * (t_max / t_min) ** (k / (n - 1)) for k in range(n)]


@dataclass
class Config:
    name: str
    graphs: list            # (L, rho, sample_id) per sample
    temperatures: list
    recompute_every: int = 0
    description: str = ""
    delta: list = field(default_factory=list)
    ensemble: str = "fixed"   # "fixed": every site Z links; "bonds": 2N bonds in all (Sec. II)
    boundary: str = "pbc"     # "bonds" ensemble: "pbc" or "fbc"
    couplings: str = "ferro"  # "ferro": J = 1; "pm": random signs, J = -1 with probability 1/2 (spin glass)
    field: float = 0.0        # magnitude of a random field on every site (uniform random direction), 0 = none
    spin_dim: int = 2         # 2: XY spins; 3: O(3) spins (plain engines)

    @property
    def n_samples(self):
        return len(self.graphs)

    @property
    def n_temps(self):
        return len(self.temperatures)

    @property
    def sites(self):
        return sum(L * L for L, _, _ in self.graphs)

    def spins_per_sweep(self):
        return self.sites * self.n_temps

    def betas(self):
        return [1.0 / t for t in self.temperatures]

    def deltas(self):
        """Metropolis half-width per slot: a fixed starting value, grown with T
        (near 50% acceptance is tuned on the host before measuring)."""
        if self.delta:
            return list(self.delta)
        return [min(math.pi, 1.2 * math.sqrt(t)) for t in self.temperatures]


def config(name: str) -> Config:
    if name == "C1":
        return Config("C1", [(16, 3.5, 0)], [1.0], description="L=16 z=6 rho=3.5, T=1.0, one replica")
    if name == "C2":
        return Config("C2", [(128, 3.5, 0)], geometric_temperatures(0.8, 1.6, 16),
                      description="L=128 z=6 rho=3.5, 16 T geometric in [0.8,1.6], PT every sweep")
    if name == "C3":
        g = [(64, rho, s) for rho in (2.5, 3.5, 4.5) for s in range(256)]
        return Config("C3", g, geometric_temperatures(1.5, 3.5, 24),
                      description="256 graphs x rho in {2.5,3.5,4.5}, L=64, 24 T")
    if name == "C4":
        g = [(L, 3.0, s) for L in (32, 48, 64, 96, 128, 192) for s in range(8)]
        return Config("C4", g, geometric_temperatures(1.5, 3.5, 20), recompute_every=100,
                      description="8 graphs x L in {32,48,64,96,128,192}, rho=3.0, 20 T, FP64 recompute every 100")
    if name == "E1":
        return Config("E1", [(16, 0.0, 0)], geometric_temperatures(1.6, 2.4, 4), ensemble="bonds",
                      description="L=16 2N bonds rho=0 periodic, 4 T geometric in [1.6,2.4]")
    if name == "E2":
        return Config("E2", [(16, 7.0 / 3.0, 0)], geometric_temperatures(1.6, 2.4, 4), ensemble="bonds",
                      boundary="fbc", description="L=16 2N bonds rho=7/3 free boundaries, 4 T geometric in [1.6,2.4]")
    if name == "G2":
        return Config("G2", [(128, 3.5, 0)], geometric_temperatures(0.3, 1.2, 16), couplings="pm",
                      description="C2's graph with random +-1 couplings (XY spin glass), 16 T geometric in [0.3,1.2]")
    if name == "G1":
        return Config("G1", [(16, 3.5, 0)], geometric_temperatures(0.4, 1.0, 4), couplings="pm",
                      description="C1's graph with random +-1 couplings, 4 T geometric in [0.4,1.0]")
    if name == "H1":
        return Config("H1", [(16, 3.5, 0)], geometric_temperatures(0.4, 1.0, 4), couplings="pm", field=0.5,
                      description="C1's graph, random +-1 couplings and random fields of magnitude 0.5, 4 T")
    if name == "H2":
        return Config("H2", [(128, 3.5, 0)], geometric_temperatures(0.3, 1.2, 16), couplings="pm", field=0.5,
                      description="C2's graph, random +-1 couplings and random fields of magnitude 0.5, 16 T")
    if name == "O1":
        return Config("O1", [(16, 3.5, 0)], geometric_temperatures(0.9, 1.8, 4), spin_dim=3,
                      description="C1's graph with O(3) spins, 4 T geometric in [0.9,1.8]")
    if name == "O2":
        return Config("O2", [(128, 3.5, 0)], geometric_temperatures(0.9, 1.8, 16), spin_dim=3,
                      description="C2's graph with O(3) spins, 16 T geometric in [0.9,1.8]")
    if name == "O3":
        return Config("O3", [(64, 3.5, s) for s in range(256)], geometric_temperatures(0.9, 1.8, 24), spin_dim=3,
                      description="256 graphs L=64 z=6 rho=3.5 with O(3) spins, 24 T geometric in [0.9,1.8]")
    if name == "O2G":
        return Config("O2G", [(128, 3.5, 0)], geometric_temperatures(0.4, 1.2, 16), spin_dim=3, couplings="pm",
                      description="C2's graph with O(3) spins and random +-1 couplings, 16 T geometric in [0.4,1.2]")
    if name == "OH1":
        return Config("OH1", [(16, 3.5, 0)], geometric_temperatures(0.4, 1.2, 4), spin_dim=3, couplings="pm",
                      field=0.5, description="O1's graph with random +-1 couplings and random 3-vector fields of "
                      "magnitude 0.5, 4 T geometric in [0.4,1.2]")
    if name == "OH2":
        return Config("OH2", [(128, 3.5, 0)], geometric_temperatures(0.4, 1.2, 16), spin_dim=3, couplings="pm",
                      field=0.5, description="O2G with random 3-vector fields of magnitude 0.5, 16 T")
    if name == "B64":
        return Config("B64", [(64, 10.0 / 3.0, s) for s in range(64)], geometric_temperatures(1.4, 2.0, 12),
                      ensemble="bonds", description="64 graphs L=64 2N bonds rho=10/3 periodic, 12 T geometric in [1.4,2.0]")
    if name == "C5":
        g = [(512, rho, s) for rho in (2.5, 4.5) for s in range(64)]
        return Config("C5", g, geometric_temperatures(1.5, 3.5, 32),
                      description="64 graphs x rho in {2.5,4.5}, L=512, 32 T")
    raise KeyError(name)


def first_samples(cfg: Config, n: int) -> Config:
    """The first n samples of a configuration (same stream ids), e.g. a subset
    small enough for a profiler capture."""
    import copy
    out = copy.copy(cfg)
    n = max(1, min(n, cfg.n_samples))
    out.stream_ids = [graph_stream_id(cfg, k) for k in range(n)]
    out.graphs = cfg.graphs[:n]
    out.description = f"{cfg.description}; first {n} of its {cfg.n_samples} samples"
    return out


def shard(cfg: Config, rank: int, world: int) -> Config:
    """Rank `rank` of `world`: its own disorder realisations.

    Samples are independent (parallel tempering couples only the replicas of
    one sample), so ranks share no data: with one sample or fewer samples than
    ranks every rank takes the whole batch under fresh stream ids (weak
    scaling); otherwise the samples are dealt out round-robin."""
    import copy
    out = copy.copy(cfg)
    if world <= 1:
        return out
    if cfg.n_samples < world or cfg.n_samples == 1:
        out.graphs = [(L, rho, s + rank * cfg.n_samples) for (L, rho, s) in cfg.graphs]
        out.stream_offset = rank * cfg.n_samples
    else:
        out.graphs = cfg.graphs[rank::world]
        out.stream_ids = list(range(rank, cfg.n_samples, world))
    return out


def build_graphs(cfg: Config, threads: int = 0):
    """Build every graph of a configuration with the library (parallel host threads)."""
    from . import xyl
    threads = threads or min(32, os.cpu_count() or 1)

    def one(k):
        L, rho, s = cfg.graphs[k]
        if cfg.ensemble == "bonds":
            return xyl.build_levy_bonds(L, rho, GRAPH_SEED, graph_stream_id(cfg, k), fbc=cfg.boundary == "fbc")
        return xyl.build_graph_csr(L, Z, rho, GRAPH_SEED, graph_stream_id(cfg, k))

    with cf.ThreadPoolExecutor(max_workers=threads) as ex:
        graphs = list(ex.map(one, range(cfg.n_samples)))
    for k, g in enumerate(graphs):
        j = couplings_for(cfg, k, g.n_edges)
        if j is not None:
            g.set_couplings(j)
        h = fields_for(cfg, k, g.n)
        if h is not None:
            g.set_fields(h)
    return graphs


COUPLING_SEED = 3


def couplings_for(cfg: Config, k: int, n_edges: int):
    """Random +-1 couplings of sample k (one per link, creation order), or None
    for the ferromagnet.  Seeded by the sample's stream id."""
    if cfg.couplings == "ferro":
        return None
    import numpy as np
    rng = np.random.default_rng([COUPLING_SEED, graph_stream_id(cfg, k)])
    return np.where(rng.random(n_edges) < 0.5, -1, 1).astype(np.int8)


def fields_for(cfg: Config, k: int, n: int):
    """Random fields of sample k, or None: (n, 2) vectors of magnitude
    cfg.field in uniformly random directions for XY spins, (n, 3) vectors
    uniform on the sphere of that radius for O(3) spins.  Seeded by the
    sample's stream id."""
    if cfg.field == 0.0:
        return None
    import numpy as np
    rng = np.random.default_rng([COUPLING_SEED + 1, graph_stream_id(cfg, k)])
    if cfg.spin_dim == 3:
        v = rng.normal(size=(n, 3))
        return cfg.field * v / np.linalg.norm(v, axis=1, keepdims=True)
    phi = rng.random(n) * 2.0 * np.pi
    return cfg.field * np.stack([np.cos(phi), np.sin(phi)], 1)


def graph_stream_id(cfg: Config, k: int) -> int:
    """Random-stream id of sample k of a (possibly sharded) configuration."""
    ids = getattr(cfg, "stream_ids", None)
    if ids is not None:
        return ids[k]
    return k + getattr(cfg, "stream_offset", 0)


def make_plan(cfg: Config, engine, graphs=None, seed=SPIN_SEED, **tuning):
    from . import xyl
    graphs = graphs if graphs is not None else build_graphs(cfg)
    samples = [(g, graph_stream_id(cfg, k), cfg.betas(), cfg.deltas()) for k, g in enumerate(graphs)]
    if "recompute_every" not in tuning:
        tuning["recompute_every"] = cfg.recompute_every
    tuning.setdefault("spin_dim", cfg.spin_dim)
    return xyl.Plan(samples, engine=engine, seed=seed, **tuning), graphs
