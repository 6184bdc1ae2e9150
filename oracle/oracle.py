"""ctypes front end of the C oracle in ``xyl_oracle.c`` (test infrastructure only).

Every routine here only marshals numpy arrays into the C functions; the
arithmetic lives in the C file, which cites the passages it follows.  Parity
status of each function is recorded in its docstring; all of them are pinned by
``tests/test_oracle_*.py`` against closed forms, exact special cases, brute force
or an independent implementation (cuRAND's Philox4x32-10).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# XYL_ORACLE_SRC / XYL_ORACLE_LIB point the pins at another copy of the oracle
# (the mutation tests build copies with planted mistakes)
_SRC = os.environ.get("XYL_ORACLE_SRC") or os.path.join(_HERE, "xyl_oracle.c")
_LIB_PATH = os.environ.get("XYL_ORACLE_LIB") or os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

OP_MET, OP_OR, OP_PT, OP_MEASURE = 1, 2, 4, 8
ACC_FIELDS = ("n", "e", "e2", "absm", "mx", "my", "m2", "m4", "chik", "mz")


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no fast-math, no FMA contraction)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
               "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        build()
        lib = C.CDLL(_LIB_PATH)
        P = C.c_void_p
        i32p, u32p, u64p, f64p, i64p = (C.POINTER(C.c_int32), C.POINTER(C.c_uint32), C.POINTER(C.c_uint64),
                                        C.POINTER(C.c_double), C.POINTER(C.c_int64))
        lib.orc_philox.argtypes = [u32p, u32p, u32p]
        lib.orc_philox.restype = None
        lib.orc_disp_table.argtypes = [C.c_int, C.c_double, i32p, i32p, u64p, i32p]
        lib.orc_disp_sample.argtypes = [C.c_int, C.c_double, C.c_uint64, C.c_uint32, C.c_int64, i32p]
        lib.orc_levy_graph.argtypes = [C.c_int, C.c_int, C.c_double, C.c_uint64, C.c_uint32, C.c_int,
                                       i32p, i32p, i32p, u64p]
        lib.orc_fbc_table.argtypes = [C.c_int, C.c_double, i32p, i32p, u64p]
        lib.orc_levy_bonds.argtypes = [C.c_int, C.c_double, C.c_int64, C.c_int, C.c_uint64, C.c_uint32, i32p, i32p,
                                       u64p]
        lib.orc_sim_set_couplings.argtypes = [P, f64p]
        lib.orc_sim_set_fields.argtypes = [P, f64p]
        lib.orc_sim_set_fields3.argtypes = [P, f64p]
        lib.orc_sim_set_dim.argtypes = [P, C.c_int]
        lib.orc_reflect.argtypes = [C.c_int, f64p, f64p, f64p]
        lib.orc_reflect.restype = None
        lib.orc_o3_propose.argtypes = [C.c_double] * 6 + [f64p, f64p, f64p]
        lib.orc_o3_propose.restype = None
        lib.orc_walk_returns.argtypes = [C.c_int, i32p, i32p, C.c_int64, i32p, C.c_int32, C.c_uint64, u64p]
        lib.orc_pick_partner_counts.argtypes = [C.c_int, C.c_int, C.c_double, C.c_uint64, i32p, i32p, i32p,
                                                C.c_int, C.c_int, C.c_int64, i64p]
        lib.orc_slo_color.argtypes = [C.c_int, C.c_int64, i32p, i32p, i32p]
        lib.orc_csr.argtypes = [C.c_int, C.c_int64, i32p, i32p, i32p, C.c_int, i32p, i32p, i32p, i32p]
        lib.orc_sim_new.argtypes = [C.c_int, C.c_int64, i32p, i32p, i32p, i32p, C.c_int, C.c_int, f64p, f64p,
                                    C.c_uint64, C.c_uint32, C.c_int]
        lib.orc_sim_new.restype = P
        lib.orc_sim_free.argtypes = [P]
        lib.orc_sim_init.argtypes = [P, C.c_int]
        lib.orc_sim_sweeps.argtypes = [P, C.c_int, C.c_uint, C.c_int]
        lib.orc_sim_get_angles.argtypes = [P, f64p]
        lib.orc_sim_set_angles.argtypes = [P, f64p]
        lib.orc_sim_get_energies.argtypes = [P, f64p]
        lib.orc_sim_get_labels.argtypes = [P, i32p]
        lib.orc_sim_get_acc.argtypes = [P, f64p, u64p, u64p, u64p, u64p]
        lib.orc_sim_reset_acc.argtypes = [P]
        lib.orc_sim_set_delta.argtypes = [P, f64p]
        lib.orc_sim_set_tie_eps.argtypes = [P, C.c_double]
        lib.orc_sim_get_ties.argtypes = [P, i64p, i64p, f64p]
        lib.orc_sim_get_vectors.argtypes = [P, f64p]
        lib.orc_sim_set_vectors.argtypes = [P, f64p]
        lib.orc_sim_set_labels.argtypes = [P, i32p, C.c_uint64]
        lib.orc_sim_get_tie_counts.argtypes = [P, i64p]
        lib.orc_sim_clear_ties.argtypes = [P]
        lib.orc_sim_get_tie_log.argtypes = [P, C.c_int, C.c_int64, i32p, i32p, i64p, i32p]
        lib.orc_sim_get_tie_log.restype = C.c_int64
        lib.orc_sim_force.argtypes = [P, C.c_int64, i32p, i32p, i32p]
        lib.orc_sim_force_pt.argtypes = [P, C.c_int64, i32p, i32p]
        lib.orc_sim_set_active.argtypes = [P, C.POINTER(C.c_uint8)]
        lib.orc_sincos_series.argtypes = [C.c_double, f64p, f64p]
        lib.orc_sincos_series.restype = None
        lib.orc_sim_sweep_index.argtypes = [P]
        lib.orc_sim_sweep_index.restype = C.c_uint64
        _lib = lib
        return lib


def _ptr(a, ctype):
    return a.ctypes.data_as(C.POINTER(ctype))


def philox(ctr, key) -> np.ndarray:
    """Philox4x32-10 block for counter ``ctr`` (4 words) and key (2 words).

    Pinned against cuRAND's host Philox4x32-10 generator (tests/test_oracle_philox.py)."""
    lib = _load()
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib.orc_philox(_ptr(c, C.c_uint32), _ptr(k, C.c_uint32), _ptr(out, C.c_uint32))
    return out


def sincos_series(x: float):
    """sin, cos by the Maclaurin series used for the Metropolis step.

    Pinned against libm (tests/test_oracle_philox.py)."""
    lib = _load()
    sn = np.zeros(1); cs = np.zeros(1)
    lib.orc_sincos_series(float(x), _ptr(sn, C.c_double), _ptr(cs, C.c_double))
    return float(sn[0]), float(cs[0])


def disp_table(L: int, rho: float):
    """Displacement table of the link law (Eq. Levyi): (dx, dy, B, n_near).

    Pinned by the proposal-law chi^2 test against an independent count of
    minimum-image distances, and by exact integer-weight invariants."""
    lib = _load()
    n = L * L - 1
    dx = np.zeros(n, np.int32); dy = np.zeros(n, np.int32); B = np.zeros(n, np.uint64)
    nn = np.zeros(1, np.int32)
    rc = lib.orc_disp_table(L, rho, _ptr(dx, C.c_int32), _ptr(dy, C.c_int32), _ptr(B, C.c_uint64),
                            _ptr(nn, C.c_int32))
    if rc:
        raise ValueError("bad lattice size")
    return dx, dy, B, int(nn[0])


def disp_sample(L: int, rho: float, seed: int, sample: int, n_draws: int) -> np.ndarray:
    """Table entries proposed by ``n_draws`` consecutive graph-stream draws."""
    lib = _load()
    out = np.zeros(n_draws, np.int32)
    rc = lib.orc_disp_sample(L, rho, seed, sample, n_draws, _ptr(out, C.c_int32))
    if rc:
        raise ValueError("bad lattice size")
    return out


def levy_graph(L: int, z: int, rho: float, seed: int, sample: int = 0, max_restarts: int = 100):
    """Fixed-degree Levy graph: (ei, ej, restarts, draws), links in creation order.

    Pinned by exact degree / symmetry / no-self-loop / no-multi-edge checks, the
    first-link law (brute force over many seeds) and the accepted-link law."""
    lib = _load()
    n = L * L
    ne = n * z // 2
    ei = np.zeros(ne, np.int32); ej = np.zeros(ne, np.int32)
    rs = np.zeros(1, np.int32); dr = np.zeros(1, np.uint64)
    rc = lib.orc_levy_graph(L, z, rho, seed, sample, max_restarts, _ptr(ei, C.c_int32), _ptr(ej, C.c_int32),
                            _ptr(rs, C.c_int32), _ptr(dr, C.c_uint64))
    if rc == -1:
        raise ValueError("bad graph arguments")
    if rc == -3:
        raise RuntimeError("graph construction hit a dead end on every restart")
    return ei, ej, int(rs[0]), int(dr[0])


def levy_bonds(L: int, rho: float, seed: int, sample: int = 0, n_bonds=None, fbc: bool = False):
    """The paper's ensemble (Sec. II): exactly ``n_bonds`` bonds (default 2N,
    mean degree 4), each pair drawn with probability proportional to r^-rho,
    periodic (minimum image) or free boundaries.  Returns (ei, ej, attempts),
    bonds in the order they were accepted.

    Pinned by exact bond count / no self-loop / no repeated pair checks, the
    law of the first bond over many streams (PBC and FBC, brute-force pair
    counts), the exact hypergeometric degree law and pair-distance law of the
    uniform graph at rho = 0, and the brute-force FBC displacement table."""
    lib = _load()
    n = L * L
    m = 2 * n if n_bonds is None else int(n_bonds)
    ei = np.zeros(max(m, 1), np.int32); ej = np.zeros(max(m, 1), np.int32)
    at = np.zeros(1, np.uint64)
    rc = lib.orc_levy_bonds(L, rho, m, 1 if fbc else 0, seed, sample, _ptr(ei, C.c_int32), _ptr(ej, C.c_int32),
                            _ptr(at, C.c_uint64))
    if rc == -1:
        raise ValueError("bad graph arguments")
    if rc == -3:
        raise RuntimeError("too many rejected bond draws")
    return ei[:m], ej[:m], int(at[0])


def walk_returns(row_ptr, col, start, n_steps: int, seed: int):
    """Self-return counts of simple random walks on a CSR graph (App. A):
    returns[tau] = walkers on their starting node after tau steps.

    Pinned by exact return probabilities (powers of the transition matrix) on
    small graphs, the closed form [C(2n, n) / 4^n]^2 and the absence of odd
    returns on the square lattice, and the isolated-node rule."""
    lib = _load()
    row_ptr = np.ascontiguousarray(row_ptr, np.int32); col = np.ascontiguousarray(col, np.int32)
    start = np.ascontiguousarray(start, np.int32)
    out = np.zeros(n_steps + 1, np.uint64)
    if lib.orc_walk_returns(len(row_ptr) - 1, _ptr(row_ptr, C.c_int32), _ptr(col, C.c_int32), len(start),
                            _ptr(start, C.c_int32), n_steps, seed, _ptr(out, C.c_uint64)):
        raise ValueError("bad walk arguments")
    return out


def fbc_table(L: int, rho: float):
    """Free-boundary link-law table: (dx, dy, B) in table order."""
    lib = _load()
    n = (2 * L - 1) ** 2 - 1
    dx = np.zeros(n, np.int32); dy = np.zeros(n, np.int32); B = np.zeros(n, np.uint64)
    if lib.orc_fbc_table(L, rho, _ptr(dx, C.c_int32), _ptr(dy, C.c_int32), _ptr(B, C.c_uint64)):
        raise ValueError("bad lattice size")
    return dx, dy, B


def pick_partner_counts(L, z, rho, seed, deg, adj, unsat, i, n_trials):
    """Outcome counts of the partner draw of site ``i`` from a given pairing
    state (index n = dead end).  Pinned against the exact conditional law."""
    lib = _load()
    n = L * L
    deg = np.ascontiguousarray(deg, np.int32); adj = np.ascontiguousarray(adj, np.int32).reshape(-1)
    unsat = np.ascontiguousarray(unsat, np.int32)
    counts = np.zeros(n + 1, np.int64)
    rc = lib.orc_pick_partner_counts(L, z, rho, seed, _ptr(deg, C.c_int32), _ptr(adj, C.c_int32),
                                     _ptr(unsat, C.c_int32), len(unsat), i, n_trials, _ptr(counts, C.c_int64))
    if rc:
        raise ValueError("bad lattice size")
    return counts


def slo_color(n: int, ei, ej):
    """Smallest-last colouring: (colour per site, number of colours).

    Pinned by properness, the degeneracy bound and hand-checked small graphs."""
    lib = _load()
    ei = np.ascontiguousarray(ei, np.int32); ej = np.ascontiguousarray(ej, np.int32)
    col = np.zeros(n, np.int32)
    q = lib.orc_slo_color(n, len(ei), _ptr(ei, C.c_int32), _ptr(ej, C.c_int32), _ptr(col, C.c_int32))
    return col, int(q)


def csr(n: int, ei, ej, color, n_colors: int):
    """Colour-sorted CSR: (perm, row_ptr, col, color_ptr)."""
    lib = _load()
    ei = np.ascontiguousarray(ei, np.int32); ej = np.ascontiguousarray(ej, np.int32)
    color = np.ascontiguousarray(color, np.int32)
    perm = np.zeros(n, np.int32); row_ptr = np.zeros(n + 1, np.int32)
    col = np.zeros(2 * len(ei), np.int32); cptr = np.zeros(n_colors + 1, np.int32)
    lib.orc_csr(n, len(ei), _ptr(ei, C.c_int32), _ptr(ej, C.c_int32), _ptr(color, C.c_int32), n_colors,
                _ptr(perm, C.c_int32), _ptr(row_ptr, C.c_int32), _ptr(col, C.c_int32), _ptr(cptr, C.c_int32))
    return perm, row_ptr, col, cptr


def lattice_xy(L: int) -> np.ndarray:
    """(x, y) of site id = x + L*y."""
    ids = np.arange(L * L, dtype=np.int32)
    return np.stack([ids % L, ids // L], axis=1).astype(np.int32).reshape(-1)


class Sim:
    """Sequential sampler (Metropolis + overrelaxation + PT + measurement).

    ``beta``/``delta`` are per temperature slot; replica r starts at slot r.
    ``u24=True`` selects the 24-bit uniforms used by the single-precision kernel.
    Pinned by the chain, ring and small-graph exact results, beta = 0 exact
    moments, the low-temperature limit, the high-temperature series and exact
    energy conservation of overrelaxation."""

    def __init__(self, n, ei, ej, color, beta, delta, seed, sample=0, xy=None, L=None, u24=False, dim=2):
        self._lib = _load()
        self.n = int(n)
        self.dim = int(dim)
        self.R = len(beta)
        self._keep = [np.ascontiguousarray(ei, np.int32), np.ascontiguousarray(ej, np.int32),
                      np.ascontiguousarray(color, np.int32)]
        xy_arr = None if xy is None else np.ascontiguousarray(xy, np.int32)
        b = np.ascontiguousarray(beta, np.float64); d = np.ascontiguousarray(delta, np.float64)
        self._h = self._lib.orc_sim_new(
            self.n, len(self._keep[0]), _ptr(self._keep[0], C.c_int32), _ptr(self._keep[1], C.c_int32),
            _ptr(self._keep[2], C.c_int32), None if xy_arr is None else _ptr(xy_arr, C.c_int32),
            int(L or 0), self.R, _ptr(b, C.c_double), _ptr(d, C.c_double), seed, sample, 1 if u24 else 0)
        if not self._h:
            raise MemoryError("oracle allocation failed")
        if self.dim != 2 and self._lib.orc_sim_set_dim(self._h, self.dim):
            raise ValueError("spin dimension must be 2 (XY) or 3 (O(3))")

    def close(self):
        if self._h:
            self._lib.orc_sim_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def init(self, aligned=False):
        self._lib.orc_sim_init(self._h, 1 if aligned else 0)

    def set_couplings(self, j_per_bond=None):
        """Random bonds: one coupling per bond (edge order given to the
        constructor); None restores J = 1.  Pinned by exact gauge invariance
        and quadrature on frustrated small graphs."""
        if j_per_bond is None:
            self._jkeep = None
            self._lib.orc_sim_set_couplings(self._h, None)
            return
        self._jkeep = np.ascontiguousarray(j_per_bond, np.float64)
        if self._lib.orc_sim_set_couplings(self._h, _ptr(self._jkeep, C.c_double)):
            raise MemoryError("oracle allocation failed")

    def set_fields(self, hxy=None):
        """Random fields: (n, 2) field vectors per site for XY spins, (n, 3)
        for O(3) spins (original ids); None removes them.  Pinned by the exact
        single-spin laws (XY: I1(b|h|)/I0(b|h|); O(3): the Langevin function
        coth(b|h|) - 1/(b|h|)) and by quadrature on 2-3-spin graphs."""
        if hxy is None:
            self._hkeep = None
            self._lib.orc_sim_set_fields(self._h, None)
            return
        h = np.ascontiguousarray(hxy, np.float64)
        comps = h.shape[-1] if h.ndim == 2 else 2
        self._hkeep = h.reshape(-1)
        setter = self._lib.orc_sim_set_fields3 if comps == 3 else self._lib.orc_sim_set_fields
        rc = setter(self._h, _ptr(self._hkeep, C.c_double))
        if rc == -2:
            raise ValueError("field vectors need as many components as the spins (2: XY, 3: O(3))")
        if rc:
            raise MemoryError("oracle allocation failed")

    def sweeps(self, n, ops=OP_MET | OP_OR | OP_PT | OP_MEASURE, measure_every=1):
        self._lib.orc_sim_sweeps(self._h, int(n), int(ops), int(measure_every))

    def angles(self) -> np.ndarray:
        out = np.zeros((self.R, self.n), np.float64)
        self._lib.orc_sim_get_angles(self._h, _ptr(out, C.c_double))
        return out

    def set_angles(self, a):
        a = np.ascontiguousarray(a, np.float64).reshape(self.R, self.n)
        self._lib.orc_sim_set_angles(self._h, _ptr(a, C.c_double))

    def vectors(self) -> np.ndarray:
        out = np.zeros((self.R, self.n, self.dim), np.float64)
        self._lib.orc_sim_get_vectors(self._h, _ptr(out, C.c_double))
        return out

    def set_vectors(self, v):
        v = np.ascontiguousarray(v, np.float64).reshape(self.R, self.n, self.dim)
        self._lib.orc_sim_set_vectors(self._h, _ptr(v, C.c_double))

    def set_labels(self, rep_at, sweep_index):
        a = np.ascontiguousarray(rep_at, np.int32)
        self._lib.orc_sim_set_labels(self._h, _ptr(a, C.c_int32), int(sweep_index))

    def tie_counts(self) -> np.ndarray:
        out = np.zeros(self.R, np.int64)
        self._lib.orc_sim_get_tie_counts(self._h, _ptr(out, C.c_int64))
        return out

    def clear_ties(self):
        self._lib.orc_sim_clear_ties(self._h)

    def tie_log(self, pt=False):
        """Near-tie tests since the last clear: (replica, original site id,
        sweep, outcome) rows for Metropolis; for PT the site column is the
        pair k and the replica column is -1."""
        n = self._lib.orc_sim_get_tie_log(self._h, 1 if pt else 0, 0, None, None, None, None)
        rep = np.zeros(n, np.int32); site = np.zeros(n, np.int32)
        sweep = np.zeros(n, np.int64); acc = np.zeros(n, np.int32)
        if n:
            self._lib.orc_sim_get_tie_log(self._h, 1 if pt else 0, n, _ptr(rep, C.c_int32), _ptr(site, C.c_int32),
                                          _ptr(sweep, C.c_int64), _ptr(acc, C.c_int32))
        return [(int(a), int(b), int(c), int(d)) for a, b, c, d in zip(rep, site, sweep, acc)]

    def force(self, decisions=()):
        """Metropolis outcomes to take instead of the test's: an iterable of
        (replica, original site id, accept); empty removes them."""
        d = list(decisions)
        rep = np.array([x[0] for x in d], np.int32); site = np.array([x[1] for x in d], np.int32)
        acc = np.array([1 if x[2] else 0 for x in d], np.int32)
        if self._lib.orc_sim_force(self._h, len(d), _ptr(rep, C.c_int32), _ptr(site, C.c_int32),
                                   _ptr(acc, C.c_int32)):
            raise ValueError("bad forced decision")

    def force_pt(self, decisions=()):
        """PT outcomes to take instead of the test's: (pair k, accept) pairs; empty removes them."""
        d = list(decisions)
        pair = np.array([x[0] for x in d], np.int32); acc = np.array([1 if x[1] else 0 for x in d], np.int32)
        if self._lib.orc_sim_force_pt(self._h, len(d), _ptr(pair, C.c_int32), _ptr(acc, C.c_int32)):
            raise ValueError("bad forced PT decision")

    def set_active(self, replicas=None):
        """Sweeps update only these replicas (None: all).  For spins and
        energies only: PT then compares stale energies of the others."""
        if replicas is None:
            self._lib.orc_sim_set_active(self._h, None)
            return
        mask = np.zeros(self.R, np.uint8)
        mask[list(replicas)] = 1
        if self._lib.orc_sim_set_active(self._h, _ptr(mask, C.c_uint8)):
            raise MemoryError("oracle allocation failed")

    def energies(self) -> np.ndarray:
        out = np.zeros(self.R, np.float64)
        self._lib.orc_sim_get_energies(self._h, _ptr(out, C.c_double))
        return out

    def labels(self) -> np.ndarray:
        out = np.zeros(self.R, np.int32)
        self._lib.orc_sim_get_labels(self._h, _ptr(out, C.c_int32))
        return out

    def set_delta(self, delta):
        d = np.ascontiguousarray(delta, np.float64)
        self._lib.orc_sim_set_delta(self._h, _ptr(d, C.c_double))

    def set_tie_eps(self, eps):
        self._lib.orc_sim_set_tie_eps(self._h, float(eps))

    def ties(self):
        ft = np.zeros(self.R, np.int64); fp = np.zeros(1, np.int64); mm = np.zeros(1, np.float64)
        self._lib.orc_sim_get_ties(self._h, _ptr(ft, C.c_int64), _ptr(fp, C.c_int64), _ptr(mm, C.c_double))
        return ft, int(fp[0]), float(mm[0])

    def accumulators(self):
        acc = np.zeros((self.R, len(ACC_FIELDS)), np.float64)
        ma = np.zeros(self.R, np.uint64); mt = np.zeros(self.R, np.uint64)
        pa = np.zeros(self.R, np.uint64); pt = np.zeros(self.R, np.uint64)
        self._lib.orc_sim_get_acc(self._h, _ptr(acc, C.c_double), _ptr(ma, C.c_uint64), _ptr(mt, C.c_uint64),
                                  _ptr(pa, C.c_uint64), _ptr(pt, C.c_uint64))
        return {"acc": acc, "met_acc": ma, "met_try": mt, "pt_acc": pa, "pt_try": pt}

    def reset_acc(self):
        self._lib.orc_sim_reset_acc(self._h)

    @property
    def sweep_index(self) -> int:
        return int(self._lib.orc_sim_sweep_index(self._h))


def graph_sim(ei, ej, n, beta, delta, seed, sample=0, xy=None, L=None, u24=False, dim=2):
    """Sampler on an explicit edge list, coloured by ``slo_color``."""
    color, _ = slo_color(n, ei, ej)
    return Sim(n, ei, ej, color, beta, delta, seed, sample=sample, xy=xy, L=L, u24=u24, dim=dim)


def reflect(s, h) -> np.ndarray:
    """The overrelaxation map: the reflection of spin ``s`` (2 or 3
    components) about the local field ``h``."""
    lib = _load()
    sv = np.ascontiguousarray(s, np.float64)
    hv = np.ascontiguousarray(h, np.float64)
    out = np.zeros_like(sv)
    lib.orc_reflect(len(sv), _ptr(sv, C.c_double), _ptr(hv, C.c_double), _ptr(out, C.c_double))
    return out


def o3_propose(s, half_width: float, u: float, uphi: float) -> np.ndarray:
    """The O(3) Metropolis proposal: a point of the spherical cap of angular
    radius ``half_width`` around the unit vector ``s``, from the cap uniform
    ``u`` and the azimuth uniform ``uphi``."""
    lib = _load()
    out = [C.c_double(), C.c_double(), C.c_double()]
    lib.orc_o3_propose(float(s[0]), float(s[1]), float(s[2]), float(half_width), float(u), float(uphi),
                       *[C.byref(o) for o in out])
    return np.array([o.value for o in out])
