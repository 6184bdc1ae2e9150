"""The oracle's pins catch plausible mistakes: each case plants one mistake (a
wrong constant, sign, factor, index or dropped term) in a copy of
oracle/xyl_oracle.c, and the pins of that part must then fail.  The copy is
compiled and loaded in a separate pytest process (XYL_ORACLE_SRC /
XYL_ORACLE_LIB); the committed oracle is untouched."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "xyl_oracle.c")

# (name, text in the oracle, planted replacement, pins that must then fail)
MUTATIONS = [
    ("philox multiplier", "(uint64_t)0xD2511F53u * (uint64_t)c0", "(uint64_t)0xD2511F55u * (uint64_t)c0",
     "tests/test_oracle_philox.py::test_philox_matches_curand"),
    ("link-law exponent (periodic table)",
     "    if (!S) { disp_table_free(t); return -1; }\n    S[0] = 0.0;\n    for (int m = 0; m < t->n; ++m) {\n"
     "        double r2 = (double)(t->dx[m] * t->dx[m] + t->dy[m] * t->dy[m]);\n"
     "        S[m + 1] = S[m] + pow(r2, -0.5 * rho);",
     "    if (!S) { disp_table_free(t); return -1; }\n    S[0] = 0.0;\n    for (int m = 0; m < t->n; ++m) {\n"
     "        double r2 = (double)(t->dx[m] * t->dx[m] + t->dy[m] * t->dy[m]);\n"
     "        S[m + 1] = S[m] + pow(r2, -0.25 * rho);",
     "tests/test_oracle_graph.py::test_proposal_law_chi2"),
    ("link-law exponent (free table)",
     "            t->dx[k] = dx; t->dy[k] = dy; ++k;\n        }\n    S[0] = 0.0;\n    for (int m = 0; m < t->n; ++m) {\n"
     "        double r2 = (double)(t->dx[m] * t->dx[m] + t->dy[m] * t->dy[m]);\n"
     "        S[m + 1] = S[m] + pow(r2, -0.5 * rho);",
     "            t->dx[k] = dx; t->dy[k] = dy; ++k;\n        }\n    S[0] = 0.0;\n    for (int m = 0; m < t->n; ++m) {\n"
     "        double r2 = (double)(t->dx[m] * t->dx[m] + t->dy[m] * t->dy[m]);\n"
     "        S[m + 1] = S[m] + pow(r2, -0.25 * rho);",
     "tests/test_oracle_bonds.py::test_first_bond_law"),
    ("Metropolis energy sign", "double dE = -((nx - x[v]) * hx + (ny - y[v]) * hy);",
     "double dE = ((nx - x[v]) * hx + (ny - y[v]) * hy);", "tests/test_oracle_physics.py::test_open_chain"),
    ("one-sided Metropolis step", "double d = s->delta[slot] * (2.0 * ud - 1.0);", "double d = s->delta[slot] * ud;",
     "tests/test_oracle_physics.py::test_small_graphs_against_quadrature"),
    ("PT temperature order", "double x = (s->beta[k] - s->beta[k + 1]) * (s->E[a] - s->E[b]);",
     "double x = (s->beta[k + 1] - s->beta[k]) * (s->E[a] - s->E[b]);",
     "tests/test_oracle_physics.py::test_parallel_tempering_slots_unbiased"),
    ("chi(k) normalisation", "out[ACC_CHIK] = (fa + fb) / (2.0 * N);", "out[ACC_CHIK] = (fa + fb) / N;",
     "tests/test_oracle_physics.py::test_beta_zero_exact_moments"),
    ("m^4 as m^2", "out[ACC_M4] = m2 * m2;", "out[ACC_M4] = m2;",
     "tests/test_oracle_physics.py::test_beta_zero_exact_moments"),
    ("reflection sign", "    for (int a = 0; a < dim; ++a) out[a] = k * h[a] - sv[a];",
     "    for (int a = 0; a < dim; ++a) out[a] = k * h[a] + sv[a];",
     "tests/test_oracle_physics.py::test_overrelaxation_map_is_an_energy_conserving_involution"),
    ("coupling dropped in x", "ax += s->jn[a] * x[s->nbr[a]];", "ax += x[s->nbr[a]];",
     "tests/test_oracle_couplings.py::test_frustrated_small_graphs_against_quadrature"),
    ("field counted twice", "        ax += s->hx[v];", "        ax += 2.0 * s->hx[v];",
     "tests/test_oracle_fields.py::test_free_spins_follow_the_bessel_law"),
    ("walk neighbour index", "v = col[row_ptr[v] + (int)(((uint64_t)x[t % 4] * (uint64_t)k) >> 32)];",
     "v = col[row_ptr[v] + (int)(((uint64_t)x[t % 4] * (uint64_t)(k - 1)) >> 32)];",
     "tests/test_oracle_walk.py::test_return_counts_match_transition_matrix_powers"),
    ("initial angles on half the circle", "double th = 2.0 * ORC_PI * u - ORC_PI;", "double th = ORC_PI * u - ORC_PI;",
     "tests/test_oracle_physics.py::test_initial_angles_are_uniform"),
    ("SLO tie-break", "return a.deg < b.deg || (a.deg == b.deg && a.id < b.id);",
     "return a.deg < b.deg || (a.deg == b.deg && a.id > b.id);",
     "tests/test_oracle_graph.py::test_slo_hand_derived_colourings"),
    ("bond duplicates kept", "        if (bonded) continue;\n        int ends[2] = { i, j };",
     "        (void)bonded;\n        int ends[2] = { i, j };", "tests/test_oracle_bonds.py::test_bonds_simple_counted_seeded"),
    ("CSR rows unsorted", "        qsort(col + row_ptr[a], (size_t)d, sizeof(int32_t), cmp_int);", "",
     "tests/test_oracle_graph.py::test_csr_layout"),
    ("O(3) cap factor", "const double w = u * (2.0 * (sh * sh));", "const double w = u * (sh * sh);",
     "tests/test_oracle_o3.py::test_cap_proposal_is_uniform_on_the_cap"),
    ("O(3) z dropped from the energy", "double d = x[i] * x[j] + y[i] * y[j] + z[i] * z[j];",
     "double d = x[i] * x[j] + y[i] * y[j];", "tests/test_oracle_o3.py::test_tree_moments_are_exact"),
    ("O(3) field z dropped from the local field", "        az += f[2];\n", "",
     "tests/test_oracle_o3.py::test_free_spins_in_fields_follow_the_langevin_law"),
    ("O(3) field term dropped from the energy",
     "E -= s->hx[v] * x[v] + s->hy[v] * y[v] + s->hz[v] * z[v];", "E -= 0.0;",
     "tests/test_oracle_o3.py::test_bond_with_fields_against_quadrature"),
]


@pytest.mark.parametrize("name,text,planted,pins", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_planted_mistake_fails_its_pins(tmp_path, name, text, planted, pins):
    src = open(SRC).read()
    assert src.count(text) == 1, f"{name}: the text to mutate is not unique in the oracle"
    mutated = tmp_path / "xyl_oracle.c"
    mutated.write_text(src.replace(text, planted))
    env = dict(os.environ, XYL_ORACLE_SRC=str(mutated), XYL_ORACLE_LIB=str(tmp_path / "liboracle.so"))
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider", pins],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 1, f"{name}: pins did not fail\n{r.stdout[-2000:]}{r.stderr[-1000:]}"
