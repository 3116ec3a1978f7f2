"""The pins catch plausible mistakes: each case compiles a copy of the oracle
with one planted error (on the CPU) and runs the pin suites against it in a
child process; at least one pin must fail for every mutant."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "mhs_oracle.c")

MUTANTS = {
    "alpha2_sign": ("- 2.0 * L->cz + p->alpha * p->alpha;", "- 2.0 * L->cz - p->alpha * p->alpha;"),
    "xi_dropped_in_y": ("L->cy[k] = one_m_xi / (L->hy * L->hy);", "L->cy[k] = 1.0 / (L->hy * L->hy);"),
    "xi_wrong_plane": ("orc_xi(p, k * L->hz)", "orc_xi(p, (k + 1) * L->hz)"),
    "x_y_coeff_swap": ("const double Au = L->cx[k] * (u[c + 1] + u[c - 1]) +\n                                  L->cy[k] * (u[c + nx] + u[c - nx]) +",
                       "const double Au = L->cy[k] * (u[c + 1] + u[c - 1]) +\n                                  L->cx[k] * (u[c + nx] + u[c - nx]) +"),
    "lower_boundary_sign": ("f[IDX(i, j, 0, nx, ny)] = -bz[IDX(i, j, 0, nx, ny)];", "f[IDX(i, j, 0, nx, ny)] = bz[IDX(i, j, 0, nx, ny)];"),
    "restriction_weights": ("static const double w[3] = {0.25, 0.5, 0.25};\n    const int nxc = C->nx, nyc = C->ny, nzc",
                            "static const double w[3] = {0.3, 0.4, 0.3};\n    const int nxc = C->nx, nyc = C->ny, nzc"),
    "prolongation_weight": ("? 0.5 : 0.0", "? 0.45 : 0.0"),
    "one_sided_d1_end": ("(3.0 * f[c] - 4.0 * f[c - s] + f[c - 2 * s])", "(3.0 * f[c] - 4.0 * f[c - s] - f[c - 2 * s])"),
    "one_sided_d2_start": ("(2.0 * f[c] - 5.0 * f[c + s] + 4.0 * f[c + 2 * s] - f[c + 3 * s])",
                           "(2.0 * f[c] - 5.0 * f[c + s] + 3.0 * f[c + 2 * s] - f[c + 3 * s])"),
    "By_alpha_sign": ("by[c] = -p->alpha * Px[c]", "by[c] = p->alpha * Px[c]"),
    "Bx_mixed_axis": ("bx[c] = p->alpha * Py[c] + d1(Pz, nx, ny, nz, i, j, k, 0, hx);",
                      "bx[c] = p->alpha * Py[c] + d1(Pz, nx, ny, nz, i, j, k, 1, hy);"),
    "rho_tension_mu0": ("xi * BgradBz / p->mu0", "xi * BgradBz * p->mu0"),
    "rho_pressure_term_sign": ("rb + (dxi * B2 +", "rb + (-dxi * B2 +"),
    "pressure_xi_dropped": ("pr[c] = pb - xi * B2;", "pr[c] = pb - B2;"),
    "pb_transition_exponent": ("(1.0 - pow(p->T_cor, -(z - p->z1) / d))", "(1.0 - pow(p->T_cor, (z - p->z1) / d))"),
    "dxi_sign": ("case 1: return -p->xi_kappa * p->xi_a", "case 1: return p->xi_kappa * p->xi_a"),
    "zline_top_dirichlet_dropped": ("if (k == nz - 2) b -= L->cz * u[c + plane];", "if (k == nz - 1) b -= L->cz * u[c + plane];"),
    "zline_wrong_columns": ("if (((i + j) & 1) != colour) continue;\n                for (int t = 0; t < m; ++t) {",
                            "if (((i + j + 1) & 1) != colour) continue;\n                for (int t = 0; t < m; ++t) {"),
    "zline_back_substitution": ("u[c] = rhs[t] - (t < m - 1 ? sup[t] * u[c + plane] : 0.0);",
                                "u[c] = rhs[t] + (t < m - 1 ? sup[t] * u[c + plane] : 0.0);"),
    "curl_y_sign": ("const double cy = (d1(Bx, nx, ny, nz, i, j, k, 2, hz) - d1(Bz, nx, ny, nz, i, j, k, 0, hx)) / p->mu0;",
                    "const double cy = (d1(Bx, nx, ny, nz, i, j, k, 2, hz) + d1(Bz, nx, ny, nz, i, j, k, 0, hx)) / p->mu0;"),
    "curl_mu0": ("const double cz = (d1(By, nx, ny, nz, i, j, k, 0, hx) - d1(Bx, nx, ny, nz, i, j, k, 1, hy)) / p->mu0;",
                 "const double cz = (d1(By, nx, ny, nz, i, j, k, 0, hx) - d1(Bx, nx, ny, nz, i, j, k, 1, hy));"),
    "trace_interp_weight": ("e[dz][dy] = f0 * (1.0 - f[0]) + f1 * f[0];", "e[dz][dy] = f0 * f[0] + f1 * (1.0 - f[0]);"),
    "rk4_stage_weight": ("(((k1[a] + 2.0 * k2[a]) + 2.0 * k3[a]) + k4[a])", "(((k1[a] + 2.0 * k2[a]) + k3[a]) + 2.0 * k4[a])"),
    "exact_level_one_cycle": ("if (rn <= 1e-15 * fn || rn > 0.5 * prev) break;", "if (it > 0) break;"),
    "exact_level_ignored": ("if (l == mg->exact_level) { exact_solve", "if (l == -2) { exact_solve"),
    "bnorm_scaled": ("const double bnorm = mg_norm(mg, 0, mg->r[0]);", "const double bnorm = 2.0 * mg_norm(mg, 0, mg->r[0]);"),
    "lift_bottom_face_only": ("for (int k = (mg->dim == 3 ? 1 : 0); k < (mg->dim == 3 ? L->nz - 1 : 1); ++k)\n        for (int j = 1; j < L->ny - 1; ++j)\n            for (int i = 1; i < L->nx - 1; ++i) lift[",
                              "for (int k = (mg->dim == 3 ? 1 : 0); k < (mg->dim == 3 ? L->nz : 1); ++k)\n        for (int j = 0; j < L->ny; ++j)\n            for (int i = 0; i < L->nx; ++i) lift["),
    "gs_divides_wrong_diag": ("u[c] = ((f ? f[c] : 0.0) - off) / L->diag[k];", "u[c] = ((f ? f[c] : 0.0) - off) / L->diag[0];"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_mutant(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) >= 1, f"mutation anchor for {name} not found"
    mutated = src.replace(old, new, 1)
    csrc = tmp_path / "mut.c"
    csrc.write_text(mutated)
    lib = tmp_path / "libmut.so"
    subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", "-o", str(lib), str(csrc), "-lm"])
    env = dict(os.environ, MHS_ORACLE_LIB=str(lib), OMP_NUM_THREADS="2")
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        "tests/test_oracle_pins.py", "tests/test_oracle_paper_examples.py",
                        "tests/test_oracle_postproc.py"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"mutant {name} survived every pin:\n{r.stdout[-2000:]}"
