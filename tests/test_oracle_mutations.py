"""Planted mistakes in the CPU oracle and in the input generator, each of which a pin must catch.

Every case copies the oracle, the input generator and the pin tests into a scratch directory,
plants one plausible mistake in the copy's source (a dropped term, a flipped sign, a wrong or
transposed index, a missing factor), rebuilds the copy and runs the pins named for it there
(`test_oracle_pins.py` for the oracle, `test_fegen.py` for the generator): at least one of them
has to fail.  The unmodified copies have to pass the same pins, so a failure is the mistake's
and not the harness's.  The sources under `oracle/` and `fegen/` are never written.

Changes that leave the result unchanged are not planted: a different order of the coarse
numbering, or the larger instead of the smaller global id between two half-way candidates of a
non-whole ratio (both relabellings, which the pins treat as the same operator), and keeping the
last instead of the first duplicate of a prolongation entry (the elements sharing a node give the
same interpolation value).
"""
import os
import re
import shutil
import subprocess
import sys
import tempfile
from concurrent.futures import ThreadPoolExecutor

import pytest

import fegen

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# name: (source file, text, replacement, occurrences, pins that must catch it: a -k expression
#        over the package's pin file, or (pin file, expression))
MUTATIONS = {
    # GLL nodes: the Legendre three-term recurrence with a flipped sign
    "gll_recurrence_sign": (
        "oracle/oracle.c", "double P2 = ((2.0 * k + 1.0) * x * P1 - k * P0) / (k + 1.0);",
        "double P2 = ((2.0 * k + 1.0) * x * P1 + k * P0) / (k + 1.0);", 1,
        "test_gll_nodes_match_fig1"),
    # P1D: the Lagrange denominator taken at a fine node instead of a coarse one
    "p1d_denominator_index": (
        "oracle/oracle.c", "(xq[b] - xq[m])", "(xp[b] - xq[m])", 1,
        "test_p1d_interpolates_degree_q_polynomials"),
    # p schedule: the smallest instead of the largest proper divisor of an odd p
    "schedule_largest_divisor": (
        "oracle/oracle.c", "for (int d = p / 2; d >= 1; --d)", "for (int d = 1; d <= p / 2; ++d)", 1,
        "test_p_schedule"),
    # the schedule by two stepping by one
    "schedule_by_two": (
        "oracle/oracle.c", "if (schedule == 2) return p > 2 ? p - 2 : 1;",
        "if (schedule == 2) return p > 2 ? p - 1 : 1;", 1,
        "test_p_schedules_by_one_and_two"),
    # modal basis: the bubbles of the coarse order mapped one mode too high
    "modal_index": (
        "oracle/oracle.c", "static int orc_modal_index(int p, int q, int b) { return b == q ? p : b; }",
        "static int orc_modal_index(int p, int q, int b) { return b == q ? p : b + 1; }", 1,
        "test_modal_injection_rap_is_the_principal_submatrix"),
    # h-coarsening continues only while the coarse level has fewer than 5% of the rows (0.9 read)
    "coarsening_stop_ratio": (
        "oracle/oracle.c", "(double)n_agg > 0.9 * (double)f->A.n", "(double)n_agg > 0.05 * (double)f->A.n", 1,
        "test_order_one_input_with_dirichlet_rows"),
    # coarse labels for non-whole ratios: rounding up where the nearest fine node is below
    "anchor_rounding": (
        "oracle/oracle.c", "if (2 * rem < q) return f;", "if (2 * rem < q) return f + 1;", 1,
        "test_coarse_labels_injective_symmetric_and_exact_for_whole_ratios"),
    # SpGEMM: the first product of every inner row dropped
    "spgemm_dropped_term": (
        "oracle/oracle.c",
        "for (int64_t u = B->rp[k]; u < B->rp[k + 1]; ++u) {\n          double prod",
        "for (int64_t u = B->rp[k] + 1; u < B->rp[k + 1]; ++u) {\n          double prod", 1,
        "test_spgemm_matches_scipy_and_boolean_pattern"),
    # Algorithm 7: the second and third tensor directions of the coarse node transposed
    "prolongation_tensor_index": (
        "oracle/oracle.c", "tab[a2 * m1 + b2] * tab[a3 * m1 + b3]", "tab[a2 * m1 + b3] * tab[a3 * m1 + b2]", 2,
        "test_prolongation_reproduces_degree_q_fields"),
    # the hash: a finaliser shift off by one
    "hash_shift": (
        "oracle/oracle.c", "z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;", "z = (z ^ (z >> 31)) * 0xBF58476D1CE4E5B9ULL;", 1,
        "test_hash_is_the_splitmix64_finaliser"),
    # the strength test reversed (weak couplings kept), in the count and the fill pass alike
    "strength_threshold": (
        "oracle/oracle.c", "if (theta > 0.0 && !(fabs(A->v[t]) >= theta * sqrt(diag[i] * diag[j]))) continue;",
        "if (theta > 0.0 && !(fabs(A->v[t]) <= theta * sqrt(diag[i] * diag[j]))) continue;", 2,
        "test_strength_threshold_keeps_only_strong_couplings"),
    # MIS-2: the hash order reversed
    "mis2_hash_order": (
        "oracle/oracle.c", "if (ha != hb) return ha > hb;", "if (ha != hb) return ha < hb;", 1,
        "test_mis2_equals_greedy_on_squared_graph"),
    # MIS-2: the second hop of the distance-2 maximum dropped (an MIS of the graph itself)
    "mis2_second_hop": (
        "oracle/oracle.c", "int64_t j = m1[ci[t]];", "int64_t j = ci[t];", 1,
        "test_mis2_hand_worked_path"),
    # aggregation, second phase: the largest instead of the smallest aggregate id
    "aggregate_second_phase": (
        "oracle/oracle.c", "if (c >= 0 && (g < 0 || c < g)) g = c;", "if (c >= 0 && (g < 0 || c > g)) g = c;", 1,
        "test_aggregates_hand_worked_second_phase"),
    # SPAI-0: the row's sum of squares replaced by its absolute sum
    "spai0_square": (
        "oracle/oracle.c", "ss = ss + A->v[t] * A->v[t];", "ss = ss + fabs(A->v[t]);", 1,
        "test_sa_prolongation_spai0_and_constants"),
    # smoothed aggregation: T + M A T instead of T - M A T
    "sa_sign": (
        "oracle/oracle.c", "P->v[d] = tij - mi * AT.v[t];", "P->v[d] = tij + mi * AT.v[t];", 1,
        "test_sa_prolongation_spai0_and_constants"),
    # Lanczos: the beta_{j-1} v_{j-1} term dropped
    "lanczos_three_term": (
        "oracle/oracle.c", "w[i] = dsq[i] * w[i] - bprev * vp[i];", "w[i] = dsq[i] * w[i];", 1,
        "test_lanczos_estimate_within_one_percent"),
    # Lanczos: alpha_j v_j not subtracted
    "lanczos_alpha_term": (
        "oracle/oracle.c", "for (int64_t i = 0; i < n; ++i) w[i] = w[i] - a * v[i];",
        "for (int64_t i = 0; i < n; ++i) w[i] = w[i];", 1,
        "test_lanczos_ritz_bounds_finite_termination_and_start_vector"),
    # Lanczos start vector: the hash scaled by 1/512 instead of 1/1024
    "lanczos_start_vector": (
        "oracle/oracle.c", "v[i] = 1.0 + (double)(orc_hash(hash_kind, i) % 1024u) / 1024.0;",
        "v[i] = 1.0 + (double)(orc_hash(hash_kind, i) % 1024u) / 512.0;", 1,
        "test_lanczos_ritz_bounds_finite_termination_and_start_vector"),
    # Sturm count: beta not squared
    "sturm_beta_square": (
        "oracle/oracle.c", "beta[i - 1] * beta[i - 1] / d", "beta[i - 1] / d", 1,
        "test_tridiagonal_eigenvalue_by_bisection"),
    # Jacobi: the diagonal instead of its inverse
    "jacobi_inverse": (
        "oracle/oracle.c", "L->dinv[i] = 1.0 / d;", "L->dinv[i] = d;", 1,
        "test_chebyshev_damping_closed_form"),
    # Chebyshev (FP64): the factor 2 of the residual coefficient dropped
    "chebyshev_coefficient": (
        "oracle/oracle.c", "double c1 = rho_new * rho, c2 = 2.0 * rho_new / delta;",
        "double c1 = rho_new * rho, c2 = rho_new / delta;", 1,
        "test_chebyshev_damping_closed_form"),
    # Chebyshev started from zero: the first step taken twice
    "chebyshev_zero_start": (
        "oracle/oracle.c", "    x[i] = x_is_zero ? d[i] : x[i] + d[i];\n  }\n  for (int s = 1; s < k; ++s) {\n    orc_spmv(&L->A, x, r);",
        "    x[i] = x_is_zero ? 2.0 * d[i] : x[i] + d[i];\n  }\n  for (int s = 1; s < k; ++s) {\n    orc_spmv(&L->A, x, r);", 1,
        "test_chebyshev_zero_start_equals_explicit_zero"),
    # Chebyshev (FP32): rho_{s-1} dropped from the direction coefficient
    "chebyshev_fp32_coefficient": (
        "oracle/oracle.c", "float c1 = (float)(rho_new * rho)", "float c1 = (float)(rho_new)", 1,
        "test_fp32_vcycle_is_the_fp64_operator_to_fp32_rounding"),
    # FP32 V-cycle: the residual step's sign flipped
    "fp32_residual_sign": (
        "oracle/oracle.c",
        "  orc_spmv32(n, L->A.rp, L->A.ci, L->A32, x, r);\n  for (int64_t i = 0; i < n; ++i) r[i] = b[i] - r[i];\n}",
        "  orc_spmv32(n, L->A.rp, L->A.ci, L->A32, x, r);\n  for (int64_t i = 0; i < n; ++i) r[i] = r[i] - b[i];\n}", 1,
        "test_fp32_single_steps_are_their_definitions"),
    # FP32 V-cycle: the correction overwrites the smoothed iterate
    "fp32_correction_overwrites": (
        "oracle/oracle.c", "for (int64_t i = 0; i < L->A.n; ++i) x[i] = x[i] + t[i];",
        "for (int64_t i = 0; i < L->A.n; ++i) x[i] = t[i];", 1,
        "test_fp32_single_steps_are_their_definitions"),
    # FP32 V-cycle: the coarsest step hands back its right-hand side instead of the solution
    "fp32_coarse_returns_rhs": (
        "oracle/oracle.c", "for (int64_t i = 0; i < n; ++i) x[i] = (float)xd[i];",
        "for (int64_t i = 0; i < n; ++i) x[i] = (float)bd[i];", 1,
        "test_fp32_single_steps_are_their_definitions"),
    # Algorithm 1: presmoothing left out (x stays zero before the residual)
    "vcycle_no_presmoothing": (
        "oracle/oracle.c", "orc_cheb(h, L, b, x, 1);                       /* presmooth */",
        "for (int64_t i = 0; i < n; ++i) x[i] = 0.0;", 1,
        "test_vcycle_is_symmetric"),
    # the prolongation entry point overwrites instead of correcting
    "prolong_overwrites": (
        "oracle/oracle.c", "for (int64_t i = 0; i < L->A.n; ++i) xf[i] = xf[i] + t[i];",
        "for (int64_t i = 0; i < L->A.n; ++i) xf[i] = t[i];", 1,
        "test_single_steps_are_their_definitions"),
    # Algorithm 1: the coarse correction subtracted
    "coarse_correction_sign": (
        "oracle/oracle.c", "x[i] = x[i] + L->r[i]; /* correct */", "x[i] = x[i] - L->r[i]; /* correct */", 1,
        "test_pcg_matches_dense_direct_solve"),
    # Cholesky: the update reads the upper triangle (a transposed operand)
    "cholesky_transposed_operand": (
        "oracle/oracle.c", "a[(size_t)i * n + k] * a[(size_t)j * n + k];",
        "a[(size_t)i * n + k] * a[(size_t)k * n + j];", 1,
        "test_cholesky_matches_numpy"),
    # back substitution with L instead of L^T
    "back_substitution_index": (
        "oracle/oracle.c", "s = s - L[(size_t)k * n + i] * x[k];", "s = s - L[(size_t)i * n + k] * x[k];", 1,
        "test_cholesky_matches_numpy"),
    # PCG: alpha inverted
    "pcg_alpha": (
        "oracle/oracle.c", "double alpha = rho / pq;", "double alpha = pq / rho;", 1,
        "test_pcg_matches_dense_direct_solve"),
    # PCG: beta inverted
    "pcg_beta": (
        "oracle/oracle.c", "double beta = rho_new / rho;", "double beta = rho / rho_new;", 1,
        "test_pcg_matches_dense_direct_solve"),
    # flexible CG: the sign of beta
    "flexible_beta_sign": (
        "oracle/oracle.c", "double beta = orc_dot(n, z, rold) / rho;", "double beta = -orc_dot(n, z, rold) / rho;", 1,
        "test_force_iters_and_flexible_cg"),
    # the iteration limit not reported
    "maxiter_status": (
        "oracle/oracle.c", "if (status == ORC_OK && force_iters <= 0 && rr > rtol) status = ORC_ERR_MAXITER;",
        "if (status == ORC_OK && force_iters <= 0 && rr > 1.0) status = ORC_ERR_MAXITER;", 1,
        "test_iteration_limit_and_zero_right_hand_side"),
    # relative residual not divided by ||b||
    "relres_unnormalised": (
        "oracle/oracle.c", "rr = sqrt(orc_dot(n, r, r)) / bnorm;", "rr = sqrt(orc_dot(n, r, r));", 1,
        "test_force_iters_and_flexible_cg"),
    # block PCG: the sign of beta
    "block_beta_sign": (
        "oracle/block_cg.py", "beta = -gram_solve(F, Q.T @ Z)", "beta = gram_solve(F, Q.T @ Z)", 1,
        "test_block_pcg_finite_termination"),
    # block PCG: alpha transposed
    "block_alpha_transposed": (
        "oracle/block_cg.py", "alpha = gram_solve(F, P.T @ R)", "alpha = gram_solve(F, P.T @ R).T", 1,
        "test_block_pcg_finite_termination"),
    # block PCG: beta from P^T Z instead of Q^T Z
    "block_beta_operand": (
        "oracle/block_cg.py", "beta = -gram_solve(F, Q.T @ Z)", "beta = -gram_solve(F, P.T @ Z)", 1,
        "test_block_pcg_finite_termination"),
    # Gram factor: row i where row j belongs
    "gram_factor_index": (
        "oracle/block_cg.py", "L[i, j] = (s[i] * G[i, j] * s[j] - np.dot(L[i, :j], L[j, :j])) / L[j, j]",
        "L[i, j] = (s[i] * G[i, j] * s[j] - np.dot(L[i, :j], L[i, :j])) / L[j, j]", 1,
        "test_gram_pseudo_inverse_full_rank_and_singular"),
    # Gram solve: back substitution with L instead of L^T
    "gram_back_substitution": (
        "oracle/block_cg.py", "w[j] = (z[j] - L[j + 1:, j] @ w[j + 1:]) / L[j, j]",
        "w[j] = (z[j] - L[j, j + 1:] @ w[j + 1:]) / L[j, j]", 1,
        "test_gram_pseudo_inverse_full_rank_and_singular"),

    # ---- the input generator, which both the oracle and the CUDA path consume (its pins are in
    # test_fegen.py): a mistake here would not show as a parity failure
    # the stiffness metric J^-T J^-1 where J^-1 J^-T belongs
    "generator_metric_transposed": (
        "fegen/fegen.c", "g += Ji[r][d] * Ji[s][d];", "g += Ji[d][r] * Ji[d][s];", 1,
        "test_patch_test_on_jittered_elements"),
    # the off-diagonal metric terms contracted once instead of twice
    "generator_offdiagonal_once": (
        "fegen/fegen.c", "for (int tr = 0; tr < (r == s ? 1 : 2); ++tr) {", "for (int tr = 0; tr < 1; ++tr) {", 1,
        "test_patch_test_on_jittered_elements"),
    # the mass term without the Jacobian determinant
    "generator_mass_without_det": (
        "fegen/fegen.c", "W[(size_t)6 * nq3 + q] = c->prm.lambda * wdet;",
        "W[(size_t)6 * nq3 + q] = c->prm.lambda * c->qw[q1] * c->qw[q2] * c->qw[q3];", 1,
        "test_mass_matrix_integrates_volume"),
    # the trilinear map's derivative along the second axis taken with the wrong coordinate
    "generator_map_direction": (
        "fegen/fegen.c", "double n1 = L[cx][0] * dL[cy] * L[cz][2];", "double n1 = L[cx][0] * dL[cy] * L[cz][1];", 1,
        "test_mass_matrix_integrates_volume"),
    # the Lagrange derivative with one factor too many
    "generator_lagrange_derivative": (
        "fegen/fegen.c", "if (m != a && m != k) v *= (t - xi[m]) / (xi[a] - xi[m]);",
        "if (m != a) v *= (t - xi[m]) / (xi[a] - xi[m]);", 1,
        "test_laplacian_rows_sum_to_zero"),
    # the Gauss-Legendre weight with 1 + x^2 for 1 - x^2
    "generator_gauss_weight": (
        "fegen/fegen.c", "w[j] = w[n - 1 - j] = 2.0 / ((1.0 - t * t) * dp * dp);",
        "w[j] = w[n - 1 - j] = 2.0 / ((1.0 + t * t) * dp * dp);", 1,
        "test_gauss_legendre_rule"),
    # the variable-coefficient source term with the wrong sign of its kappa' term
    "generator_kappa_term_sign": (
        "fegen/fegen.c", "f -= FG_PI * FG_PI * cos(2.0 * FG_PI * x[0])", "f += FG_PI * FG_PI * cos(2.0 * FG_PI * x[0])", 1,
        "test_variable_coefficient_manufactured_solution"),
    # Dirichlet rows keep their load
    "generator_dirichlet_load": (
        "fegen/fegen.c", "    if (!c->bnd[g])\n      for (int64_t t", "    if (1)\n      for (int64_t t", 1,
        "test_variable_coefficient_manufactured_solution"),
    # modal basis: the Jacobi recurrence's last term with the wrong sign
    "generator_jacobi_recurrence": (
        "fegen/fegen.c", "const double p2 = (a2 * p1 - a3 * p0) / a1;", "const double p2 = (a2 * p1 + a3 * p0) / a1;", 1,
        ("test_oracle_pins.py", "test_modal_pcg_matches_dense_solve_and_nodal_energy")),
    # modal basis: the derivative identity's factor (n + 2)/2 for (n + 3)/2
    "generator_modal_derivative_factor": (
        "fegen/fegen.c", "const double dp = n > 0 ? 0.5 * (n + 3.0) * fg_jacobi(n - 1, 2.0, 2.0, x) : 0.0;",
        "const double dp = n > 0 ? 0.5 * (n + 2.0) * fg_jacobi(n - 1, 2.0, 2.0, x) : 0.0;", 1,
        "test_patch_test_modal_basis"),
    # modal basis: the product rule's first term with the wrong sign
    "generator_modal_derivative_sign": (
        "fegen/fegen.c", "return -0.5 * x * fg_jacobi(n, 1.0, 1.0, x) + 0.25", "return 0.5 * x * fg_jacobi(n, 1.0, 1.0, x) + 0.25", 1,
        "test_patch_test_modal_basis"),
    # the jitter drawn on [0, 1) instead of [-1, 1) times 0.2 h (every vertex pushed one way)
    "generator_jitter_range": (
        "fegen/fegen.c", "x += (2.0 * fg_unif(prm->mesh_seed, 3 * vid + 0) - 1.0) * prm->jitter / c->nx;",
        "x += fg_unif(prm->mesh_seed, 3 * vid + 0) * prm->jitter / c->nx;", 1,
        "test_jittered_mesh_recipe"),
    # the Fourier modes start at k = 0
    "generator_fourier_mode": (
        "fegen/fegen.c", "sx[k] = sin((k + 1) * FG_PI * x[0]);", "sx[k] = sin(k * FG_PI * x[0]);", 1,
        "test_fourier_load_moments"),
}

PIN_FILES = {"oracle": "test_oracle_pins.py", "fegen": "test_fegen.py"}


def _copy_tree(dst, rebuild_generator):
    skip = shutil.ignore_patterns("__pycache__", "liboracle.so*")
    shutil.copytree(os.path.join(ROOT, "oracle"), os.path.join(dst, "oracle"), ignore=skip)
    gen_skip = ("__pycache__", "libfegen.so*") if rebuild_generator else ("__pycache__",)
    shutil.copytree(os.path.join(ROOT, "fegen"), os.path.join(dst, "fegen"),
                    ignore=shutil.ignore_patterns(*gen_skip))
    os.makedirs(os.path.join(dst, "tests"))
    for f in ("conftest.py", "fp32_bounds.py", *PIN_FILES.values()):
        shutil.copy2(os.path.join(ROOT, "tests", f), os.path.join(dst, "tests", f))
    shutil.copytree(os.path.join(ROOT, "tests", "golden"), os.path.join(dst, "tests", "golden"))


def _run_pins(dst, pin_file, pins, package):
    env = {k: v for k, v in os.environ.items() if k != "PYTHONPATH"}
    env.update(OMP_NUM_THREADS="2", PYTHONDONTWRITEBYTECODE="1")
    r = subprocess.run([sys.executable, "-m", "pytest", "tests/" + pin_file, "-x", "-q",
                        "-p", "no:cacheprovider", "-k", pins],
                       cwd=dst, env=env, capture_output=True, text=True, timeout=600)
    lib = {"oracle": "liboracle.so", "fegen": "libfegen.so"}[package]
    built = os.path.exists(os.path.join(dst, package, lib))
    return r.returncode, built, r.stdout[-2000:] + r.stderr[-2000:]


def _case(base, name):
    dst = os.path.join(base, name)
    if name.startswith("control_"):
        package = name[len("control_"):]
        _copy_tree(dst, rebuild_generator=package == "fegen")
        pins = " or ".join(sorted({m[4] for m in MUTATIONS.values()
                                   if m[0].startswith(package + "/") and isinstance(m[4], str)}))
        return name, _run_pins(dst, PIN_FILES[package], pins, package)
    fname, old, new, count, pins = MUTATIONS[name]
    package = fname.split("/")[0]
    _copy_tree(dst, rebuild_generator=package == "fegen")
    path = os.path.join(dst, fname)
    with open(path) as f:
        src = f.read()
    if src.count(old) != count:
        return name, ("missing", src.count(old), "")
    with open(path, "w") as f:
        f.write(src.replace(old, new))
    pin_file, expr = pins if isinstance(pins, tuple) else (PIN_FILES[package], pins)
    return name, _run_pins(dst, pin_file, expr, package)


@pytest.fixture(scope="module")
def outcomes():
    fegen.build()
    base = tempfile.mkdtemp(prefix="oracle_mutations_")
    try:
        names = ["control_oracle", "control_fegen"] + list(MUTATIONS)
        workers = max(1, min(8, (os.cpu_count() or 2) // 2))
        with ThreadPoolExecutor(workers) as ex:
            yield dict(ex.map(lambda n: _case(base, n), names))
    finally:
        shutil.rmtree(base, ignore_errors=True)


@pytest.mark.parametrize("package", sorted(PIN_FILES))
def test_unmodified_copy_passes_every_named_pin(outcomes, package):
    rc, built, out = outcomes["control_" + package]
    assert built, "the copy's library was not the one imported"
    assert rc == 0, out


@pytest.mark.parametrize("name", list(MUTATIONS))
def test_planted_mistake_fails_a_pin(outcomes, name):
    rc, built, out = outcomes[name]
    assert rc != "missing", f"mutation site not found ({built} occurrences): the oracle changed"
    if MUTATIONS[name][0].endswith(".c"):
        assert built, "the mutated library was not the one imported"
    # pytest exits 1 when a test failed; 2 (interrupted), 4 (usage) or 5 (nothing collected)
    # would be a harness error, not a caught mistake
    assert rc == 1 and re.search(r"\b1 failed\b", out), out
