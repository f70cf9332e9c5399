"""Plant plausible mistakes in a copy of the oracle and check the pins catch them.

Each mutant is a one-line textual change to ``oracle/pcg_oracle.c`` (a dropped
term, a flipped sign, a wrong index or operand), compiled on the CPU into a
temporary library.  The committed oracle is never modified.  A mutant passes
this test only if at least one pin of ``test_oracle_pins`` rejects it.
"""
import os
import subprocess

import numpy as np
import pytest

from oracle import oracle as O
from tests import test_oracle_gibbs as gibbs
from tests import test_oracle_pins as pins

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                   "oracle", "pcg_oracle.c")

MUTANTS = {
    "drop_eta_term": ("        b[j] = b[j] + t[j];", "        b[j] = b[j];"),
    "eta_without_sqrt": ("w[i] = sqrt(omega[i]) * eta[i];", "w[i] = omega[i] * eta[i];"),
    "delta_term_squared_scale": ("b[j] = b[j] + delta[j] / (tau * lam[j]);",
                                 "b[j] = b[j] + delta[j] / (tau * tau * lam[j] * lam[j]);"),
    "residual_sign": ("r[j] = r[j] - alpha * v[j];", "r[j] = r[j] + alpha * v[j];"),
    "wrong_preconditioner": ("z[j] = minv ? minv[j] * r[j] : prior_var(tau, lam[j]) * r[j];\n            }",
                             "z[j] = minv ? minv[j] * r[j] : prior_prec(tau, lam[j]) * r[j];\n            }"),
    "gamma_inverted": ("double gamma = rho_new / rho;", "double gamma = rho / rho_new;"),
    "omega_index": ("work[i] = omega[i] * work[i];", "work[i] = omega[i / 2] * work[i];"),
    "prior_diag_dropped": ("out[j] = out[j] + prior_prec(tau, lam[j]) * v[j];",
                           "out[j] = out[j];"),
    "xt_uses_wrong_index": ("acc += w[row_idx[k]];", "acc += w[row_idx[k] / 2];"),
    "dense_phi_omega_index": ("+= omega[i];", "+= omega[col_idx[a] % n];"),
    "chol_transposed_operand": ("e -= a[i * p + k] * a[j * p + k];", "e -= a[i * p + k] * a[k * p + j];"),
    "rms_divisor": ("return sqrt(rho / (double)p) <= tol;", "return sqrt(rho) <= tol;"),
    "beta_step_uses_v": ("beta[j] = beta[j] + alpha * s[j];", "beta[j] = beta[j] + alpha * v[j];"),
    "comp_sum_drops_compensation": ("        a->c += (a->s - t) + x;", "        a->c += 0.0;"),
    "phi_diag_without_prior": ("        out[j] = out[j] + prior_prec(tau, lam[j]);\n}",
                               "        out[j] = out[j];\n}"),
    "warm_start_residual_sign": ("r[j] = b[j] - v[j];            /* r_0 = b - Phi beta_0 */",
                                 "r[j] = b[j] + v[j];            /* r_0 = b - Phi beta_0 */"),
    "jacobi_stop_uses_cg_rho": ("rho_s = (minv == NULL) ? rho_new : stop_norm2(sum_mode, p, r, lam, tau, tmp);",
                                "rho_s = rho_new;"),
    "lsqr_theta_uses_c": ("const double theta = sn * alf;", "const double theta = c * alf;"),
    "lsqr_bottom_block_dropped": ("u[n + j] = v[j] - alf * u[n + j];", "u[n + j] = - alf * u[n + j];"),
    "lsqr_eta_dropped": ("u[i] = sqrt(omega[i]) * z[i] + eta[i];", "u[i] = sqrt(omega[i]) * z[i];"),
    "philox_wrong_weyl": ("k1 += 0xBB67AE85u;", "k1 += 0xBB67AE86u;"),
    "pg_coef_exponent": ("exp(-h * h * 9.869604401089358 * x / 2.0)", "exp(-h * h * 9.869604401089358 * x)"),
    "pg_mixture_weight": ("const double r = p / (p + q);", "const double r = q / (p + q);"),
    "pg_half_tilt": ("const double t = 0.64, z = 0.5 * fabs(c);", "const double t = 0.64, z = fabs(c);"),
    "lambda_scale_tau_not_squared": ("beta[j] * beta[j] / (2.0 * (*tau) * (*tau))) / orng_exp(&g));",
                                     "beta[j] * beta[j] / (2.0 * (*tau))) / orng_exp(&g));"),
    "tau_shape_drops_one": ("orng_gamma(&g, 0.5 * (double)(p + 1))", "orng_gamma(&g, 0.5 * (double)(p + 3))"),
    "augmented_response_times_omega": ("z[i] = (y[i] - 0.5) / omega[i];", "z[i] = (y[i] - 0.5) * omega[i];"),
}

# the pins that run against each mutant (the slow statistical ones are left out:
# every mutant below is caught by a deterministic pin)
PIN_TESTS = [
    pins.test_b_design_without_nonzeros_is_prior_term,
    pins.test_b_single_row_by_hand,
    pins.test_phi_mul_equals_dense_phi_times_v,
    pins.test_xt_mul_is_transpose_of_x_mul,
    pins.test_dense_phi_matches_numpy,
    pins.test_cholesky_and_solve_match_lapack,
    lambda: pins.test_direct_draw_equals_least_squares("small"),
    pins.test_tiny_exact_rational_draw,
    pins.test_cg_matches_cholesky_config1,
    pins.test_cg_exact_after_p_iterations,
    lambda: pins.test_thm22_low_rank_converges_in_k_plus_1(3),
    pins.test_design_without_nonzeros_one_iteration,
    pins.test_rho_is_true_preconditioned_residual,
    pins.test_stop_rule_rms_is_first_crossing,
    pins.test_thm21_error_bound_and_monotone_phi_norm_error,
    pins.test_compensated_sums_match_correctly_rounded_sums,
    pins.test_phi_diag_is_diagonal_of_dense_phi,
    pins.test_jacobi_pcg_reaches_the_cholesky_solution,
    pins.test_warm_start,
    pins.test_lsqr_solves_the_normal_equations,
    pins.test_lsqr_iterates_equal_pcg_iterates,
    pins.test_lsqr_residual_estimate_is_eq_s2,
    gibbs.test_philox_known_answers,
    gibbs.test_polya_gamma_series_forms_agree,
    lambda: gibbs.test_polya_gamma_moments(0.4),
    lambda: gibbs.test_polya_gamma_moments(8.0),
    gibbs.test_scale_updates_draw_their_conditionals,
    gibbs.test_gibbs_step_composes_the_cycle,
]


def _caught(lib_path):
    prev = O.use_library(lib_path)
    try:
        for t in PIN_TESTS:
            try:
                with np.errstate(all="ignore"):
                    t()
            except Exception:
                return True
        return False
    finally:
        O.use_library(prev)


def test_unmutated_copy_passes(tmp_path):
    """Control: the same harness accepts an unmodified copy."""
    src = open(SRC).read()
    c = tmp_path / "ok.c"
    c.write_text(src)
    so = str(tmp_path / "ok.so")
    subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-o", so, str(c), "-lm"])
    assert not _caught(so)


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_reject_mutant(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation site for {name} not unique"
    c = tmp_path / f"{name}.c"
    c.write_text(src.replace(old, new))
    so = str(tmp_path / f"{name}.so")
    subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-o", so, str(c), "-lm"])
    assert _caught(so), f"no pin rejects mutant {name}"


# --------------------------------------------------------------------------
# the unshrunk-coefficient functions of oracle.py (Sec. S4.3), plain numpy:
# each mutant is a one-line change to a copy of the module's source
# --------------------------------------------------------------------------
PY_SRC = os.path.join(os.path.dirname(SRC), "oracle.py")

PY_MUTANTS = {
    "unshrunk_prior_term_without_sqrt": ("    sd[:q1] = np.sqrt(prior_prec)", "    sd[:q1] = prior_prec"),
    "unshrunk_gamma_not_squared": ("    m[:q1] = np.asarray(gamma, dtype=np.float64) ** 2",
                                   "    m[:q1] = np.asarray(gamma, dtype=np.float64)"),
    "unshrunk_keeps_shrinkage_prior": ("    d[:q1] = prior_prec\n", "    d[:q1] = d[:q1]\n"),
    "unshrunk_eta_without_sqrt": ("omega * z + np.sqrt(omega) * eta) + sd * delta",
                                  "omega * z + omega * eta) + sd * delta"),
    "unshrunk_pcg_wrong_preconditioner": ("        zz = m * r\n        rho_new", "        zz = d * r\n        rho_new"),
    "unshrunk_phi_drops_omega": ("xd.T @ (_f64(omega)[:, None] * xd) + np.diag(d)", "xd.T @ xd + np.diag(d)"),
}

UNSHRUNK_PINS = [
    pins.test_unshrunk_reduces_to_shrunk_when_scales_match,
    pins.test_unshrunk_flat_prior_intercept_closed_form,
    pins.test_unshrunk_cg_matches_cholesky_and_ignores_gamma,
]


def _py_module(src):
    import types
    mod = types.ModuleType("oracle_copy")
    mod.__file__ = PY_SRC   # the compiled C routines are found beside the source
    exec(compile(src, PY_SRC, "exec"), mod.__dict__)
    return mod


def _py_caught(mod, monkeypatch):
    monkeypatch.setattr(pins, "O", mod)
    for t in UNSHRUNK_PINS:
        try:
            with np.errstate(all="ignore"):
                t()
        except Exception:
            return True
    return False


def test_unmutated_python_copy_passes(monkeypatch):
    """Control: the harness accepts an unmodified copy of oracle.py."""
    assert not _py_caught(_py_module(open(PY_SRC).read()), monkeypatch)


@pytest.mark.parametrize("name", sorted(PY_MUTANTS))
def test_unshrunk_pins_reject_mutant(name, monkeypatch):
    old, new = PY_MUTANTS[name]
    src = open(PY_SRC).read()
    assert src.count(old) == 1, f"mutation site for {name} not unique"
    assert _py_caught(_py_module(src.replace(old, new)), monkeypatch), f"no pin rejects mutant {name}"
