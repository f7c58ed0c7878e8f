"""Planted mistakes in the oracle and in the input generators (no GPU).

Each mutant changes one expression of one oracle (or generator) function the way a
transcription slip would -- a dropped term, a wrong sign, index or coefficient,
a transposed operand, a stale variable -- and at least one of the oracle's own
pins must then fail.  This is the evidence that the pins constrain every part
of the oracle, not only the code paths they happen to exercise.

A mutant is compiled from the function's source with one substring replaced and
installed in place of the original (module attribute, class attribute and every
`from module import name` binding) for the duration of the check only; the
oracle's files are never modified.
"""
import ast
import contextlib
import importlib
import inspect
import sys
import textwrap

import numpy as np
import pytest

import test_oracle_adjoint as TD
import test_oracle_amg as TA
import test_oracle_mlp as TM
import test_oracle_params as TP
import test_oracle_sa as TSA
import test_oracle_smoother as TS
import test_problems as TPR
from oracle import smoother as oracle_smoother
from paper_2407_09848_gb300 import problems as pr


def _resolve(target):
    modname, qual = target.split(":")
    mod = importlib.import_module(modname)
    owner = mod
    parts = qual.split(".")
    for p in parts[:-1]:
        owner = getattr(owner, p)
    return mod, owner, parts[-1]


@contextlib.contextmanager
def mutant(target, old, new):
    """Install ``target`` ("module:function" or "module:Class.method") with the
    first occurrence of ``old`` in its source replaced by ``new``."""
    mod, owner, name = _resolve(target)
    orig = getattr(owner, name)
    src = textwrap.dedent(inspect.getsource(orig))
    # search the code only: skip the docstring, which may spell out the formula
    fn = ast.parse(src).body[0]
    start = 0
    if ast.get_docstring(fn) is not None:
        doc = fn.body[0]
        lines = src.splitlines(keepends=True)
        start = sum(len(l) for l in lines[:doc.end_lineno - 1]) + doc.end_col_offset
    i = src.find(old, start)
    assert i >= 0, f"{target}: {old!r} not in the code"
    ns = dict(mod.__dict__)
    exec(compile(src[:i] + new + src[i + len(old):], f"<mutant of {target}>", "exec"), ns)
    mut = ns[name]
    rebound = []
    setattr(owner, name, mut)
    if owner is mod:
        for m in list(sys.modules.values()):
            d = getattr(m, "__dict__", None)
            if m is not mod and isinstance(d, dict) and d.get(name) is orig:
                d[name] = mut
                rebound.append(m)
    oracle_smoother._OPT4_CACHE.clear()
    try:
        yield
    finally:
        setattr(owner, name, orig)
        for m in rebound:
            m.__dict__[name] = orig
        oracle_smoother._OPT4_CACHE.clear()


# ---- pin groups (each calls pins of the oracle's own test files) ----

def smoother_pins(*kinds):
    def run():
        for kind, extra in TS.KIND_CASES:
            if kind in kinds:
                for k in (1, 2, 4):
                    TS.test_diagonal_error_propagation(kind, extra, k)
                TS.test_periodic_laplacian_fourier(kind, extra, 3)
    return run


def l1_pins():
    TS.test_l1_diag_by_hand()
    TS.test_periodic_laplacian_fourier("l1jacobi", None, 1)


def power_pins():
    TS.test_power_lambda_closed_form()


def astar_pins():
    TP.test_a_star_k1_closed_form()
    for row in TP.ROWS[:5]:
        TP.test_a_star_matches_printed(row)


def poly_pins():
    TP.test_W4_is_fourth_kind()
    TP.test_opt4_with_unit_weights_is_plain_cheb4()
    for row in TP.ROWS[:4]:
        TP.test_gamma_cheb4(row)


def opt4_pins():
    TP.test_opt4_k1_k2_closed_forms()
    TP.test_opt4_weights_reach_printed_gamma(TP.ROWS[3])


def cheb1_param_pins():
    for row in TP.ROWS[:4]:
        TP.test_gamma_cheb1_opt(row)
    TP.test_cheb1_coeffs_reproduce_tau(3)
    TP.test_tau_recurrence_matches_closed_form()


def vcycle_pins():
    TA.test_vcycle_equals_dense_composition("cheb4_opt", {}, 2)


def pcg_pins():
    TA.test_pcg_matches_dense_solve("cheb4_opt", {})
    TA.test_pcg_precond_hook_textbook_cases()
    TA.test_flexible_pcg_matches_dense_solve_and_standard_on_linear_precond()
    for flexible in (True, False):
        TA.test_conjugacy_defect_under_a_variable_preconditioner(flexible)


def fcg_pins():
    TA.test_fcg1_textbook_cases()
    TA.test_fcg1_equals_pcg_on_fixed_spd_preconditioner()


def coarse_pins():
    TA.test_coarse_l1jacobi_sweeps_dense_composition()


def sa_pins():
    TSA.test_1d_pairs_closed_form()
    TSA.test_constant_preserved_where_rows_sum_to_zero()
    for st in (pr.poisson(8), pr.varcoef(7, 1.0, 3.0, seed=3, ny=6, nz=5), pr.aniso(6, 1e-2)):
        TSA.test_galerkin_dense_brute_force_and_spd(st)


def adjoint_pins(*kinds):
    def run():
        for kind, kw in TD.KINDS + [("weights", {})]:
            if kind in kinds:
                for k in (2, 4):
                    TD.test_smooth_backward_central_differences(kind, kw, k)
                TD.test_smooth_operator_is_symmetric(kind, kw)
    return run


def sa_hierarchy_pins():
    TSA.test_sa_hierarchy_pcg_32()


def vcycle_adjoint_pins():
    TD.test_vcycle_backward_symmetric_and_fd()


def loss_pins():
    TD.test_error_reduction_loss_gradient_fd()


def generator_pins():
    TPR.test_poisson_stencil_values()
    TPR.test_aniso_weak_direction_is_z()
    TPR.test_varcoef_faces_are_harmonic_means_and_boundary_faces_the_cell_value()
    TPR.test_grf_correlation_length()


def mlp_pins():
    TM.test_forward_by_hand()
    TM.test_backward_central_differences()
    TM.test_adam_first_step_closed_form()


SM = "oracle.smoother:"
PA = "oracle.params:"
AM = "oracle.amg:OracleAMG."
SA = "oracle.sa:"
AD = "oracle.adjoint:"
ML = "oracle.mlp:"
GE = "paper_2407_09848_gb300.problems:"

# (id, target, original text, planted mistake, pins that must catch it)
MUTANTS = [
    # 4th-kind recurrence (Eq. polsmoother / polsmootheropt)
    ("cheb4_c1_index", SM + "cheb4", "(2 * j - 3) / (2 * j + 1) * z", "(2 * j - 1) / (2 * j + 1) * z",
     smoother_pins("cheb4", "cheb4_opt")),
    ("cheb4_c2_denominator", SM + "cheb4", "(8 * j - 4) / (2 * j + 1) / rho",
     "(8 * j - 4) / (2 * j - 1) / rho", smoother_pins("cheb4")),
    ("cheb4_no_Minv", SM + "cheb4", "/ rho * (r / M)", "/ rho * r", smoother_pins("cheb4")),
    ("cheb4_rho_inverted", SM + "cheb4", "(8 * j - 4) / (2 * j + 1) / rho", "(8 * j - 4) / (2 * j + 1) * rho",
     smoother_pins("cheb4")),
    ("cheb4opt_weighted_r", SM + "cheb4", "r = r - A @ z", "r = r - bj * (A @ z)",
     smoother_pins("cheb4_opt")),
    ("cheb4_drops_a_residual", SM + "cheb4", "if j < k:", "if j < k - 1:", smoother_pins("cheb4")),
    ("cheb4_residual_sign", SM + "cheb4", "r = b - A @ x", "r = b + A @ x", smoother_pins("cheb4")),
    ("cheb4opt_weights_ignored", SM + "smooth", "cheb4(A, b, x0, spec.k, spec.beta, spec.rho, M=M)",
     "cheb4(A, b, x0, spec.k, None, spec.rho, M=M)", smoother_pins("cheb4_opt")),
    # Algorithm 1
    ("cheb1_r_sign", SM + "cheb1", "r = r - s", "r = r + s", smoother_pins("cheb1_opt")),
    ("cheb1_dropped_rho_prev", SM + "cheb1", "d = rho_j * rho_prev * d", "d = rho_j * d",
     smoother_pins("cheb1_opt")),
    ("cheb1_delta_for_theta", SM + "cheb1", "d = r / theta", "d = r / delta",
     smoother_pins("cheb1_opt")),
    ("cheb1_theta_for_delta", SM + "cheb1", "(2.0 * rho_j / delta) * r", "(2.0 * rho_j / theta) * r",
     smoother_pins("cheb1_opt")),
    ("cheb1_stale_rho", SM + "cheb1", "rho_prev = rho_j", "rho_prev = rho_prev",
     smoother_pins("cheb1_opt")),
    ("cheb1_rho_dropped_in_s", SM + "cheb1", "s = ((A @ d) / M) / rho", "s = ((A @ d) / M)",
     smoother_pins("cheb1")),
    # l1-Jacobi, l1 diagonal, power estimate
    ("jacobi_times_M", SM + "l1jacobi", "(b - A @ x) / M", "(b - A @ x) * M",
     smoother_pins("l1jacobi")),
    ("l1_diag_counts_diagonal_twice", SM + "l1_diag", "d + (absrow - np.abs(d))", "d + absrow",
     l1_pins),
    ("l1_diag_signed_sum", SM + "l1_diag", "abs(A).sum(axis=1)", "A.sum(axis=1)", l1_pins),
    ("power_not_normalised", SM + "power_lambda", "v = w / lam", "v = w", power_pins),
    # scalar parameters (Sec. 2.1-2.3)
    ("W4_third_kind", PA + "W4", "np.sin((j + 0.5) * th[big]) / np.sin(0.5 * th[big])",
     "np.cos((j + 0.5) * th[big]) / np.cos(0.5 * th[big])", poly_pins),
    ("p_cheb4_argument", PA + "p_cheb4", "1.0 - 2.0 * np.asarray", "1.0 - np.asarray", poly_pins),
    ("p_opt4_weight_difference", PA + "p_opt4", "(b[j] - b[j + 1])", "(b[j + 1] - b[j])", poly_pins),
    ("astar_not_squared", PA + "a_star", "return r * r", "return r", astar_pins),
    ("astar_equation_coefficient", PA + "phi_astar", "8 * k *", "4 * k *", astar_pins),
    ("theta_delta_swapped", PA + "theta_delta", "0.5 * (1.0 + a), 0.5 * (1.0 - a)",
     "0.5 * (1.0 - a), 0.5 * (1.0 + a)", cheb1_param_pins),
    ("c1_binomial_index", PA + "inv_two_c1", "math.comb(2 * k, 2 * j + 1)", "math.comb(2 * k, 2 * j)",
     cheb1_param_pins),
    ("cheb1_coeffs_recurrence", PA + "cheb1_coeffs", "1.0 / (2.0 * s1 - rhos[-1])",
     "1.0 / (2.0 * s1 + rhos[-1])", cheb1_param_pins),
    ("opt4_derivative_condition_sign", PA + "opt4_weights", "d0 @ beta_of(g) + 1.0 / (2.0 * g)",
     "d0 @ beta_of(g) - 1.0 / (2.0 * g)", opt4_pins),
    ("opt4_alternation_dropped", PA + "opt4_weights", "signs * w - 1.0", "w - 1.0", opt4_pins),
    # V-cycle (Eq. amg) and the outer solvers (Sec. 4)
    ("vcycle_restricts_b", AM + "vcycle", "bc = P.T @ r", "bc = P.T @ b", vcycle_pins),
    ("vcycle_no_post_smoothing", AM + "vcycle", "x = smooth(A, b, x, spec, M=M)", "x = x", vcycle_pins),
    ("vcycle_correction_sign", AM + "vcycle", "x = x + P @ xc", "x = x - P @ xc", vcycle_pins),
    ("vcycle_residual_sign", AM + "vcycle", "r = b - A @ x", "r = b + A @ x", vcycle_pins),
    ("pcg_beta_inverted", AM + "pcg", "beta = rz_new / rz", "beta = rz / rz_new", pcg_pins),
    ("pcg_alpha_denominator", AM + "pcg", "alpha = rz / (p @ q)", "alpha = rz / (p @ p)", pcg_pins),
    ("pcg_flexible_term_dropped", AM + "pcg", "beta = (rz_new - r @ z_old) / rz",
     "beta = (rz_new + r @ z_old) / rz", pcg_pins),
    ("fcg1_beta_sign", AM + "fcg1", "beta = gamma / eta", "beta = -gamma / eta", fcg_pins),
    ("fcg1_eta_update", AM + "fcg1", "eta = delta - beta * gamma", "eta = delta", fcg_pins),
    ("coarse_sweep_count", AM + "coarse_solve", 'SmootherSpec("l1jacobi", self.coarse_sweeps)',
     'SmootherSpec("l1jacobi", self.coarse_sweeps - 1)', coarse_pins),
    # smoothed aggregation (Sec. 4) and the Galerkin product (Sec. 2)
    ("sa_omega_inverted", SA + "sa_prolongator", "omega = 4.0 / (3.0 * lambda_bound(A))",
     "omega = 3.0 / (4.0 * lambda_bound(A))", sa_pins),
    ("sa_smoothing_sign", SA + "sa_prolongator", "P = Ph - omega *", "P = Ph + omega *", sa_pins),
    ("sa_lambda_unscaled", SA + "lambda_bound", "/ A.diagonal()", "/ A.diagonal().max()", sa_pins),
    ("galerkin_drops_A", SA + "galerkin", "P.T @ (sp.csr_matrix(A) @ P)", "P.T @ P", sa_pins),
    # reverse mode
    ("adjoint_beta_index", AD + "_cheb4_backward", "gbeta[j] = xbar @ zs[j]",
     "gbeta[j] = xbar @ zs[j - 1]", adjoint_pins("weights")),
    ("adjoint_r_update_sign", AD + "_cheb4_backward", "zbar = zbar - A @ rbar",
     "zbar = zbar + A @ rbar", adjoint_pins("cheb4")),
    ("adjoint_cheb1_theta", AD + "_cheb1_backward", "rbar = rbar + dbar / theta",
     "rbar = rbar + dbar / delta", adjoint_pins("cheb1_opt")),
    ("adjoint_jacobi_transposed_scaling", AD + "_jacobi_backward", "t = xbar / M", "t = xbar * M",
     adjoint_pins("l1jacobi")),
    ("adjoint_vcycle_restriction", AD + "vcycle_backward", "gres = P @ gbc", "gres = P @ gxc",
     vcycle_adjoint_pins),
    ("cheb1_zero_start_rho", SM + "cheb1", "r = (np.asarray(b, dtype=np.float64) / M) / rho",
     "r = (np.asarray(b, dtype=np.float64) / M)", smoother_pins("cheb1")),
    ("tau_map_reversed", PA + "tau_scaled", "(th - x) / de", "(x - th) / de", cheb1_param_pins),
    ("c1_numerator_power", PA + "inv_two_c1", "a ** j for j in range(k + 1)",
     "a ** (j + 1) for j in range(k + 1)", cheb1_param_pins),
    ("vcycle_no_pre_smoothing", AM + "vcycle", "x = smooth(A, b, None, spec, M=M)",
     "x = np.zeros_like(b)", vcycle_pins),
    ("coarse_cholesky_transposed", AM + "coarse_solve", "sla.solve_triangular(self.L.T, y, lower=False)",
     "sla.solve_triangular(self.L, y, lower=True)", vcycle_pins),
    ("pcg_x_along_z", AM + "pcg", "x = x + alpha * p", "x = x + alpha * z", pcg_pins),
    ("sa_tentative_transposed", SA + "tentative", "(np.arange(n), agg)", "(agg, np.arange(n))", sa_pins),
    ("loss_gradient_factor", AD + "error_reduction_loss", "gz = -2.0 * Ae1 / den / m",
     "gz = -Ae1 / den / m", loss_pins),
    ("power_one_step_short", SM + "power_lambda", "for _ in range(iters):",
     "for _ in range(iters - 1):", power_pins),
    ("jacobi_polynomial_exponent", PA + "p_jacobi", "** k", "** (k + 1)", smoother_pins("l1jacobi")),
    # (the 4th-kind and optimal 1st-kind sups equal the limit at x -> 0, which
    # gamma_sup takes analytically, so the objective itself is pinned by the
    # optimised 4th-kind series, whose maxima the Remez exchange locates with it)
    ("objective_denominator", PA + "f_objective", "(1.0 - p * p)", "(1.0 + p * p)", opt4_pins),
    ("gamma_limit_at_zero", PA + "gamma_sup", "best = 1.0 / (2.0 * abs(pprime0))",
     "best = 1.0 / abs(pprime0)", poly_pins),
    ("W4_derivative", PA + "W4_deriv_at_one", "j * (j + 1) * (2 * j + 1) / 3.0",
     "j * (j + 1) * (2 * j + 1) / 6.0", poly_pins),
    ("T1_outside_sign", PA + "T1", "(-1.0) ** k * np.cosh", "np.cosh", cheb1_param_pins),
    ("value_at_one_q", PA + "value_at_one", "q = (1 + s) / (1 - s)", "q = (1 + a) / (1 - a)",
     cheb1_param_pins),
    ("opt4_basis_index", PA + "_phi_basis", "W4(j - 1, t) / (2 * j - 1)", "W4(j - 1, t) / (2 * j + 1)",
     opt4_pins),
    ("amg_coarse_diag_level", AM + "__init__", "self.Mc = l1_diag(self.A[-1])",
     "self.Mc = l1_diag(self.A[0])[:self.A[-1].shape[0]]", coarse_pins),
    ("sa_hierarchy_stale_level", SA + "sa_hierarchy", "P, om = sa_prolongator(As[-1], agg, nc)",
     "P, om = sa_prolongator(As[0], agg, nc)", sa_hierarchy_pins),
    ("sa_lambda_signed", SA + "lambda_bound", "abs(A).sum(axis=1)", "A.sum(axis=1)", sa_pins),
    ("adjoint_cheb1_recurrence", AD + "_cheb1_backward", "c1, c2 = rhos[j] * rhos[j - 1], 2.0 * rhos[j] / delta",
     "c1, c2 = rhos[j], 2.0 * rhos[j] / delta", adjoint_pins("cheb1_opt")),
    ("adjoint_cheb1_rho", AD + "_cheb1_backward", "gb = (rbar / M) / rho", "gb = rbar / M",
     adjoint_pins("cheb1")),
    ("adjoint_vcycle_pre_input", AD + "vcycle_backward", "gx1 = gx1 - A @ gres", "gx1 = gx1 + A @ gres",
     vcycle_adjoint_pins),
    ("adjoint_vcycle_prolong_transposed", AD + "vcycle_backward", "gxc = P.T @ gx2", "gxc = P.T @ xbar",
     vcycle_adjoint_pins),
    ("adjoint_dispatch_beta", AD + "smooth_backward", 'beta = None if kd == "cheb4" else spec.beta',
     "beta = None", adjoint_pins("weights")),
    # the seeded input generators both sides consume
    ("gen_arithmetic_mean_faces", GE + "varcoef", "2.0 * a[..., :-1] * a[..., 1:] / (a[..., :-1] + a[..., 1:])",
     "0.5 * (a[..., :-1] + a[..., 1:])", generator_pins),
    ("gen_neumann_boundary", GE + "varcoef", "f = np.concatenate([a[..., :1], inner, a[..., -1:]], axis=-1)",
     "f = np.concatenate([0 * a[..., :1], inner, 0 * a[..., -1:]], axis=-1)", generator_pins),
    ("gen_aniso_axis", GE + "aniso", "np.full((nz + 1, ny, nx), float(eps))",
     "np.ones((nz + 1, ny, nx))", generator_pins),
    ("gen_grf_filter_width", GE + "grf", "s = ell / np.sqrt(2.0)", "s = ell", generator_pins),
    ("gen_diag_drops_face", GE + "_from_faces", "+ fz[:-1, :, :] + fz[1:, :, :]", "+ fz[1:, :, :]",
     generator_pins),
    # MLP of the learned weights
    ("mlp_output_scale", ML + "forward", "np.exp(2.0 * t)", "np.exp(t)", mlp_pins),
    ("mlp_tanh_argument", ML + "forward", "t = np.tanh(0.5 * o)", "t = np.tanh(o)", mlp_pins),
    ("mlp_layer1_bias", ML + "forward", 'a1 = F @ P["W1"].T + P["b1"]', 'a1 = F @ P["W1"].T', mlp_pins),
    ("mlp_layer2_transposed", ML + "forward", 'a2 = h1 @ P["W2"].T + P["b2"]',
     'a2 = h1 @ P["W2"] + P["b2"]', mlp_pins),
    ("mlp_hidden_relu", ML + "forward", "h2 = np.maximum(a2, 0.0)", "h2 = a2", mlp_pins),
    ("mlp_layer2_gradient", ML + "backward", "gW2 = ga2.T @ h1", "gW2 = ga2.T @ a1", mlp_pins),
    ("adam_second_moment", ML + "adam", "v = b2 * v + (1 - b2) * grad * grad",
     "v = b2 * v + (1 - b2) * grad", mlp_pins),
    ("mlp_tanh_derivative", ML + "backward", "(1.0 - t * t)", "(1.0 - t)", mlp_pins),
    ("mlp_relu_mask", ML + "backward", "ga1 = gh1 * (a1 > 0)", "ga1 = gh1", mlp_pins),
    ("adam_bias_correction", ML + "adam", "mh = m / (1 - b1 ** step)", "mh = m", mlp_pins),
]


def test_pin_groups_pass_on_the_oracle():
    groups = {id(m[4]): m[4] for m in MUTANTS}
    for run in groups.values():
        run()


@pytest.mark.filterwarnings("ignore::RuntimeWarning")   # a mutant may produce NaNs
@pytest.mark.parametrize("mid,target,old,new,pins", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_is_caught(mid, target, old, new, pins):
    with mutant(target, old, new):
        with pytest.raises(Exception):
            pins()
