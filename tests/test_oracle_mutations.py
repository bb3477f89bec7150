"""Planted mistakes: each case edits a copy of the oracle's C source (a flipped sign, a
dropped term, a transposed operand, a wrong constant), builds it, and checks that at
least one of the pins in test_oracle_pins.py fails against it.  This shows the pins
would catch such a mistake in the oracle itself.  Everything runs on the CPU."""
import os
import subprocess

import pytest

import oracle
import test_oracle_pins as pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "tron_oracle.c")

# (name, original text, mutated text, pins expected to catch it)
MUTATIONS = [
    ("flow p_ij: sign of the g_ij wR term",
     "F[0] = cf[0] * wi - cf[2] * wR + cf[3] * wI;",
     "F[0] = cf[0] * wi + cf[2] * wR + cf[3] * wI;",
     [pins.test_branch_flows_match_complex_power]),
    ("branch Hessian: sign of d2 wR / dv_i dth_i",
     "HwR[0 * 4 + 2] = -vj * sn;", "HwR[0 * 4 + 2] = vj * sn;",
     [pins.test_branch_gradient_hessian_finite_differences]),
    ("line-limit gradient: factor 2 dropped",
     "dm[a] = 2.0 * p * dF[kp][a] + 2.0 * q * dF[kq][a];",
     "dm[a] = 1.0 * p * dF[kp][a] + 2.0 * q * dF[kq][a];",
     [pins.test_branch_gradient_hessian_finite_differences]),
    ("dense gradient: quartic coefficient",
     "if (g) g[i] = qx + cv[i] + 4.0 * d[i] * x2 * x[i];",
     "if (g) g[i] = qx + cv[i] + 3.0 * d[i] * x2 * x[i];",
     [pins.test_dense_eval_closed_form, pins.test_separable_quartic_closed_form]),
    ("Cholesky: transposed operand in the column update",
     "for (int k = 0; k < j; k++) v -= L[(size_t)i * m + k] * L[(size_t)j * m + k];",
     "for (int k = 0; k < j; k++) v -= L[(size_t)k * m + i] * L[(size_t)j * m + k];",
     [pins.test_chol_matches_numpy]),
    ("trqsol: wrong root",
     "return (rad - ptx) / ptp;", "return (-rad - ptx) / ptp;",
     [pins.test_trqsol_is_positive_root]),
    ("projected gradient: upper-bound rule",
     "if (x[i] >= u[i] && p < 0.0) p = 0.0;", "if (x[i] >= u[i] && p > 0.0) p = 0.0;",
     [pins.test_pgnorm_definition_cases]),
    ("PCG: residual not updated",
     "res[i] -= alpha * q[i];", "res[i] -= 0.0 * q[i];",
     [pins.test_steihaug_one_iteration_on_pd]),
    ("Cauchy search: sufficient-decrease test reversed",
     "ok = (q <= o->mu0 * gts) && (cauchy_len(n, s, Hd, o, c) <= o->mu1 * delta);",
     "ok = (q >= o->mu0 * gts) && (cauchy_len(n, s, Hd, o, c) <= o->mu1 * delta);",
     [pins.test_separable_quadratic_closed_form, pins.test_newton_step_solves_an_interior_quadratic_in_one_iteration]),
    ("back transform: direction sign",
     "for (int a = 0; a < m; a++) w[F[a]] = sh[a];",
     "for (int a = 0; a < m; a++) w[F[a]] = -sh[a];",
     [pins.test_newton_step_solves_an_interior_quadratic_in_one_iteration]),
    ("hs45 gradient sign",
     "g[i] = -q;", "g[i] = q;",
     [pins.test_hs45_printed_solution]),
    ("ADMM bus update: sign of mu on the flow copies",
     "st->br_tilde[4 * (size_t)k + kp] = val[kp] + lam[kp] / rho + mu1 / rho;",
     "st->br_tilde[4 * (size_t)k + kp] = val[kp] + lam[kp] / rho - mu1 / rho;",
     [pins.test_admm_bus_update_kkt_and_multipliers]),
    ("ADMM generator update: linear cost dropped",
     "double p = (rho * pt - lp - net->gen_c1[g]) / (2.0 * net->gen_c2[g] + rho);",
     "double p = (rho * pt - lp) / (2.0 * net->gen_c2[g] + rho);",
     [pins.test_admm_generator_update_is_scalar_qp_minimiser]),
    ("ADMM multiplier update sign",
     "*lam += rho * (xv - xt);",
     "*lam -= rho * (xv - xt);",
     [pins.test_admm_bus_update_kkt_and_multipliers]),
    ("generator chain: sign of the ramp gradient",
     "g[t] += rr * e * s;", "g[t] -= rr * e * s;",
     [pins.test_genramp_gradient_hessian_finite_differences]),
    ("generator chain: sign of the Hessian's subdiagonal",
     "H[t * n + (t - 1)] -= rr;", "H[t * n + (t - 1)] += rr;",
     [pins.test_genramp_gradient_hessian_finite_differences]),
    ("generator chain: ramp term dropped from f",
     "val += 0.5 * rr * e * e;", "val += 0.0 * rr * e * e;",
     [pins.test_genramp_binding_ramps_vs_lbfgsb]),
    ("multi-period record: targets from the multipliers",
     "rec[8 + T + t] = mp->states[t].gen_tilde[2 * g];",
     "rec[8 + T + t] = mp->states[t].gen_lam[2 * g];",
     [pins.test_multiperiod_admm_without_binding_ramps_equals_single_period_runs]),
    ("line limit: a NaN excess counted as exceeded",
     "    if (m > 0.0) {", "    if (!(m <= 0.0)) {",
     [pins.test_branch_entries_that_enter_f_only_past_the_line_limit]),
    ("acceptance: ratio test reversed",
     "if (rho > o->eta0) {", "if (rho < o->eta0) {",
     [pins.test_separable_quadratic_closed_form, pins.test_dense_convex_vs_lbfgsb]),
    ("dense Hessian: quartic term halved",
     "H[(size_t)i * n + i] += 12.0 * d[i] * x[i] * x[i];",
     "H[(size_t)i * n + i] += 6.0 * d[i] * x[i] * x[i];",
     [pins.test_dense_eval_closed_form]),
    ("radius update: expansion factor 2 instead of 4",
     "o->sigma3 = 4.0;", "o->sigma3 = 2.0;",
     [pins.test_cauchy_interpolation_preconditioned_boundary_and_expansion,
      pins.radius_update_all_cases]),
    ("radius update: shrink factor 0.5 instead of 0.25",
     "o->sigma1 = 0.25;", "o->sigma1 = 0.5;",
     [pins.test_radius_shrinks_to_a_quarter_of_the_shorter_of_step_and_radius]),
    ("radius update: shrink ignores the step length",
     "delta = o->sigma1 * (snorm < delta ? snorm : delta);", "delta = o->sigma1 * delta;",
     [pins.test_radius_shrinks_to_a_quarter_of_the_shorter_of_step_and_radius]),
    ("radius update: eta2 test on the wrong side",
     "} else if (rho > o->eta2 && snorm >= 0.99 * delta) {",
     "} else if (rho < o->eta2 && snorm >= 0.99 * delta) {",
     [pins.radius_update_all_cases]),
    ("radius update: expansion needs the full radius",
     "} else if (rho > o->eta2 && snorm >= 0.99 * delta) {",
     "} else if (rho > o->eta2 && snorm >= 1.0 * delta) {",
     [pins.radius_update_all_cases]),
    ("radius update: step measured in the Euclidean norm under the PCG's norm",
     "double snorm = o->tr_norm == 0 ? nu : nrm2(n, s, c);", "double snorm = nrm2(n, s, c);",
     [pins.test_cauchy_interpolation_preconditioned_boundary_and_expansion]),
    ("Cauchy search: extrapolation factor 5 instead of 10",
     "o->extrapf = 10.0;", "o->extrapf = 5.0;",
     [pins.test_cauchy_extrapolation_stops_at_the_largest_breakpoint]),
    ("Cauchy search: interpolation factor 0.2 instead of 0.1",
     "o->interpf = 0.1;", "o->interpf = 0.2;",
     [pins.test_cauchy_interpolation_preconditioned_boundary_and_expansion]),
    ("Cauchy search: extrapolation does not stop at the largest breakpoint",
     "if (!(alpha < bmax)) break;", "if (!(alpha < 1e300)) break;",
     [pins.test_cauchy_extrapolation_stops_at_the_largest_breakpoint]),
    ("Cauchy search: alpha restarts at 1 every iteration",
     "    alpha_c = alpha;\n", "    alpha_c = 1.0;\n",
     [pins.test_cauchy_alpha_persists_between_iterations]),
    ("projected search: step quartered instead of halved",
     "o->proj_shrink = 0.5;", "o->proj_shrink = 0.25;",
     [pins.test_projected_search_halves_the_step_until_the_model_decreases]),
    ("PCG: boundary tested on w instead of the CG iterate",
     "if (nrm2(m, norm == 0 ? sn : wn, c) >= delta) {", "if (nrm2(m, wn, c) >= delta) {",
     [pins.test_steihaug_one_iteration_on_pd,
      pins.test_cauchy_interpolation_preconditioned_boundary_and_expansion]),
    ("ratio guard: scaled by |f| instead of the magnitude of the terms",
     "double fl = o->ared_guard * (fs > 1.0 ? fs : 1.0);",
     "double fl = o->ared_guard * (fabs(f) > 1.0 ? fabs(f) : 1.0);",
     [pins.test_branch_solves_at_an_admm_state_all_converge]),
    ("Hessian-norm Cauchy test: no fallback where s'Hs <= 0",
     "    if (h > 0.0) return sqrt(h);\n", "    return sqrt(fabs(h));\n",
     [pins.test_cauchy_test_in_the_hessian_norm_option]),
    ("Hessian-norm Cauchy test: the option ignored",
     "  if (o->cauchy_norm == 1) {\n    double h", "  if (o->cauchy_norm == 7) {\n    double h",
     [pins.test_cauchy_test_in_the_hessian_norm_option]),
    ("guard scale: the branch flows' own terms left out",
     "mag += fabs(lam[k] * r) + 0.5 * rh[k] * r * r + (fabs(lam[k]) + rh[k] * fabs(r)) * M[k];",
     "mag += fabs(lam[k] * r) + 0.5 * rh[k] * r * r;",
     [pins.test_guard_scale_is_the_magnitude_of_the_terms_of_f]),
]


@pytest.fixture(scope="module")
def source():
    with open(SRC) as fh:
        return fh.read()


@pytest.mark.parametrize("case", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_pins_catch_planted_mistake(case, source, tmp_path):
    name, old, new, catchers = case
    assert source.count(old) == 1, f"mutation site not unique: {old}"
    src = tmp_path / "tron_oracle.c"
    src.write_text(source.replace(old, new))
    lib = tmp_path / "liboracle_mut.so"
    hdr = os.path.dirname(SRC)
    subprocess.run(["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fPIC", "-shared",
                    "-I", hdr, "-o", str(lib), str(src), "-lm", "-lpthread"], check=True)
    caught = []
    with oracle.using_library(str(lib)):
        for pin in catchers:
            try:
                pin()
            except Exception:  # an assertion, or a numerical failure of the pin
                caught.append(pin.__name__)
    assert caught, f"no pin caught: {name}"
