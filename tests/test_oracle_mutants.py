"""Plant plausible mistakes in the oracle (on the CPU) and check that the pins
catch every one of them.

Each mutant rewrites one line of an oracle function's source (a flipped sign,
a dropped term, a transposed operand, a wrong index) and re-executes it in the
oracle module's namespace; the pin suite of ``test_oracle_pins`` must then
fail.  A replacement that does not match the current source fails the test
too, so a mutant can never silently become a no-op.
"""
import inspect
import textwrap

import numpy as np
import pytest

import oracle.vfpi as ov
import oracle.adjoint as oadj
import oracle.checks as ochk
import oracle.delassus as odel
from tests import test_oracle_chebyshev as cheb
from tests import test_oracle_proximal as prox
from tests import test_oracle_bb as bbt
from tests import test_oracle_anisotropic as ani
from tests import test_oracle_checks as chk
from tests import test_oracle_pins as pins

MUTANTS = {
    "scatter_sign": (ov, "sweep", "v_next = v_star + w * (P.Jc.T @", "v_next = v_star - w * (P.Jc.T @"),
    "dropped_phi": (ov, "sweep", "rhs[:, 0] += P.phi", "rhs[:, 0] += 0.0 * P.phi"),
    "gradient_sign": (ov, "sweep", "v_star = v - w * (P.A @ v - P.b)", "v_star = v - w * (P.A @ v + P.b)"),
    "eta_from_v": (ov, "sweep", "eta = (P.Jc @ v_star)", "eta = (P.Jc @ v)"),
    "transposed_R": (ov, "make_problem", "data.append((sign * R[m]).ravel())",
                     "data.append((sign * R[m].transpose(0, 2, 1)).ravel())"),
    "d_contact_sign": (ov, "make_problem", "(-1.0, node_j, node_j >= 0)", "(1.0, node_j, node_j >= 0)"),
    "gamma_transposed": (ov, "gamma_blocks", '"kab,kb,kcb->kac"', '"kba,kb,kbc->kac"'),
    "w_no_square": (ov, "frobenius_w", "s = np.asarray(A.multiply(A).sum(axis=1)).ravel()",
                    "s = np.asarray(abs(A).sum(axis=1)).ravel() ** 2"),
    "w_untied": (ov, "frobenius_w", "w[dofs] = d[dofs].sum() / s[dofs].sum()", "pass"),
    "friction_radius": (ov, "project_strict", "radius = mu * lam[:, 0]", "radius = mu * np.abs(lam_star[:, 0])"),
    "slip_scale": (ov, "project_strict", "radius / np.where(inside, 1.0, rho)",
                   "rho / np.where(inside, 1.0, radius + 1e-300)"),
    "theta_no_sqrt": (ov, "sweep", "theta = math.sqrt(math.fsum(dv * dv))", "theta = math.fsum(dv * dv)"),
    "prox_no_scale": (ov, "project_proximal", "/ (1.0 + mu[edge] ** 2)", "/ (1.0 + mu[edge])"),
    "stop_off_by_one": (ov, "solve", "if r.theta < theta_th or l == l_max:",
                        "if r.theta < theta_th or l == l_max + 1:"),
    "adjoint_no_transpose": (oadj, "adjoint", "np.linalg.solve((np.eye(n) - D).T,",
                             "np.linalg.solve((np.eye(n) - D),"),
    "adjoint_mu_sign": (oadj, "strict_jacobian", "dmu[1:] = ln * t", "dmu[1:] = -ln * t"),
    "prox_jac_kappa": (oadj, "proximal_jacobian", "Pp[1:, 1:] += mu * (ln / r) * (np.eye(2) - np.outer(t, t))",
                       "Pp[1:, 1:] += (ln / r) * (np.eye(2) - np.outer(t, t))"),
    "omega_sign": (ov, "sweep", "Gam = Gam + omega", "Gam = Gam - 0.5 * omega"),
    "ccp_no_phi": (odel, "ccp_apgd", "q[0::3] += P.phi", "q[0::3] += 0.0 * P.phi"),
    "bb1_inverted": (ov, "bb_alpha", 'a = ss / sz if rule == "bb1"', 'a = sz / ss if rule == "bb1"'),
    "bb_residual_lag": (ov, "solve_bb", "v_prev, r_prev, v = v, r_l, res.v_next",
                        "v_prev, r_prev, v = v, P.A @ res.v_next - P.b, res.v_next"),
    "elliptic_axes_swapped": (ov, "project_strict_elliptic", "a = np.array([mu1[m], mu2[m]]) * ln",
                              "a = np.array([mu2[m], mu1[m]]) * ln"),
    "cheby_nu_first": (ov, "chebyshev_nu", "return 2.0 / (2.0 - rho * rho)", "return 2.0 / (2.0 - rho)"),
    "cheby_nu_rec": (ov, "chebyshev_nu", "return 4.0 / (4.0 - rho * rho * nu_prev)",
                     "return 4.0 / (4.0 - rho * nu_prev)"),
    "cheby_anchor": (ov, "solve_chebyshev", "v_next = nu * (u * (r.v_next - v) + v - v_prev) + v_prev",
                     "v_next = nu * (u * (r.v_next - v) + v - v_prev) + v"),
    "cheby_rho_latest": (ov, "solve_chebyshev",
                         "rho = min(thetas[l - 2] / thetas[l - 3], 1.0) if thetas[l - 3] > 0 else 1.0",
                         "rho = min(thetas[l - 1] / thetas[l - 2], 1.0) if thetas[l - 2] > 0 else 1.0"),
    "cheby_ls_three": (ov, "solve_chebyshev", "if l_s < (2 if rho_fixed is not None else 4):",
                       "if l_s < (2 if rho_fixed is not None else 3):"),
    "scc_zero": (ochk, "scc_terms", "return np.stack([t1, t2, t3, t4], axis=1)",
                 "return np.zeros((u.shape[0], 4))"),
    "scc_drop_normal": (ochk, "scc_terms", "np.stack([t1, t2, t3, t4], axis=1)",
                        "np.stack([0 * t1, t2, t3, t4], axis=1)"),
    "scc_drop_cone": (ochk, "scc_terms", "np.stack([t1, t2, t3, t4], axis=1)",
                      "np.stack([t1, 0 * t2, t3, t4], axis=1)"),
    "scc_drop_slip": (ochk, "scc_terms", "np.stack([t1, t2, t3, t4], axis=1)",
                      "np.stack([t1, t2, 0 * t3, t4], axis=1)"),
    "scc_drop_dissipation": (ochk, "scc_terms", "np.stack([t1, t2, t3, t4], axis=1)",
                             "np.stack([t1, t2, t3, 0 * t4], axis=1)"),
    "scc_dissipation_sign": (ochk, "scc_terms", "ut[:, None] * lam[:, 1:] + lt[:, None] * u[:, 1:]",
                             "ut[:, None] * lam[:, 1:] - lt[:, None] * u[:, 1:]"),
    "scc_residual_min": (ochk, "scc_residual", "scc_terms(u, lam, P.mu, v_scale).max()",
                         "scc_terms(u, lam, P.mu, v_scale).min()"),
    "scc_no_gap": (ochk, "contact_velocity", "u[:, 0] += P.phi", "u[:, 0] += 0.0 * P.phi"),
    "dynamics_no_contact": (ochk, "dynamics_residual", "- P.Jc.T @", "- 0.0 * P.Jc.T @"),
    "mode_slip_flipped": (ochk, "mode_of", "(lt >= mu * lam[:, 0] * (1 - 1e-9))",
                          "(lt <= mu * lam[:, 0] * (1 - 1e-9))"),
    "mode_open_strict": (ochk, "mode_of", "np.where(lam[:, 0] <= rel * scale, 0, 1)",
                         "np.where(lam[:, 0] < 0, 0, 1)"),
}


def _pin_suite():
    """Run the pins; return True if all pass."""
    rng = lambda: np.random.default_rng(1234)
    calls = [
        lambda: pins.test_strict_projection_is_disk_projection(rng()),
        lambda: pins.test_strict_projection_tie_cases(),
        lambda: pins.test_proximal_projection_is_euclidean_cone_projection(rng()),
        lambda: pins.test_lemma2_slip_derivative_norm_is_mu(rng()),
        lambda: pins.test_frobenius_w_is_the_tied_minimiser(rng()),
        lambda: pins.test_prop3_surrogate_delassus_is_diagonal(rng()),
        lambda: pins.test_single_point_mass_matches_textbook_coulomb(rng()),
        lambda: pins.test_independent_point_masses_one_sweep(rng()),
        lambda: pins.test_iterates_satisfy_surrogate_scc_exactly(rng()),
        lambda: pins.test_theta_is_two_norm_of_the_update(rng()),
        lambda: pins.test_two_point_masses_d_contact_match_textbook_impact(rng(), True),
        lambda: pins.test_gamma_blocks_are_the_dense_product_for_any_diagonal_w(rng()),
        lambda: pins.test_solve_counts_iterations_like_alg1(rng()),
        lambda: pins.test_fixed_point_is_in_enumerated_scc_set(2, 17),
        lambda: pins.test_fixed_point_is_in_enumerated_scc_set(3, 21),
        lambda: pins.test_dense_adjoint_matches_central_differences(0),
        lambda: cheb.test_nu_schedule_is_the_chebyshev_polynomial_ratio(),
        lambda: cheb.test_same_fixed_point_and_fewer_iterations(0.9),
        lambda: cheb.test_fixed_rho_is_the_textbook_chebyshev_semi_iteration(),
        lambda: prox.test_proximal_jacobian_matches_finite_differences(rng()),
        lambda: prox.test_proximal_fixed_point_is_the_ccp_solution(0, True),
        lambda: prox.test_invertible_model_recovers_impulse_from_velocity(ov.STRICT, rng()),
        lambda: bbt.test_bb_quotients_on_an_eigenvector(),
        lambda: bbt.test_without_contacts_bb_is_the_textbook_gradient_method(),
        lambda: ani.test_elliptic_projection_is_the_nearest_point(rng()),
        lambda: cheb.test_rho_is_eq_varrho_with_the_current_l(4, 1.0),
        lambda: cheb.test_rho_is_eq_varrho_with_the_current_l(6, 0.8),
        lambda: cheb.test_slow_start_before_eq_varrho_exists_is_rejected(),
        lambda: chk.test_scc_terms_flag_each_violation_in_its_column(),
        lambda: chk.test_scc_residual_is_zero_on_valid_and_at_least_the_violation_on_each_case(),
        lambda: chk.test_scc_residual_scales_with_the_gap_term(),
        lambda: chk.test_contact_velocity_uses_the_frame_and_the_d_contact_sign(),
        lambda: chk.test_dynamics_residual_hand_value(),
        lambda: chk.test_mode_of_classifies_open_stick_slip(),
    ]
    for call in calls:
        try:
            with np.errstate(all="ignore"):
                call()
        except (AssertionError, np.linalg.LinAlgError, ValueError, ArithmeticError,
                IndexError, pytest.fail.Exception):
            return False
    return True


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_planted_mistake(name, monkeypatch):
    module, fname, old, new = MUTANTS[name]
    src = textwrap.dedent(inspect.getsource(getattr(module, fname)))
    assert src.count(old) == 1, f"mutant {name} no longer matches the oracle source"
    ns = dict(vars(module))
    exec(compile(src.replace(old, new), f"<mutant {name}>", "exec"), ns)
    monkeypatch.setattr(module, fname, ns[fname])
    monkeypatch.setattr(pins, fname, ns[fname], raising=False)
    monkeypatch.setattr(prox, fname, ns[fname], raising=False)
    monkeypatch.setattr(cheb, fname, ns[fname], raising=False)
    if module is ov:
        # functions imported by name elsewhere in the oracle follow the mutant
        monkeypatch.setattr(oadj, fname, ns[fname], raising=False)
        monkeypatch.setattr(odel, fname, ns[fname], raising=False)
    assert not _pin_suite(), f"no pin caught the planted mistake {name!r}"


def test_unmutated_oracle_passes_the_suite():
    assert _pin_suite()
