"""Pins of the proximal operator, the invertible (regularised) contact model and
their adjoints (Prop. 5, eq. ccp, eq. invt)."""
import copy

import numpy as np
import pytest

from oracle import vfpi as ov
from oracle.adjoint import adjoint, proximal_jacobian
from oracle.checks import mode_of
from oracle.delassus import ccp_apgd
from paper_2201_09212_gb300 import scenes
from tests.conftest import oracle_problem


def test_proximal_jacobian_matches_finite_differences(rng):
    eps = 1e-7
    n = 0
    while n < 60:
        x = rng.normal(0, 1, 3)
        mu = rng.uniform(0.1, 1.5)
        Pp, dmu = proximal_jacobian(x, mu)
        for k in range(3):
            e = np.zeros(3)
            e[k] = eps
            col = (ov.project_proximal((x + e)[None], np.array([mu]))[0]
                   - ov.project_proximal((x - e)[None], np.array([mu]))[0]) / (2 * eps)
            assert np.allclose(Pp[:, k], col, atol=1e-6)
        dm = (ov.project_proximal(x[None], np.array([mu + eps]))[0]
              - ov.project_proximal(x[None], np.array([mu - eps]))[0]) / (2 * eps)
        assert np.allclose(dmu, dm, atol=1e-6)
        n += 1


@pytest.mark.parametrize("seed", range(4))
@pytest.mark.parametrize("reg", [False, True])
def test_proximal_fixed_point_is_the_ccp_solution(seed, reg):
    """Sec. III.D: converged V-FPI with the proximal operator solves the convex
    contact problem (eq. ccp), with Gamma + Omega for the invertible model
    (eq. invt); checked against accelerated projected gradient on the dense
    Delassus QP."""
    rng = np.random.default_rng(700 + seed)
    sc = scenes.random_problem(rng, 10, 4, d_contacts=1, mu_range=(0.2, 0.9), couple=0.4,
                               phi_scale=1.0)
    P = oracle_problem(sc)
    omega = rng.uniform(0.05, 0.3, P.n_c) if reg else None
    om = None if omega is None else omega[:, None, None] * np.eye(3)
    w = ov.frobenius_w(P)
    r = ov.solve(P, w, sc.v0, theta_th=1e-13, l_max=200000, operator=ov.PROXIMAL, omega=om)
    assert r.converged
    v_ccp, lam_ccp, _ = ccp_apgd(P, omega)
    assert np.linalg.norm(r.v - v_ccp) <= 1e-8 * np.linalg.norm(v_ccp)
    assert np.abs(r.lam - lam_ccp).max() <= 1e-7 * np.abs(lam_ccp).max()


@pytest.mark.parametrize("operator", [ov.STRICT, ov.PROXIMAL])
def test_invertible_model_recovers_impulse_from_velocity(operator, rng):
    """eq. invt: with Omega_m = omega_m I the impulse follows from the velocity
    alone, lambda = ProjectFC(-(J v + phi e_n) / omega)."""
    sc = scenes.random_problem(rng, 12, 5, mu_range=(0.2, 0.9), couple=0.4, phi_scale=1.0)
    P = oracle_problem(sc)
    omega = rng.uniform(0.05, 0.3, P.n_c)
    w = ov.frobenius_w(P)
    r = ov.solve(P, w, sc.v0, theta_th=1e-13, l_max=200000, operator=operator,
                 omega=omega[:, None, None] * np.eye(3))
    u = (P.Jc @ r.v).reshape(-1, 3)
    u[:, 0] += P.phi
    proj = ov.project_strict if operator == ov.STRICT else ov.project_proximal
    lam_inv = proj(-u / omega[:, None], P.mu)
    assert np.abs(lam_inv - r.lam).max() <= 1e-9 * np.abs(r.lam).max()
    assert (mode_of(r.lam, P.mu) > 0).any()


@pytest.mark.parametrize("operator,reg", [(ov.PROXIMAL, False), (ov.PROXIMAL, True),
                                          (ov.STRICT, True)])
def test_adjoint_with_operator_and_regularisation_matches_fd(operator, reg):
    rng = np.random.default_rng(31)
    sc = scenes.random_problem(rng, 8, 3, mu_range=(0.2, 0.8), couple=0.3, phi_scale=1.0)
    P = oracle_problem(sc)
    omega = rng.uniform(0.05, 0.3, P.n_c) if reg else None
    om = None if omega is None else omega[:, None, None] * np.eye(3)
    w = ov.frobenius_w(P)
    solve = lambda Q, v0: ov.solve(Q, w, v0, theta_th=1e-14, l_max=300000, operator=operator,
                                   omega=om)
    base = solve(P, sc.v0)
    c = rng.normal(0, 1, P.n)
    g_b, g_phi, g_mu, _ = adjoint(P, w, base.v, c, operator=operator, omega=omega)
    eps = 1e-6
    for field, k, g in [("b", 3, g_b), ("b", 11, g_b), ("phi", 0, g_phi), ("phi", 2, g_phi),
                        ("mu", 1, g_mu)]:
        vals = []
        for d in (eps, -eps):
            Q = copy.copy(P)
            arr = getattr(P, field).copy()
            arr[k] += d
            setattr(Q, field, arr)
            vals.append(c @ solve(Q, base.v).v)
        fd = (vals[0] - vals[1]) / (2 * eps)
        assert abs(fd - g[k]) <= 1e-5 * max(1.0, abs(fd)), (field, k, fd, g[k])
