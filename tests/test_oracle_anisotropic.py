"""Pins of the anisotropic (elliptic-cone) strict operator and Prop. 6."""
import numpy as np
import scipy.optimize as so

from oracle import vfpi as ov
from oracle.checks import dynamics_residual
from paper_2201_09212_gb300 import scenes
from tests.conftest import oracle_problem


def test_elliptic_projection_is_the_nearest_point(rng):
    """Nearest point of the ellipse (dense boundary sampling) and its KKT
    conditions: on the boundary, t* - t parallel to the outer normal."""
    for _ in range(200):
        ls = rng.normal(0, 1, 3)
        mu1, mu2 = rng.uniform(0.1, 1.2, 2)
        lam = ov.project_strict_elliptic(ls[None], np.array([mu1]), np.array([mu2]))[0]
        assert lam[0] == max(ls[0], 0.0)
        a = np.array([mu1, mu2]) * lam[0]
        t, ts = lam[1:], ls[1:]
        if lam[0] == 0:
            assert np.array_equal(t, [0.0, 0.0])
            continue
        q = (t[0] / a[0]) ** 2 + (t[1] / a[1]) ** 2
        assert q <= 1 + 1e-12
        ang = np.linspace(0, 2 * np.pi, 20001)
        bd = np.stack([a[0] * np.cos(ang), a[1] * np.sin(ang)], 1)
        inside = (ts[0] / a[0]) ** 2 + (ts[1] / a[1]) ** 2 <= 1
        if inside:
            assert np.array_equal(t, ts)
            continue
        assert abs(q - 1) <= 1e-10
        assert np.linalg.norm(t - ts) <= np.linalg.norm(bd - ts, axis=1).min() + 1e-12
        nrm = np.array([t[0] / a[0] ** 2, t[1] / a[1] ** 2])
        d = ts - t
        assert abs(d[0] * nrm[1] - d[1] * nrm[0]) <= 1e-9 * np.linalg.norm(d) * np.linalg.norm(nrm)
        assert d @ nrm > 0


def test_isotropic_limit_is_the_disk_projection(rng):
    ls = rng.normal(0, 1, (300, 3))
    mu = rng.uniform(0.1, 1.2, 300)
    a = ov.project_strict_elliptic(ls, mu, mu)
    b = ov.project_strict(ls, mu)
    assert np.allclose(a, b, rtol=1e-12, atol=1e-14)


def test_prop6_strict_output_is_the_maximal_dissipation_solution(rng):
    """Prop. 6: with Gamma = gamma I and lambda_n fixed by the Signorini
    condition, the strict output minimises 1/2 gamma |lambda|^2 + lambda . (eta + phi)
    over the elliptic cone section (SLSQP from several starts)."""
    for _ in range(30):
        gamma = rng.uniform(0.5, 2.0)
        eta = rng.normal(0, 1, 3)
        eta[0] = -abs(eta[0]) - 0.5            # a closing contact
        phi = 0.0
        mu1, mu2 = rng.uniform(0.2, 1.0, 2)
        ls = -(eta + [phi, 0, 0]) / gamma
        lam = ov.project_strict_elliptic(ls[None], np.array([mu1]), np.array([mu2]))[0]
        ln = lam[0]
        f = lambda t: 0.5 * gamma * (t @ t) + t @ eta[1:]
        con = {"type": "ineq", "fun": lambda t: 1 - (t[0] / (mu1 * ln)) ** 2 - (t[1] / (mu2 * ln)) ** 2}
        best = min((so.minimize(f, x0, constraints=[con], method="SLSQP",
                                options=dict(ftol=1e-15, maxiter=500))
                    for x0 in (np.zeros(2), lam[1:] * 0.5, -eta[1:] * 0.1)), key=lambda r: r.fun)
        assert f(lam[1:]) <= best.fun + 1e-9


def test_anisotropic_friction_is_not_opposite_to_sliding():
    """Sec. III.E: with mu1 != mu2 the maximal-dissipation impulse is in
    general not antiparallel to the sliding velocity (unlike the isotropic case)."""
    m = 1.0
    R = np.eye(3)[[2, 0, 1]]          # normal e_z, t1 = e_x, t2 = e_y
    b = m * np.array([1.0, 1.0, -1.0])
    P = ov.make_problem([0, 1], [0], [m * np.eye(3)], b, [0], [-1], R[None], [0.8], [0.0])
    w = ov.frobenius_w(P)
    r = ov.solve(P, w, np.zeros(3), theta_th=1e-15, l_max=10, mu2=np.array([0.2]))
    u = (P.Jc @ r.v).reshape(-1, 3)[0]
    lt, ut = r.lam[0, 1:], u[1:]
    assert np.linalg.norm(ut) > 1e-3
    cos = lt @ ut / (np.linalg.norm(lt) * np.linalg.norm(ut))
    assert cos > -0.99                 # isotropic friction would give exactly -1
    # and the isotropic case does give -1
    r0 = ov.solve(P, w, np.zeros(3), theta_th=1e-15, l_max=10)
    u0 = (P.Jc @ r0.v).reshape(-1, 3)[0]
    c0 = r0.lam[0, 1:] @ u0[1:] / (np.linalg.norm(r0.lam[0, 1:]) * np.linalg.norm(u0[1:]))
    assert c0 < -1 + 1e-12


def test_anisotropic_fixed_point_is_consistent():
    sc = scenes.terrain_lattice(dims=(10, 8, 3)).as_f64()
    P = oracle_problem(sc)
    mu2 = 0.5 * P.mu
    w = ov.frobenius_w(P)
    r = ov.solve(P, w, sc.v0, theta_th=1e-13, l_max=200000, mu2=mu2)
    assert r.converged
    assert dynamics_residual(P, r.v, r.lam) < 1e-10
