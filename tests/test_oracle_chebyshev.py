"""Pins of the Chebyshev-accelerated oracle (Alg. 3)."""
import numpy as np
import pytest
from numpy.polynomial import chebyshev as C

from oracle import vfpi as ov
from oracle.checks import dynamics_residual, scc_residual
from paper_2201_09212_gb300 import scenes
from tests.conftest import oracle_problem


def test_nu_schedule_is_the_chebyshev_polynomial_ratio():
    """From l_s on, the recurrence of Alg. 3 reproduces
    nu = 2 P_k(1/rho) / (rho P_{k+1}(1/rho)) of eq. (chebyup) for a fixed rho."""
    for rho in (0.3, 0.8, 0.95, 0.999):
        nu = 1.0
        l_s = 5
        for l in range(1, 30):
            nu = ov.chebyshev_nu(l, l_s, rho, nu)
            if l < l_s:
                assert nu == 1.0
                continue
            k = l - l_s + 1        # nu_{l_s} is the 2nd Chebyshev weight
            Tk = C.chebval(1 / rho, [0] * k + [1])
            Tk1 = C.chebval(1 / rho, [0] * (k + 1) + [1])
            assert abs(nu - 2 * Tk / (rho * Tk1)) <= 1e-12 * nu


def test_without_acceleration_it_is_alg1():
    rng = np.random.default_rng(4)
    sc = scenes.random_problem(rng, 12, 4)
    P = oracle_problem(sc)
    w = ov.frobenius_w(P)
    a = ov.solve(P, w, sc.v0, theta_th=0.0, l_max=25)
    b = ov.solve_chebyshev(P, w, sc.v0, theta_th=0.0, l_max=25, l_s=1000, u=1.0)
    # nu = u = 1 makes the update v** up to the rounding of its three additions
    assert np.abs(a.v - b.v).max() <= 1e-14 * np.abs(a.v).max()
    assert np.allclose(a.thetas, b.thetas, rtol=1e-10, atol=0)


@pytest.mark.parametrize("u", [1.0, 0.9])
def test_same_fixed_point_and_fewer_iterations(u):
    """The accelerated iteration converges to the consistent SCC solution of
    Alg. 1 (the fixed point does not depend on the schedule) and needs fewer
    sweeps (the paper's ablation, Sec. V.H)."""
    sc = scenes.small_lattice()
    P = oracle_problem(sc)
    w = ov.frobenius_w(P)
    plain = ov.solve(P, w, sc.v0, theta_th=1e-12, l_max=100000)
    acc = ov.solve_chebyshev(P, w, sc.v0, theta_th=1e-12, l_max=100000, l_s=10, u=u)
    assert acc.converged and plain.converged
    assert np.linalg.norm(acc.v - plain.v) <= 1e-9 * np.linalg.norm(plain.v)
    assert dynamics_residual(P, acc.v, acc.lam) < 1e-9
    assert scc_residual(P, acc.v, acc.lam) < 1e-9
    assert acc.iters < 0.7 * plain.iters, (acc.iters, plain.iters)


def test_chebyshev_on_terrain_patch_with_slip():
    sc = scenes.terrain_lattice(dims=(12, 10, 4)).as_f64()
    P = oracle_problem(sc)
    w = ov.frobenius_w(P)
    plain = ov.solve(P, w, sc.v0, theta_th=1e-12, l_max=100000)
    acc = ov.solve_chebyshev(P, w, sc.v0, theta_th=1e-12, l_max=100000)
    assert np.linalg.norm(acc.v - plain.v) <= 1e-8 * np.linalg.norm(plain.v)
    assert acc.iters < plain.iters


def test_fixed_rho_is_the_textbook_chebyshev_semi_iteration():
    """Without contacts and with W = alpha I, one sweep is the linear map
    v -> G v + alpha b with symmetric G = I - alpha A; with the exact spectral
    radius rho of G and l_s = 2, Alg. 3 is the Chebyshev semi-iteration, whose
    error after k accelerated steps is T_k(G / rho) e_0 / T_k(1 / rho)
    (evaluated here through the eigendecomposition of G)."""
    rng = np.random.default_rng(11)
    sc = scenes.random_problem(rng, 10, 0, density=0.3)
    P = oracle_problem(sc)
    A = P.A.toarray()
    alpha = ov.optimal_alpha(P)
    G = np.eye(P.n) - alpha * A
    lam, V = np.linalg.eigh(G)
    rho = np.abs(lam).max()
    x_star = np.linalg.solve(A, P.b)
    v0 = np.asarray(sc.v0, float)
    e0 = v0 - x_star
    for k in (1, 2, 5, 9):
        # k sweeps: the first plain (nu = 1), then the Chebyshev weights
        r = ov.solve_chebyshev(P, ov.scalar_w(P, alpha), v0, theta_th=0.0, l_max=k,
                               l_s=2, u=1.0, rho_fixed=rho)
        Tk = lambda t: C.chebval(t, [0] * k + [1])
        ek = V @ ((Tk(lam / rho) / Tk(1 / rho)) * (V.T @ e0))
        assert np.linalg.norm(r.v - x_star - ek) <= 1e-10 * np.linalg.norm(e0)


def test_gain_grows_with_the_plain_iteration_count_as_in_the_paper():
    """The paper's ablation (tests/golden/chebyshev_iterations.txt, Sec. V.H):
    Alg. 3 needs 2.2x fewer sweeps on the scenario whose plain iteration is
    short (40 sweeps) and 3.7-5.0x fewer on the three that need 139-167.  On
    the oracle, stiffer springs on the 6x6x6 lattice lengthen the plain
    iteration, and the gain of Alg. 3 (l_s = 10, u = 0.9) grows with it in
    the same way, reaching the paper's range."""
    import pathlib
    rows = [ln.split() for ln in (pathlib.Path(__file__).parent / "golden" /
                                  "chebyshev_iterations.txt").read_text().splitlines()
            if ln and not ln.startswith("#")]
    paper = sorted((float(a), float(a) / float(b)) for _, a, b in rows)
    assert [round(g, 1) for _, g in paper] == [2.2, 3.7, 5.0, 4.2]
    assert paper[0][1] < min(g for _, g in paper[1:])          # short plain runs gain least
    gains = []
    for k in (1e3, 1e4, 1e5):
        sc = scenes.lattice_scene(6, 6, 6, seed=scenes.SEED_BASE + 1, mu=0.5, k=k)
        P = oracle_problem(sc)
        w = ov.frobenius_w(P)
        plain = ov.solve(P, w, sc.v0, theta_th=1e-9, l_max=200000, norm="rms")
        acc = ov.solve_chebyshev(P, w, sc.v0, theta_th=1e-9, l_max=200000, l_s=10, u=0.9,
                                 norm="rms")
        assert plain.converged and acc.converged
        # both stop on the same step size, each within theta / (1 - rho) of the
        # fixed point, which on the stiffest lattice is a few 1e-5 relative
        assert np.linalg.norm(acc.v - plain.v) <= 1e-3 * np.linalg.norm(plain.v)
        gains.append((plain.iters, plain.iters / acc.iters))
    assert gains[0][0] < gains[1][0] < gains[2][0]
    assert gains[0][1] < gains[1][1] < gains[2][1]
    assert paper[0][1] <= gains[1][1] <= max(g for _, g in paper) + 0.5
