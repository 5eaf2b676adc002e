"""Pins of the Barzilai-Borwein step-size oracle (Sec. IV.C)."""
import numpy as np
import pytest

from oracle import vfpi as ov
from oracle.checks import dynamics_residual, scc_residual
from paper_2201_09212_gb300 import scenes
from tests.conftest import oracle_problem


def test_bb_quotients_on_an_eigenvector():
    """On an eigenvector of A (z = sigma s) both BB rules return 1 / sigma."""
    rng = np.random.default_rng(0)
    Q, _ = np.linalg.qr(rng.normal(size=(6, 6)))
    sig = np.array([1.0, 2.0, 3.0, 5.0, 7.0, 11.0])
    A = Q @ np.diag(sig) @ Q.T
    for k in range(6):
        s = Q[:, k] * 0.7
        z = A @ s
        assert abs(ov.bb_alpha(s, z, "bb1", -1.0) - 1 / sig[k]) < 1e-14
        assert abs(ov.bb_alpha(s, z, "bb2", -1.0) - 1 / sig[k]) < 1e-14
    # Cauchy-Schwarz: bb2 <= bb1 for any SPD A
    s = rng.normal(size=6)
    assert ov.bb_alpha(s, A @ s, "bb2", 0) <= ov.bb_alpha(s, A @ s, "bb1", 0)
    # non-positive curvature keeps the previous step
    assert ov.bb_alpha(s, -s, "bb1", 0.123) == 0.123


def test_without_contacts_bb_is_the_textbook_gradient_method():
    """No contacts: v^{l+1} = v^l - alpha_l (A v^l - b) with alpha_l the BB
    quotient of the last two iterates -- checked against a direct transcription
    of the gradient method on the dense system."""
    rng = np.random.default_rng(5)
    sc = scenes.random_problem(rng, 8, 0, density=0.4)
    P = oracle_problem(sc)
    A = P.A.toarray()
    a0 = 0.5 / np.linalg.eigvalsh(A).max()
    r = ov.solve_bb(P, sc.v0, theta_th=0.0, l_max=12, alpha0=a0, rule="bb1")
    x_prev, x, alpha = None, np.asarray(sc.v0, float), a0
    for l in range(12):
        g = A @ x - P.b
        if x_prev is not None:
            s, y = x - x_prev, g - (A @ x_prev - P.b)
            alpha = (s @ s) / (s @ y)
        x_prev, x = x, x - alpha * g
    assert np.allclose(r.v, x, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("rule", ["bb1", "bb2", "alt"])
def test_bb_converges_to_the_same_contact_solution(rule):
    sc = scenes.small_lattice()
    P = oracle_problem(sc)
    w = ov.frobenius_w(P)
    ref = ov.solve(P, w, sc.v0, theta_th=1e-13, l_max=100000)
    a0 = float(np.median(w))
    r = ov.solve_bb(P, sc.v0, theta_th=1e-13, l_max=100000, alpha0=a0, rule=rule)
    assert r.converged
    assert np.linalg.norm(r.v - ref.v) <= 1e-9 * np.linalg.norm(ref.v)
    assert dynamics_residual(P, r.v, r.lam) < 1e-9 and scc_residual(P, r.v, r.lam) < 1e-9
