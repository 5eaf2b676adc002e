"""Proximal operator and invertible (regularised) contact on the GPU against the
oracle, the independent CCP solver and the dense adjoint."""
import numpy as np
import pytest

from oracle import vfpi as ov
from oracle.adjoint import adjoint as dense_adjoint
from oracle.delassus import ccp_apgd
from paper_2201_09212_gb300 import scenes
from tests.conftest import oracle_problem

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2201_09212_gb300 import vfpi  # noqa: E402


def relmax(a, b):
    a, b = np.asarray(a, float), np.asarray(b, float)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def problem(seed, n=40, nc=10, nd=3):
    rng = np.random.default_rng(seed)
    sc = scenes.random_problem(rng, n, nc, d_contacts=nd, density=0.1, couple=0.4,
                               mu_range=(0.2, 0.9), phi_scale=1.0)
    return sc, rng


@pytest.mark.parametrize("operator", ["strict", "proximal"])
@pytest.mark.parametrize("reg", [False, True])
@pytest.mark.parametrize("path", [1, 2])
def test_ladder_f64(operator, reg, path):
    sc, rng = problem(5)
    P = oracle_problem(sc)
    omega = rng.uniform(0.05, 0.3, sc.n_c) if reg else None
    om = None if omega is None else omega[:, None, None] * np.eye(3)
    w = ov.frobenius_w(P)
    with vfpi.Solver.from_scene(sc, theta_th=0.0, l_max=12, operator=operator,
                                force_path=path) as s:
        s.set_regularization(omega)
        r = s.solve(sc.v0)
    ref = ov.solve(P, w, sc.v0, theta_th=0.0, l_max=12,
                   operator=ov.PROXIMAL if operator == "proximal" else ov.STRICT, omega=om)
    assert relmax(r.v, ref.v) <= 1e-11
    assert relmax(np.asarray(r.lam).reshape(-1, 3), ref.lam) <= 1e-10


@pytest.mark.parametrize("reg", [False, True])
def test_proximal_converges_to_the_ccp_solution(reg):
    sc, rng = problem(8, n=20, nc=5, nd=1)
    P = oracle_problem(sc)
    omega = rng.uniform(0.05, 0.3, sc.n_c) if reg else None
    v_ccp, lam_ccp, _ = ccp_apgd(P, omega)
    with vfpi.Solver.from_scene(sc, theta_th=1e-13, l_max=200000, operator="proximal") as s:
        s.set_regularization(omega)
        r = s.solve(sc.v0)
    assert r.converged
    assert np.linalg.norm(r.v - v_ccp) <= 1e-8 * np.linalg.norm(v_ccp)


def test_invertible_model_f32_recovers_impulse():
    sc = scenes.terrain_lattice(dims=(24, 20, 4))
    P = oracle_problem(sc)
    omega = np.full(sc.n_c, 1e-3 * 0 + 0.2 * float(np.median(ov.frobenius_w(P))), dtype=np.float32)
    with vfpi.Solver.from_scene(sc, theta_th=1e-9, l_max=20000, operator="proximal") as s:
        s.set_regularization(omega)
        r = s.solve(sc.v0)
    v = np.asarray(r.v, float)
    lam = np.asarray(r.lam, float).reshape(-1, 3)
    u = (P.Jc @ v).reshape(-1, 3)
    u[:, 0] += P.phi
    lam_inv = ov.project_proximal(-u / omega.astype(float)[:, None], P.mu)
    assert relmax(lam_inv, lam) <= 1e-3
    assert (lam[:, 0] > 0).any()


@pytest.mark.parametrize("operator,reg", [("proximal", False), ("proximal", True),
                                          ("strict", True)])
def test_adjoint_f64_with_operator_and_regularisation(operator, reg):
    sc, rng = problem(12)
    P = oracle_problem(sc)
    omega = rng.uniform(0.05, 0.3, sc.n_c) if reg else None
    om = None if omega is None else omega[:, None, None] * np.eye(3)
    w = ov.frobenius_w(P)
    opk = ov.PROXIMAL if operator == "proximal" else ov.STRICT
    ref = ov.solve(P, w, sc.v0, theta_th=1e-14, l_max=300000, operator=opk, omega=om)
    assert ref.converged
    g_v = rng.normal(0, 1, sc.n)
    g_b, g_phi, g_mu, _ = dense_adjoint(P, w, ref.v, g_v, operator=opk, omega=omega)
    with vfpi.Solver.from_scene(sc, theta_th=1e-13, l_max=300000, operator=operator) as s:
        s.set_regularization(omega)
        r = s.solve(sc.v0)
        assert r.converged
        gb, gp, gm, _, _ = s.adjoint(g_v)
    assert relmax(gb, g_b) <= 1e-8
    assert relmax(gp, g_phi) <= 1e-8
    assert relmax(gm, g_mu) <= 1e-7


def test_regularization_rejects_negative_omega():
    sc, _ = problem(1)
    with vfpi.Solver.from_scene(sc) as s:
        with pytest.raises(vfpi.VfpiError):
            s.set_regularization(np.full(sc.n_c, -1.0))
