"""Anisotropic (elliptic-cone) friction on the GPU against the oracle (Prop. 6)."""
import numpy as np
import pytest

from oracle import vfpi as ov
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


@pytest.mark.parametrize("path", [1, 2])
def test_ladder_f64_with_s_and_d_contacts(path):
    rng = np.random.default_rng(41)
    sc = scenes.random_problem(rng, 50, 12, d_contacts=4, density=0.1, couple=0.4,
                               mu_range=(0.2, 1.0), phi_scale=1.0)
    P = oracle_problem(sc)
    mu2 = rng.uniform(0.05, 1.2, sc.n_c)
    w = ov.frobenius_w(P)
    ref = ov.solve(P, w, sc.v0, theta_th=0.0, l_max=15, mu2=mu2)
    with vfpi.Solver.from_scene(sc, theta_th=0.0, l_max=15, force_path=path) as s:
        s.set_anisotropic_friction(mu2)
        r = s.solve(sc.v0)
    assert relmax(r.v, ref.v) <= 1e-11
    assert relmax(np.asarray(r.lam).reshape(-1, 3), ref.lam) <= 1e-10
    slip = np.hypot(ref.lam[:, 1] / sc.mu, ref.lam[:, 2] / mu2) >= ref.lam[:, 0] * (1 - 1e-9)
    assert (slip & (ref.lam[:, 0] > 0)).any(), "no contact on the elliptic boundary"


def test_f32_terrain_converged_and_isotropic_limit():
    sc = scenes.terrain_lattice(dims=(30, 24, 4))
    P = oracle_problem(sc)
    mu2 = (0.4 * sc.mu).astype(np.float32)
    ref = ov.solve(P, ov.frobenius_w(P), sc.v0, theta_th=1e-13, l_max=200000, mu2=mu2)
    with vfpi.Solver.from_scene(sc, theta_th=1e-9, l_max=20000) as s:
        s.set_anisotropic_friction(mu2)
        r = s.solve(sc.v0)
        assert np.linalg.norm(r.v - ref.v) <= 1e-5 * np.linalg.norm(ref.v)
        # mu2 = mu gives back the isotropic solve bit for bit up to the projection's rounding
        s.set_anisotropic_friction(sc.mu)
        r1 = s.solve(sc.v0)
        s.set_anisotropic_friction(None)
        r0 = s.solve(sc.v0)
    assert np.linalg.norm(r1.v - r0.v) <= 1e-6 * np.linalg.norm(r0.v)


def test_unsupported_combinations_are_reported():
    rng = np.random.default_rng(2)
    sc = scenes.random_problem(rng, 10, 3)
    with vfpi.Solver.from_scene(sc) as s:
        s.set_anisotropic_friction(np.full(sc.n_c, 0.3))
        s.solve(sc.v0)
        with pytest.raises(vfpi.VfpiError) as e:
            s.adjoint(np.ones(sc.n))
        assert e.value.status == -7
    with vfpi.Solver.from_scene(sc, operator="proximal") as s:
        with pytest.raises(vfpi.VfpiError) as e:
            s.set_anisotropic_friction(np.full(sc.n_c, 0.3))
        assert e.value.status == -7
