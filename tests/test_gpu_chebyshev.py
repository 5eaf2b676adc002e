"""Chebyshev-accelerated V-FPI (Alg. 3) on the GPU against the oracle's Alg. 3."""
import numpy as np
import pytest

from oracle import vfpi as ov
from oracle.checks import scc_residual
from paper_2201_09212_gb300 import scenes
from tests.conftest import oracle_problem

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2201_09212_gb300 import vfpi  # noqa: E402


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, float) - b) / np.linalg.norm(b))


@pytest.mark.parametrize("path", [1, 2])
@pytest.mark.parametrize("l_s,u", [(5, 0.9), (4, 1.0)])
def test_ladder_f64_matches_oracle_alg3(path, l_s, u):
    rng = np.random.default_rng(21)
    sc = scenes.random_problem(rng, 60, 10, d_contacts=4, density=0.08, couple=0.4)
    P = oracle_problem(sc)
    w = ov.frobenius_w(P)
    with vfpi.Solver.from_scene(sc, theta_th=0.0, l_max=1, force_path=path,
                                chebyshev_ls=l_s, chebyshev_u=u) as s:
        for k in (2, 7, 25):
            s.set_tolerance(0.0, k)
            r = s.solve(sc.v0)
            ref = ov.solve_chebyshev(P, w, sc.v0, theta_th=0.0, l_max=k, l_s=l_s, u=u)
            assert rel(r.v, ref.v) <= 1e-11, k
            # theta is a difference of iterates: its error scales with ||v||
            assert abs(r.theta - ref.theta) <= 1e-9 * ref.theta + 1e-13 * np.linalg.norm(ref.v)


def test_converged_f64_same_iterations_and_fixed_point():
    sc = scenes.small_lattice(np.float64)
    P = oracle_problem(sc)
    w = ov.frobenius_w(P)
    ref = ov.solve_chebyshev(P, w, sc.v0, theta_th=1e-10, l_max=100000, l_s=10, u=0.9)
    plain = ov.solve(P, w, sc.v0, theta_th=1e-13, l_max=100000)
    with vfpi.Solver.from_scene(sc, theta_th=1e-10, l_max=100000, chebyshev_ls=10,
                                chebyshev_u=0.9) as s:
        r = s.solve(sc.v0)
    assert r.converged and r.iters == ref.iters
    assert rel(r.v, plain.v) <= 1e-8


def test_f32_terrain_fewer_sweeps_same_solution():
    sc = scenes.terrain_lattice(dims=(40, 36, 6))
    P = oracle_problem(sc)
    plain = ov.solve(P, ov.frobenius_w(P), sc.v0, theta_th=1e-13, l_max=100000)
    with vfpi.Solver.from_scene(sc, theta_th=1e-7, l_max=5000, norm="rms") as s:
        r0 = s.solve(sc.v0)
        s.set_chebyshev(10, 0.9)
        r1 = s.solve(sc.v0)
    assert r1.converged and r0.converged
    assert r1.iters < 0.8 * r0.iters, (r1.iters, r0.iters)
    assert rel(r1.v, plain.v) <= 1e-5
    assert scc_residual(P, np.asarray(r1.v, float), np.asarray(r1.lam, float).reshape(-1, 3)) <= 1e-6


def test_batched_chebyshev_equals_per_scene():
    lat = scenes.batched_lattices(8, seed=3, side_range=(4, 7))
    batch = scenes.concat_scenes(lat)
    kw = dict(theta_th=1e-6, l_max=500, block_threads=128, chebyshev_ls=6, chebyshev_u=0.9)
    with vfpi.Solver.from_scene(batch, **kw) as s:
        rb = s.solve(batch.v0)
    o = 0
    for q, sc in enumerate(lat):
        with vfpi.Solver.from_scene(sc, force_path=2, **kw) as s1:
            r1 = s1.solve(sc.v0)
        assert r1.iters == rb.iters[q]
        assert np.array_equal(r1.v, rb.v[o:o + sc.n])
        o += sc.n


def test_invalid_chebyshev_settings_are_rejected():
    sc = scenes.small_lattice(np.float64)
    with pytest.raises(vfpi.VfpiError):
        vfpi.Solver.from_scene(sc, chebyshev_ls=2)
    with pytest.raises(vfpi.VfpiError):
        vfpi.Solver.from_scene(sc, chebyshev_ls=3)   # eq. varrho has no value yet at l = 3
    with vfpi.Solver.from_scene(sc) as s:
        with pytest.raises(vfpi.VfpiError):
            s.set_chebyshev(5, 1.5)
