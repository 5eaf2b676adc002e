"""Barzilai-Borwein step sizes (Sec. IV.C) on the GPU against the oracle."""
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


@pytest.mark.parametrize("rule", ["bb1", "bb2", "alt"])
@pytest.mark.parametrize("path", [1, 2])
def test_ladder_f64_matches_oracle(rule, path):
    rng = np.random.default_rng(61)
    sc = scenes.random_problem(rng, 50, 10, d_contacts=4, density=0.1, couple=0.4)
    P = oracle_problem(sc)
    a0 = float(np.median(ov.frobenius_w(P)))
    with vfpi.Solver.from_scene(sc, theta_th=0.0, l_max=1, force_path=path) as s:
        s.set_barzilai_borwein(rule, a0)
        for k in (1, 2, 9, 25):
            s.set_tolerance(0.0, k)
            r = s.solve(sc.v0)
            ref = ov.solve_bb(P, sc.v0, theta_th=0.0, l_max=k, alpha0=a0, rule=rule)
            assert np.abs(r.v - ref.v).max() <= 1e-10 * np.abs(ref.v).max(), k


def test_converged_f32_terrain_same_solution_fewer_sweeps():
    sc = scenes.terrain_lattice(dims=(40, 36, 6))
    P = oracle_problem(sc)
    plain = ov.solve(P, ov.frobenius_w(P), sc.v0, theta_th=1e-13, l_max=100000)
    a0 = float(np.median(ov.frobenius_w(P)))
    with vfpi.Solver.from_scene(sc, theta_th=1e-7, l_max=5000, norm="rms") as s:
        r0 = s.solve(sc.v0)
        s.set_barzilai_borwein("bb1", a0)
        r1 = s.solve(sc.v0)
    assert r0.converged and r1.converged
    assert r1.iters < r0.iters
    assert np.linalg.norm(r1.v - plain.v) <= 1e-5 * np.linalg.norm(plain.v)


def test_batched_bb_equals_per_scene():
    lat = scenes.batched_lattices(6, seed=9, side_range=(4, 7))
    batch = scenes.concat_scenes(lat)
    with vfpi.Solver.from_scene(batch, theta_th=1e-6, l_max=500, block_threads=128) as s:
        s.set_barzilai_borwein("alt", 50.0)
        rb = s.solve(batch.v0)
    o = 0
    for q, sc in enumerate(lat):
        with vfpi.Solver.from_scene(sc, theta_th=1e-6, l_max=500, block_threads=128,
                                    force_path=2) as s1:
            s1.set_barzilai_borwein("alt", 50.0)
            r1 = s1.solve(sc.v0)
        assert r1.iters == rb.iters[q]
        assert np.array_equal(r1.v, rb.v[o:o + sc.n])
        o += sc.n


def test_bb_exclusions():
    rng = np.random.default_rng(1)
    sc = scenes.random_problem(rng, 10, 2)
    with vfpi.Solver.from_scene(sc, chebyshev_ls=5, chebyshev_u=0.9) as s:
        with pytest.raises(vfpi.VfpiError) as e:
            s.set_barzilai_borwein("bb1", 0.1)
        assert e.value.status == -7
    with vfpi.Solver.from_scene(sc) as s:
        s.set_barzilai_borwein("bb1", 0.1)
        s.solve(sc.v0)
        with pytest.raises(vfpi.VfpiError) as e:
            s.adjoint(np.ones(sc.n))
        assert e.value.status == -7
        with pytest.raises(vfpi.VfpiError):
            s.set_barzilai_borwein(1, -1.0)
