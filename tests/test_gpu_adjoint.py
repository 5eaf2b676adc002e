"""Adjoint of the converged V-FPI fixed point on the GPU against the dense FP64
oracle adjoint (itself pinned by central differences and Lemma 2)."""
import numpy as np
import pytest

from oracle import vfpi as ov
from oracle.adjoint import adjoint as dense_adjoint
from oracle.checks import mode_of
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


def reference(sc, g_v):
    P = oracle_problem(sc)
    w = ov.frobenius_w(P)
    ref = ov.solve(P, w, sc.v0, theta_th=1e-14, l_max=200000)
    assert ref.converged
    g_b, g_phi, g_mu, _ = dense_adjoint(P, w, ref.v, g_v)
    return ref, g_b, g_phi, g_mu, P


@pytest.mark.parametrize("seed", range(3))
def test_adjoint_f64_s_and_d_contacts(seed):
    rng = np.random.default_rng(900 + seed)
    sc = scenes.random_problem(rng, 60, 10, d_contacts=5, density=0.08, couple=0.3,
                               mu_range=(0.2, 0.8), phi_scale=1.0)
    g_v = rng.normal(0, 1, sc.n)
    ref, g_b, g_phi, g_mu, P = reference(sc, g_v)
    modes = mode_of(ref.lam, P.mu)
    with vfpi.Solver.from_scene(sc, theta_th=1e-13, l_max=100000) as s:
        r = s.solve(sc.v0)
        assert r.converged
        gb, gp, gm, it, th = s.adjoint(g_v)
        assert th < 1e-13 and it > 1
        # the same with lambda* handed in explicitly
        ls = s.get_lambda_star()
        gb2, gp2, gm2, _, _ = s.adjoint(g_v, lambda_star=ls)
    assert np.array_equal(gb, gb2) and np.array_equal(gp, gp2) and np.array_equal(gm, gm2)
    assert relmax(gb, g_b) <= 1e-9
    assert relmax(gp, g_phi) <= 1e-9
    assert relmax(gm, g_mu) <= 1e-9 or np.abs(g_mu).max() == 0
    assert set(modes.tolist()) >= {1, 2} or set(modes.tolist()) >= {0, 2}


def test_adjoint_f32_terrain_patch():
    sc = scenes.terrain_lattice(dims=(12, 10, 4))
    rng = np.random.default_rng(3)
    g_v = rng.normal(0, 1, sc.n)
    ref, g_b, g_phi, g_mu, P = reference(sc.as_f64(), g_v)
    modes = mode_of(ref.lam, P.mu)
    assert (modes == 2).any() and (modes == 1).any()
    with vfpi.Solver.from_scene(sc, theta_th=1e-9, l_max=20000) as s:
        s.solve(sc.v0)
        gb, gp, gm, it, th = s.adjoint(g_v.astype(np.float32))
    # FP32 forward fixed point and adjoint against FP64: a few 1e-5 of the largest entry
    assert relmax(gb, g_b) <= 5e-5
    assert relmax(gp, g_phi) <= 5e-5
    assert relmax(gm, g_mu) <= 5e-4


def test_batched_adjoint_equals_per_scene():
    lat = scenes.batched_lattices(6, seed=77, side_range=(4, 6))
    batch = scenes.concat_scenes(lat)
    rng = np.random.default_rng(1)
    g_v = rng.normal(0, 1, batch.n).astype(np.float32)
    with vfpi.Solver.from_scene(batch, theta_th=1e-8, l_max=3000, block_threads=128) as s:
        s.solve(batch.v0)
        gb, gp, gm, its, ths = s.adjoint(g_v)
    o, oc = 0, 0
    for q, sc in enumerate(lat):
        with vfpi.Solver.from_scene(sc, theta_th=1e-8, l_max=3000, block_threads=128,
                                    force_path=2) as s1:
            s1.solve(sc.v0)
            gb1, gp1, gm1, it1, th1 = s1.adjoint(g_v[o:o + sc.n])
        assert it1 == its[q]
        assert np.array_equal(gb1, gb[o:o + sc.n])
        assert np.array_equal(gp1, gp[oc:oc + sc.n_c])
        o += sc.n
        oc += sc.n_c
