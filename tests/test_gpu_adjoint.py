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


@pytest.mark.parametrize("seed", range(2))
def test_adjoint_chebyshev_keeps_the_fixed_point(seed):
    """Alg. 3 on the adjoint iteration (linear at the frozen active set): the
    same gradients as the dense FP64 reference (these small problems converge
    in a few dozen sweeps, too few for the slow start to pay off; the lattice
    test below checks the saving)."""
    rng = np.random.default_rng(950 + seed)
    sc = scenes.random_problem(rng, 60, 10, d_contacts=5, density=0.08, couple=0.3,
                               mu_range=(0.2, 0.8), phi_scale=1.0)
    g_v = rng.normal(0, 1, sc.n)
    ref, g_b, g_phi, g_mu, P = reference(sc, g_v)
    with vfpi.Solver.from_scene(sc, theta_th=1e-13, l_max=100000) as s:
        s.solve(sc.v0)
        gb0, gp0, gm0, it0, _ = s.adjoint(g_v)
        s.set_adjoint_chebyshev(10, 0.9)
        gb, gp, gm, it, th = s.adjoint(g_v)
        s.set_adjoint_chebyshev(0)
        gb2, _, _, it2, _ = s.adjoint(g_v)
    assert th < 1e-13 and it <= it0 + 5
    assert it2 == it0 and np.array_equal(gb2, gb0)
    assert relmax(gb, g_b) <= 1e-9
    assert relmax(gp, g_phi) <= 1e-9
    assert relmax(gm, g_mu) <= 1e-9 or np.abs(g_mu).max() == 0


def test_adjoint_chebyshev_batched_f32():
    lat = scenes.batched_lattices(12, seed=78, side_range=(4, 8))
    batch = scenes.concat_scenes(lat)
    # (scaled so that an rms change of 1e-7 stays well above FP32 rounding of
    # the adjoint iterate, which is about W g_v ~ 40 g_v here)
    g_v = (1e-3 * np.random.default_rng(2).normal(0, 1, batch.n)).astype(np.float32)
    with vfpi.Solver.from_scene(batch, theta_th=1e-7, l_max=5000, norm="rms") as s:
        s.solve(batch.v0)
        gb0, gp0, gm0, it0, _ = s.adjoint(g_v)
        s.set_adjoint_chebyshev(10, 0.9)
        gb, gp, gm, it, _ = s.adjoint(g_v)
    assert (it0 < 5000).all() and (it < 5000).all()
    assert it.sum() < it0.sum()
    assert relmax(gb, gb0) <= 1e-3
    assert relmax(gp, gp0) <= 1e-3


@pytest.mark.parametrize("path,variant", [(2, 0), (1, 7), (2, 19)],
                         ids=["scene_kernel", "grid_kernel", "cluster_kernel"])
def test_relative_adjoint_tolerance_scales_exactly(path, variant):
    """With the stop test relative to ||g_v|| the adjoint iteration is
    invariant under scaling g_v: a power-of-two factor scales every iterate,
    hence the result, bit for bit, after the same number of sweeps."""
    if path == 1:
        sc = scenes.terrain_lattice(dims=(40, 36, 8))
    else:
        sc = scenes.concat_scenes(scenes.batched_lattices(10, seed=5, side_range=(4, 10)))
    g_v = np.random.default_rng(8).normal(0, 1, sc.n).astype(np.float32)
    k = np.float32(2.0 ** -20)
    with vfpi.Solver.from_scene(sc, theta_th=1e-7, l_max=5000, norm="rms", force_path=path,
                                kernel_variant=variant) as s:
        s.solve(sc.v0)
        # (1e-4: the FP32 rounding of the iterate, ~40-200 g_v, sits near 1e-5 ||g_v||)
        s.set_adjoint_tolerance(1e-4, 5000, relative=True)
        gb, gp, gm, it, th = s.adjoint(g_v)
        gb2, gp2, gm2, it2, th2 = s.adjoint(g_v * k)
        s.set_adjoint_tolerance(1e-4, 5000, relative=False)
        _, _, _, it_abs, _ = s.adjoint(g_v * k)
    assert np.all(np.asarray(it) < 5000)
    assert np.array_equal(it, it2)
    assert np.array_equal(gb2, gb * k) and np.array_equal(gp2, gp * k) and np.array_equal(gm2, gm * k)
    assert np.all(np.asarray(it_abs) <= 2)   # the absolute test stops at once on the tiny load


def test_relative_adjoint_tolerance_f64_against_dense_reference():
    rng = np.random.default_rng(977)
    sc = scenes.random_problem(rng, 60, 10, d_contacts=5, density=0.08, couple=0.3,
                               mu_range=(0.2, 0.8), phi_scale=1.0)
    g_v = 1e-7 * rng.normal(0, 1, sc.n)
    ref, g_b, g_phi, g_mu, P = reference(sc, g_v)
    with vfpi.Solver.from_scene(sc, theta_th=1e-13, l_max=100000) as s:
        s.solve(sc.v0)
        s.set_adjoint_tolerance(1e-13, 100000, relative=True)
        gb, gp, gm, it, th = s.adjoint(g_v)
    assert relmax(gb, g_b) <= 1e-9
    assert relmax(gp, g_phi) <= 1e-9
    assert relmax(gm, g_mu) <= 1e-9 or np.abs(g_mu).max() == 0


def test_relative_adjoint_tolerance_is_per_scene():
    """Each scene of a batch stops on its own load's norm: with loads of very
    different sizes the batched adjoint equals each scene's own solve bit for
    bit (one shared threshold would change the iteration counts)."""
    lat = scenes.batched_lattices(6, seed=31, side_range=(4, 8))
    batch = scenes.concat_scenes(lat)
    rng = np.random.default_rng(12)
    parts = [(rng.normal(0, 1, sc.n) * 2.0 ** (-6 * q)).astype(np.float32) for q, sc in enumerate(lat)]
    g_v = np.concatenate(parts)
    with vfpi.Solver.from_scene(batch, theta_th=1e-7, l_max=5000, norm="rms", block_threads=128) as s:
        s.solve(batch.v0)
        s.set_adjoint_tolerance(1e-4, 5000, relative=True)
        gb, gp, gm, its, _ = s.adjoint(g_v)
    assert (its < 5000).all() and len(set(its.tolist())) > 1
    o = 0
    for q, sc in enumerate(lat):
        with vfpi.Solver.from_scene(sc, theta_th=1e-7, l_max=5000, norm="rms", block_threads=128,
                                    force_path=2) as s1:
            s1.solve(sc.v0)
            s1.set_adjoint_tolerance(1e-4, 5000, relative=True)
            gb1, _, _, it1, _ = s1.adjoint(parts[q])
        assert it1 == its[q], q
        assert np.array_equal(gb1, gb[o:o + sc.n]), q
        o += sc.n
