"""Symmetric storage of A on the grid path (launch shapes 12-15): only the
blocks c >= r are stored and each row reads its blocks c < r back transposed.
The row sums keep their order and operations, so every result must be bitwise
that of the full storage -- solve, single sweeps, Chebyshev, the adjoint --
and a matrix that is not exactly symmetric must never take that path."""
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

SYM = (12, 13, 14, 15)


def solve(sc, variant, dtype="f32", theta=1e-6, l_max=400, setup=None, grid=0):
    with vfpi.Solver.from_scene(sc, theta_th=theta, l_max=l_max, force_path=1, dtype=dtype,
                                kernel_variant=variant, grid_ctas=grid) as s:
        if setup:
            setup(s)
        r = s.solve(sc.v0)
    return r


@pytest.mark.parametrize("make", [lambda: scenes.terrain_lattice(dims=(64, 48, 12)),
                                  lambda: scenes.fem_block(cells=(24, 20, 8))],
                         ids=["terrain_lattice", "fem_block"])
def test_symmetric_storage_is_bitwise_the_full_one(make):
    sc = make()
    ref = solve(sc, 7)
    for var in SYM:
        for grid in (0, 31):
            r = solve(sc, var, grid=grid)
            assert r.iters == ref.iters, (var, grid)
            assert np.array_equal(r.v, ref.v), (var, grid)
            assert np.array_equal(r.lam, ref.lam), (var, grid)


def test_symmetric_storage_f64_against_oracle():
    sc = scenes.terrain_lattice(np.float64, dims=(20, 18, 5))
    r = solve(sc, 12, dtype="f64", theta=0.0, l_max=30)
    full = solve(sc, 7, dtype="f64", theta=0.0, l_max=30)
    assert np.array_equal(r.v, full.v)
    P = oracle_problem(sc)
    ref = ov.solve(P, ov.frobenius_w(P), sc.v0, theta_th=0.0, l_max=30)
    assert np.abs(r.v - ref.v).max() <= 1e-11 * np.abs(ref.v).max()


def test_symmetric_storage_chebyshev_adjoint_and_single_sweeps():
    sc = scenes.terrain_lattice(dims=(48, 40, 10))
    cheb = lambda s: s.set_chebyshev(10, 0.9)  # noqa: E731
    a = solve(sc, 12, setup=cheb, theta=1e-7)
    b = solve(sc, 7, setup=cheb, theta=1e-7)
    assert a.iters == b.iters and np.array_equal(a.v, b.v)
    g_v = np.random.default_rng(3).normal(0, 1, sc.n).astype(np.float32)
    out = {}
    for var in (7, 12):
        with vfpi.Solver.from_scene(sc, theta_th=1e-7, l_max=2000, force_path=1,
                                    kernel_variant=var) as s:
            s.solve(sc.v0)
            adj = s.adjoint(g_v)
            s.set_velocity(sc.v0)
            th = [s.step() for _ in range(3)]
            out[var] = (adj, th, s.get_velocity())
    (gb, gp, gm, it, _), th7, v7 = out[7]
    (gb2, gp2, gm2, it2, _), th12, v12 = out[12]
    assert it == it2 and np.array_equal(gb, gb2) and np.array_equal(gp, gp2) and np.array_equal(gm, gm2)
    assert np.array_equal(v7, v12)
    assert np.allclose(th7, th12, rtol=1e-12)


def test_barzilai_borwein_runs_on_the_full_storage():
    sc = scenes.terrain_lattice(dims=(40, 36, 8))

    def bb(s):
        s.set_barzilai_borwein("alt", float(np.median(s.get_w())))
    a = solve(sc, 12, setup=bb, theta=1e-7, l_max=3000)
    b = solve(sc, 7, setup=bb, theta=1e-7, l_max=3000)
    assert a.iters == b.iters and np.array_equal(a.v, b.v)


def test_unsymmetric_matrix_never_uses_the_symmetric_storage():
    sc = scenes.terrain_lattice(dims=(40, 36, 8))
    vals = sc.vals.copy()
    i = 100
    e = next(e for e in range(sc.row_ptr[i], sc.row_ptr[i + 1]) if sc.col_idx[e] != i)
    vals[e, 0, 1] *= np.float32(1.0 + 2.0 ** -20)       # one entry off by a few ulps
    bad = scenes.dataclasses.replace(sc, vals=vals)
    with pytest.raises(vfpi.VfpiError) as err:
        vfpi.Solver.from_scene(bad, force_path=1, kernel_variant=12)
    assert err.value.status == -1
    with vfpi.Solver.from_scene(bad, force_path=1) as s:
        with pytest.raises(vfpi.VfpiError):
            s.configure_launch(12, 0, 0)
    # a symmetric context updated to the unsymmetric values keeps its shape
    # but reads the full storage; updated back, it is symmetric again
    ref_bad = solve(bad, 7)
    ref_sym = solve(sc, 7)
    with vfpi.Solver.from_scene(sc, theta_th=1e-6, l_max=400, force_path=1, kernel_variant=12) as s:
        s.update(vals=bad.vals)
        r = s.solve(sc.v0)
        assert r.iters == ref_bad.iters and np.array_equal(r.v, ref_bad.v)
        s.update(vals=sc.vals)
        r = s.solve(sc.v0)
        assert r.iters == ref_sym.iters and np.array_equal(r.v, ref_sym.v)
        y = s.matvec(sc.v0)
    with vfpi.Solver.from_scene(sc, force_path=1) as s0:
        assert np.array_equal(y, s0.matvec(sc.v0))
