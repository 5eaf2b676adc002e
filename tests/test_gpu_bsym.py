"""Symmetric-block storage (launch variants 28, 29 and 30): when every 3x3
block of A equals its transpose bit for bit, the forward kernels stream each
block as its 6 distinct values and rebuild the same 9 entries, so the
iterates must be bitwise those of the full storage (FP32 and FP64).  Also:
a matrix with an asymmetric block refuses the variants, and an update that
makes a block asymmetric falls back to the full storage (and back again)."""
import numpy as np
import pytest

from paper_2201_09212_gb300 import scenes

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2201_09212_gb300 import vfpi  # noqa: E402


def solve(sc, variant, block_threads=0, storage=None, **kw):
    with vfpi.Solver.from_scene(sc, **kw) as s:
        s.configure_launch(variant, block_threads, 0)
        if storage is not None:
            assert s.storage()["storage"] == storage
        r = s.solve(sc.v0)
        return r, s.get_lambda()


@pytest.mark.parametrize("bt", [64, 128, 256, 512])
def test_batched_scenes_on_symmetric_blocks_equal_the_full_storage(bt):
    sc = scenes.concat_scenes(scenes.batched_lattices(48, seed=17))
    for kw in (dict(theta_th=-1.0, l_max=11), dict(theta_th=1e-6, l_max=300, norm="rms")):
        ref, lref = solve(sc, 0, bt, storage="full", force_path=2, **kw)
        got, lgot = solve(sc, 30, bt, storage="blocks6", force_path=2, **kw)
        assert np.array_equal(np.asarray(got.iters), np.asarray(ref.iters))
        assert np.array_equal(got.v, ref.v) and np.array_equal(lgot, lref)


def test_full_size_terrain_on_symmetric_blocks_equals_the_full_storage():
    sc = scenes.terrain_lattice()
    kw = dict(theta_th=1e-6, l_max=200, norm="rms", force_path=1)
    ref, lref = solve(sc, 7, storage="full", **kw)
    for var in (28, 29):
        got, lgot = solve(sc, var, storage="blocks6", **kw)
        assert got.iters == ref.iters and np.array_equal(got.v, ref.v)
        assert np.array_equal(lgot, lref)


def test_asymmetric_blocks_refuse_the_variants_and_updates_fall_back():
    fem = scenes.fem_block_scene(8, 8, 4, seed=1, dtype=np.float32)
    with vfpi.Solver.from_scene(fem, force_path=1) as s:
        for var in (28, 29):
            with pytest.raises(vfpi.VfpiError) as x:
                s.configure_launch(var, 0, 0)
            assert x.value.status == vfpi.STATUS_CODES["VFPI_ERR_INVALID_ARG"]
    # a lattice whose update makes one block asymmetric, then symmetric again
    sc = scenes.terrain_lattice(dims=(40, 36, 6))
    bad = sc.vals.copy()
    k = int(np.nonzero(np.abs(bad[:, 0, 1]) > 0)[0][5])
    bad[k, 0, 1] *= np.float32(1.0 + 2.0 ** -10)
    kw = dict(theta_th=-1.0, l_max=9, force_path=1)
    for var in (28, 29):
        with vfpi.Solver.from_scene(sc, **kw) as s:
            s.configure_launch(var, 0, 0)
            for vals in (bad, sc.vals):
                s.update(vals=vals)
                assert s.storage()["storage"] == ("full" if vals is bad else "blocks6")
                r = s.solve(sc.v0)
                with vfpi.Solver(sc.row_ptr, sc.col_idx, vals, sc.b, sc.node_i, sc.node_j, sc.R,
                                 sc.mu, sc.phi, h=sc.h, **kw) as full:
                    ref = full.solve(sc.v0)
                assert np.array_equal(r.v, ref.v)


@pytest.mark.parametrize("path,var_full,var_b6", [(2, 0, 30), (1, 7, 29)])
def test_adjoint_on_symmetric_blocks_equals_the_full_storage(path, var_full, var_b6):
    """The adjoint sweep is the forward product with b := g_v (A is
    symmetric): on the 6-value blocks it gives dL/db, dL/dphi and dL/dmu bit
    for bit as on the full storage."""
    sc = (scenes.concat_scenes(scenes.batched_lattices(24, seed=23)) if path == 2
          else scenes.terrain_lattice(dims=(40, 36, 6)))
    g_v = np.random.default_rng(5).standard_normal(sc.n).astype(np.float32)
    out = []
    for var in (var_full, var_b6):
        with vfpi.Solver.from_scene(sc, theta_th=1e-6, l_max=300, norm="rms",
                                    force_path=path) as s:
            s.configure_launch(var, 256 if path == 2 else 0, 0)
            s.solve(sc.v0)
            out.append(s.adjoint(g_v))
    for a, b in zip(out[0][:3], out[1][:3]):
        assert np.array_equal(a, b)
    assert np.array_equal(np.asarray(out[0][3]), np.asarray(out[1][3]))


def test_fp64_symmetric_blocks_equal_the_full_storage():
    sc = scenes.concat_scenes(scenes.batched_lattices(16, seed=29, dtype=np.float64))
    kw = dict(theta_th=1e-9, l_max=300, norm="rms", force_path=2)
    with vfpi.Solver.from_scene(sc, **kw) as s:
        assert s.storage()["blocks_symmetric"]
    ref, lref = solve(sc, 0, 128, storage="full", **kw)
    got, lgot = solve(sc, 30, 128, storage="blocks6", **kw)
    assert np.array_equal(np.asarray(got.iters), np.asarray(ref.iters))
    assert np.array_equal(got.v, ref.v) and np.array_equal(lgot, lref)


def test_storage_query_follows_the_launch_shape():
    sc = scenes.terrain_lattice(dims=(40, 36, 6))
    with vfpi.Solver.from_scene(sc, theta_th=-1.0, l_max=4, force_path=1) as s:
        seen = {}
        for var in (0, 12, 26, 28):
            s.configure_launch(var, 0, 0)
            seen[var] = s.storage()["storage"]
        assert seen == {0: "full", 12: "symmetric", 26: "full", 28: "blocks6"}
