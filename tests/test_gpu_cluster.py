"""Batched solve with the scene matrices resident in shared memory (cluster
kernel).  Each shape must reproduce the CTA-per-scene kernel bit for bit: the
rows do the same arithmetic in the same order, whether a scene runs on one CTA,
is split over the CTAs of a cluster, or is only partly cached.  Also checked
against the FP64 oracle, with D-contacts, the adjoint, Chebyshev steps,
Barzilai-Borwein steps (run on the CTA-per-scene kernel), single sweeps and a
graph-captured time step."""
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

# threads per CTA, CTAs per cluster, CTAs per SM of VFPI_VARIANT_CL_*
SHAPES = {16: (256, 1, 1), 17: (256, 2, 1), 18: (256, 4, 1), 19: (256, 8, 1), 20: (128, 4, 2),
          21: (128, 8, 2), 22: (256, 4, 2), 23: (256, 8, 2), 24: (512, 8, 1), 25: (128, 8, 4)}


def split(vec, sc_list, per):
    out, o = [], 0
    for s in sc_list:
        k = per(s)
        out.append(vec[o:o + k])
        o += k
    return out


@pytest.fixture(scope="module")
def uneven():
    # sides 4..12: 2 to 54 slices per scene, 0.07 to 1.9 MB of sliced-ELL
    # entries -- some scenes fit one CTA's shared memory, some need a cluster,
    # some exceed even a cluster's (partly cached)
    return scenes.batched_lattices(40, seed=2468, side_range=(4, 12))


def run(batch, variant, bt=0, theta=1e-6, l_max=300, setup=None, v0=None):
    with vfpi.Solver.from_scene(batch, theta_th=theta, l_max=l_max, kernel_variant=variant,
                                block_threads=bt) as s:
        if setup:
            setup(s)
        r = s.solve(batch.v0 if v0 is None else v0)
        lay = s.layout()
    return r, lay


def test_every_cluster_shape_matches_the_scene_kernel_bitwise(uneven):
    batch = scenes.concat_scenes(uneven)
    ref, _ = run(batch, 0, 256)
    assert len(set(ref.iters.tolist())) > 1
    for var, (nt, C, per_sm) in SHAPES.items():
        r, lay = run(batch, var)
        assert lay["threads"] == nt and lay["grid"] % C == 0, (var, lay)
        assert lay["grid"] <= lay["max_grid"]
        assert np.array_equal(r.iters, ref.iters), var
        assert np.array_equal(r.v, ref.v), var
        assert np.array_equal(r.lam, ref.lam), var


def test_cluster_kernel_against_oracle(uneven):
    sub = [uneven[q] for q in (0, 5, 11, 17)]
    batch = scenes.concat_scenes(sub)
    r, _ = run(batch, 19, theta=0.0, l_max=25)
    assert (r.iters == 25).all()
    for sc, v in zip(sub, split(r.v, sub, lambda q: q.n)):
        P = oracle_problem(sc)
        ref = ov.solve(P, ov.frobenius_w(P), sc.v0, theta_th=0.0, l_max=25)
        assert np.abs(v - ref.v).max() <= 1e-5 * np.abs(ref.v).max()


def test_d_contacts_split_over_a_cluster():
    # random problems with D-contacts, large enough (up to ~500 entries) that
    # the bigger ones are split over the cluster's CTAs
    rng = np.random.default_rng(11)
    parts = [scenes.random_problem(rng, n, max(2, n // 20), density=d, d_contacts=max(1, n // 25),
                                   dtype=np.float32)
             for n, d in ((40, 0.3), (300, 0.05), (900, 0.02), (1500, 0.012), (120, 0.1), (700, 0.03))]
    batch = scenes.concat_scenes(parts)
    ref, _ = run(batch, 0, 256, theta=1e-7, l_max=2000)
    for var in (16, 19, 21, 23, 25):
        r, _ = run(batch, var, theta=1e-7, l_max=2000)
        assert np.array_equal(r.iters, ref.iters), var
        assert np.array_equal(r.v, ref.v), var
        assert np.array_equal(r.lam, ref.lam), var


def test_adjoint_on_the_cluster_kernel(uneven):
    sub = uneven[:16]
    batch = scenes.concat_scenes(sub)
    g_v = np.random.default_rng(5).normal(0, 1, batch.n).astype(np.float32)
    out = {}
    for var, bt in ((0, 256), (19, 0), (23, 0)):
        with vfpi.Solver.from_scene(batch, theta_th=1e-7, l_max=3000, kernel_variant=var,
                                    block_threads=bt) as s:
            s.solve(batch.v0)
            out[var] = s.adjoint(g_v)
    gb, gp, gm, it, _ = out[0]
    for var in (19, 23):
        gb1, gp1, gm1, it1, _ = out[var]
        assert np.array_equal(it1, it), var
        assert np.array_equal(gb1, gb) and np.array_equal(gp1, gp) and np.array_equal(gm1, gm), var


def test_chebyshev_on_the_cluster_kernel(uneven):
    # the Chebyshev weights depend on the residual history, whose FP64 sum is
    # ordered differently when a scene is split over a cluster: equal to
    # rounding, not bit for bit
    sub = uneven[:20]
    batch = scenes.concat_scenes(sub)
    ref, _ = run(batch, 0, 256, theta=1e-7, l_max=2000, setup=lambda s: s.set_chebyshev(10, 0.9))
    plain, _ = run(batch, 0, 256, theta=1e-7, l_max=2000)
    assert ref.iters.sum() < plain.iters.sum()
    r, _ = run(batch, 19, theta=1e-7, l_max=2000, setup=lambda s: s.set_chebyshev(10, 0.9))
    assert np.abs(r.iters - ref.iters).max() <= 2
    scale = np.abs(ref.v).max()
    assert np.abs(r.v - ref.v).max() <= 1e-5 * scale


def test_barzilai_borwein_falls_back_to_the_scene_kernel(uneven):
    sub = uneven[:10]
    batch = scenes.concat_scenes(sub)
    bb = lambda s: s.set_barzilai_borwein("alt", float(np.median(s.get_w())))  # noqa: E731
    ref, _ = run(batch, 0, 256, theta=1e-7, l_max=3000, setup=bb)
    r, _ = run(batch, 19, theta=1e-7, l_max=3000, setup=bb)
    assert np.array_equal(r.iters, ref.iters) and np.array_equal(r.v, ref.v)


def test_single_sweeps_and_graph_replay(uneven):
    sub = uneven[:24]
    batch = scenes.concat_scenes(sub)
    stream = torch.cuda.Stream()
    v0 = torch.from_numpy(batch.v0).cuda()
    with vfpi.Solver.from_scene(batch, theta_th=1e-6, l_max=300, kernel_variant=19,
                                stream=stream) as s, \
         vfpi.Solver.from_scene(batch, theta_th=1e-6, l_max=300, block_threads=256,
                                stream=stream) as s0:
        for solver in (s, s0):
            solver.set_velocity(v0)
            for _ in range(3):
                solver.step()
        assert np.array_equal(s.get_velocity(), s0.get_velocity())
        s0.set_velocity(v0)
        s0.solve_async()
        it0, _, _ = s0.status()
        v_ref = s0.get_velocity()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.stream(stream):
            s.set_velocity(v0)
            torch.cuda.synchronize()
            with torch.cuda.graph(g, stream=stream):
                s.set_velocity(v0)
                s.solve_async()
        for _ in range(2):
            g.replay()
        torch.cuda.synchronize()
        it, _, _ = s.status()
        assert np.array_equal(it, it0)
        assert np.array_equal(s.get_velocity(), v_ref)


def test_cluster_shapes_need_the_scene_path():
    sc = scenes.terrain_lattice(dims=(32, 32, 8))
    with pytest.raises(vfpi.VfpiError) as e:
        vfpi.Solver.from_scene(sc, kernel_variant=19, force_path=1)
    assert e.value.status == -1
    with vfpi.Solver.from_scene(sc, force_path=1) as s:
        with pytest.raises(vfpi.VfpiError):
            s.configure_launch(19, 0, 0)
        r = s.solve(sc.v0)            # the previous shape still works
        assert np.isfinite(r.theta)


def test_batched_tuner_times_whole_solves_and_restores_the_warm_start(uneven, tmp_path):
    from paper_2201_09212_gb300 import tune
    batch = scenes.concat_scenes(uneven[:16])
    ref, _ = run(batch, 0, 256)
    with vfpi.Solver.from_scene(batch, theta_th=1e-6, l_max=300) as s:
        s.set_velocity(batch.v0)
        res = tune.tune(s, sweeps=5, reps=1, cache=str(tmp_path / "t.json"))
        assert not res["cached"]
        shapes = {(t["kernel_variant"], t["block_threads"]) for t in res["trials"]}
        assert {(0, 64), (0, 128), (0, 256), (0, 512)} <= shapes and (19, 0) in shapes
        assert all("ms_per_solve" in t for t in res["trials"])
        assert np.array_equal(s.get_velocity(), batch.v0)      # warm start put back
        r = s.solve(batch.v0)
    assert np.array_equal(r.iters, ref.iters) and np.array_equal(r.v, ref.v)


def test_cluster_shapes_f64():
    """The FP64 instantiations (two 16-byte st.async pushes per row on the
    shared-memory exchange path) give the CTA-per-scene kernel's iterates."""
    lat = scenes.batched_lattices(12, seed=1357, side_range=(4, 11), dtype=np.float64)
    batch = scenes.concat_scenes(lat)
    ref, _ = run(batch, 0, 256, theta=1e-10, l_max=2000)
    for var in (16, 19, 23, 25):
        r, _ = run(batch, var, theta=1e-10, l_max=2000)
        assert np.array_equal(r.iters, ref.iters), var
        assert np.array_equal(r.v, ref.v) and np.array_equal(r.lam, ref.lam), var
