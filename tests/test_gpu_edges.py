"""GPU parity on the degenerate inputs of the method: no contacts (the fixed
point of eq. pgd1 is then the linear solve A v = b), a one-node scene, node
counts around the 32-row slice boundary, and a batch that mixes such scenes
with an ordinary lattice.  Each on both kernel paths, against the FP64 oracle
at fixed sweep counts (the ladder of test_gpu_parity, same tolerances) and,
where the answer has a closed form, against it."""
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
from tests.test_gpu_parity import F32_LADDER, F64_LADDER, close, ladder, rel  # noqa: E402

PATHS = ({"force_path": 1}, {"force_path": 2})


def no_contact_scene(dtype):
    return scenes.random_problem(np.random.default_rng(41), 40, 0, density=0.1, couple=0.5,
                                 dtype=dtype)


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
@pytest.mark.parametrize("path", PATHS)
def test_no_contacts_ladder_and_linear_solve(dtype, path):
    sc = no_contact_scene(dtype)
    assert sc.n_c == 0
    ladder(sc, ks=(1, 2, 10), **path)
    P = oracle_problem(sc)
    x = np.linalg.solve(P.A.toarray(), P.b)
    th = 1e-13 if dtype == np.float64 else 1e-6
    with vfpi.Solver.from_scene(sc, theta_th=th, l_max=20000, **path) as s:
        r = s.solve(sc.v0)
        assert r.status == vfpi.VFPI_OK
        assert s.get_lambda().size == 0
    # FP32: the converged iterate carries the rounding of one sweep's A v - b
    assert rel(r.v, x) <= (1e-11 if dtype == np.float64 else 5e-6), rel(r.v, x)


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
@pytest.mark.parametrize("path", PATHS)
def test_one_node_scene(dtype, path):
    """One node on a plane: one row in a 32-row slice whose other 31 rows are padding."""
    sc = scenes.random_problem(np.random.default_rng(101), 1, 1, density=0.1, couple=0.5,
                               dtype=dtype)
    assert sc.n_nodes == 1 and sc.n_c == 1
    ladder(sc, ks=(1, 2, 10, 30), **path)
    with vfpi.Solver.from_scene(sc, **path) as s:
        assert s.layout()["n_pad"] == 32 and s.layout()["n_slices"] == 1


@pytest.mark.parametrize("n", [31, 32, 33, 65])
@pytest.mark.parametrize("path", PATHS)
def test_node_counts_around_the_slice_boundary(n, path):
    """31/32/33/65 nodes: a full slice, a padded one, one row in a second or
    third slice; S- and D-contacts."""
    rng = np.random.default_rng(100 + n)
    sc = scenes.random_problem(rng, n, 5, d_contacts=3, density=0.1, couple=0.5)
    ladder(sc, ks=(1, 3, 15), **path)
    with vfpi.Solver.from_scene(sc, **path) as s:
        assert s.layout()["n_slices"] == -(-n // 32)


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_batch_with_degenerate_scenes(dtype):
    """One launch over a one-node scene, a scene without contacts, a 33-node
    scene with S- and D-contacts and a small lattice: each scene's iterate
    after k sweeps equals its own oracle iterate, and the converged solve of
    each scene its own solve."""
    parts = [
        scenes.random_problem(np.random.default_rng(101), 1, 1, density=0.1, couple=0.5),
        scenes.random_problem(np.random.default_rng(41), 40, 0, density=0.1, couple=0.5),
        scenes.random_problem(np.random.default_rng(133), 33, 5, d_contacts=3, density=0.1,
                              couple=0.5),
        scenes.small_lattice(np.float64),
    ]
    sc = scenes.concat_scenes(parts, dtype=dtype)
    tol = F64_LADDER if dtype == np.float64 else F32_LADDER
    offs = sc.scene_ptr
    c_off = np.concatenate([[0], np.cumsum([p.n_c for p in parts])])
    for k in (1, 4, 15):
        with vfpi.Solver.from_scene(sc, theta_th=0.0, l_max=k, force_path=2) as s:
            r = s.solve(sc.v0)
            assert np.all(np.asarray(r.iters) == k)
            lam = s.get_lambda().reshape(-1, 3)
        for q, p in enumerate(parts):
            P = oracle_problem(p)
            ref = ov.solve(P, ov.frobenius_w(P), np.asarray(p.v0, float), theta_th=0.0, l_max=k)
            vq = r.v[3 * offs[q]:3 * offs[q + 1]]
            assert close(vq, ref.v, tol), (k, q, rel(vq, ref.v))
            if p.n_c:
                assert close(lam[c_off[q]:c_off[q + 1]], ref.lam, 10 * tol), (k, q)
    # the batch at the stop test = each scene solved alone (bitwise: same rows,
    # same per-scene sums)
    th = 1e-12 if dtype == np.float64 else 1e-6
    with vfpi.Solver.from_scene(sc, theta_th=th, l_max=5000, force_path=2) as s:
        rb = s.solve(sc.v0)
    for q, p in enumerate(parts):
        with vfpi.Solver.from_scene(p, theta_th=th, l_max=5000, force_path=2,
                                    dtype="f64" if dtype == np.float64 else "f32") as s:
            rq = s.solve(np.asarray(p.v0, dtype))
        assert int(rb.iters[q]) == rq.iters
        assert np.array_equal(rb.v[3 * offs[q]:3 * offs[q + 1]], rq.v), q


def test_page_locked_input_may_change_once_the_call_returns():
    """A host input may be changed as soon as the call returns, also from
    page-locked memory (which the runtime reads only when the stream gets to
    the copy): with a long solve still on the stream, vfpi_set_velocity from a
    pinned array that is overwritten right after the call keeps the values it
    was given."""
    sc = scenes.terrain_lattice(dims=(64, 64, 16))
    v_new = torch.from_numpy(np.asarray(sc.v0) * 0.5 + 0.25).pin_memory()
    want = v_new.numpy().copy()
    with vfpi.Solver.from_scene(sc, theta_th=-1.0, l_max=200) as s:
        s.set_velocity(sc.v0)
        s.solve_async()                      # keeps the stream busy for a while
        s.set_velocity(v_new)
        v_new.fill_(float("nan"))            # the caller reuses its buffer
        got = s.get_velocity()
    assert np.array_equal(got, want)


def test_page_locked_input_under_stream_capture_is_read_at_each_replay():
    """Under stream capture the copy from page-locked memory is a graph node:
    a captured (set_velocity, solve) replays with whatever the pinned buffer
    holds at replay time, as the eager calls would."""
    sc = scenes.terrain_lattice(dims=(40, 36, 6))
    stream = torch.cuda.Stream()
    v_pin = torch.from_numpy(np.asarray(sc.v0).copy()).pin_memory()
    starts = [np.asarray(sc.v0) * f for f in (1.0, 0.5, -0.25)]
    with vfpi.Solver.from_scene(sc, theta_th=-1.0, l_max=9, force_path=1, stream=stream) as s:
        ref = []
        for v in starts:                               # eager
            s.set_velocity(v)
            s.solve_async()
            ref.append(s.get_velocity())
        g = torch.cuda.CUDAGraph()
        with torch.cuda.stream(stream):
            s.set_velocity(v_pin)                      # warm the path outside capture
            torch.cuda.synchronize()
            with torch.cuda.graph(g, stream=stream):
                s.set_velocity(v_pin)
                s.solve_async()
        for v, r in zip(starts, ref):
            v_pin.copy_(torch.from_numpy(v))
            g.replay()
            torch.cuda.synchronize()
            assert np.array_equal(s.get_velocity(), r)
