"""vfpi_advance, one time step in one call (eq. disc_dyn: right-hand side,
warm start, Alg. 1, v_hat and lambda out, x += h v_hat), against the separate
calls it stands for: bitwise the same v_hat, lambda, x, iteration count and
theta, with host (page-locked and pageable) and device arrays, on both kernel
paths; NULL arguments leave the corresponding input or output alone; host
arrays may be reused as soon as the call returns; and a stream capture is
refused (the call waits for its step)."""
import numpy as np
import pytest

from paper_2201_09212_gb300 import scenes

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2201_09212_gb300 import vfpi  # noqa: E402


def next_rhs(sc, k):
    """A second step's inputs: b and phi changed, a different warm start."""
    rng = np.random.default_rng(100 + k)
    b = (np.asarray(sc.b) * (1.0 + 0.01 * k)).astype(sc.b.dtype)
    phi = (np.asarray(sc.phi) + 1e-4 * rng.standard_normal(sc.n_c)).astype(sc.phi.dtype)
    v = (np.asarray(sc.v0) * (1.0 - 0.1 * k)).astype(sc.v0.dtype)
    return b, phi, v


def separate_calls(s, b, phi, v, x):
    s.set_rhs(b, phi)
    r = s.solve(v)
    s.integrate(x)
    return r, x


def same(r, q):
    assert np.array_equal(np.asarray(r.v), np.asarray(q.v))
    assert np.array_equal(np.asarray(r.lam), np.asarray(q.lam))
    assert np.array_equal(np.asarray(r.iters), np.asarray(q.iters))
    assert np.array_equal(np.asarray(r.theta), np.asarray(q.theta))


@pytest.mark.parametrize("memory", ["pageable", "pinned", "device"])
@pytest.mark.parametrize("path", [1, 2])
def test_advance_equals_the_separate_calls(memory, path):
    sc = (scenes.terrain_lattice(dims=(40, 36, 6)) if path == 1
          else scenes.concat_scenes(scenes.batched_lattices(24, seed=31)))
    kw = dict(theta_th=1e-6, l_max=300, norm="rms", force_path=path)

    def put(a):
        if memory == "pageable":
            return np.array(a, copy=True)
        t = torch.from_numpy(np.ascontiguousarray(a).copy())
        return t.pin_memory() if memory == "pinned" else t.cuda()

    def get(a):
        return a.cpu().numpy() if torch.is_tensor(a) else np.asarray(a)

    for k in range(2):
        b, phi, v = next_rhs(sc, k)
        x0 = np.asarray(sc.x0, dtype=np.float64)
        with vfpi.Solver.from_scene(sc, **kw) as s:
            ref, x_ref = separate_calls(s, b, phi, v, x0.copy())
        with vfpi.Solver.from_scene(sc, **kw) as s:
            xa = put(x0)
            vo, lo = put(np.zeros(sc.n, sc.v0.dtype)), put(np.zeros(3 * sc.n_c, sc.v0.dtype))
            r = s.advance(put(b), put(phi), put(v), out_v=vo, out_lam=lo, x=xa)
            r.v, r.lam = get(r.v), get(r.lam)
            same(r, ref)
            assert np.array_equal(get(xa), x_ref)


def test_null_arguments_leave_inputs_and_outputs_alone():
    sc = scenes.terrain_lattice(dims=(40, 36, 6))
    kw = dict(theta_th=1e-6, l_max=300, norm="rms", force_path=1)
    b, phi, v = next_rhs(sc, 1)
    with vfpi.Solver.from_scene(sc, **kw) as s:
        s.set_rhs(b, phi)
        s.set_velocity(v)
        ref = s.solve()
    with vfpi.Solver.from_scene(sc, **kw) as s:
        s.set_rhs(b, phi)
        s.set_velocity(v)
        r = s.advance()                       # all NULL: the current b, phi and iterate
        same(r, ref)
        x = np.asarray(sc.x0, dtype=np.float64).copy()
        r2 = s.advance(v=v, x=x)              # b, phi kept; no lambda wanted
        assert np.array_equal(r2.v, ref.v)
        assert np.array_equal(x, np.asarray(sc.x0) + sc.h * ref.v.astype(np.float64))


def test_page_locked_inputs_may_change_once_the_call_returns():
    sc = scenes.terrain_lattice(dims=(64, 64, 16))
    kw = dict(theta_th=1e-6, l_max=300, norm="rms", force_path=1)
    b, phi, v = next_rhs(sc, 1)
    with vfpi.Solver.from_scene(sc, **kw) as s:
        ref, x_ref = separate_calls(s, b, phi, v, np.asarray(sc.x0, dtype=np.float64).copy())
    pin = [torch.from_numpy(np.ascontiguousarray(a).copy()).pin_memory() for a in (b, phi, v)]
    with vfpi.Solver.from_scene(sc, **kw) as s:
        s.set_velocity(sc.v0)
        s.solve_async()                       # keeps the stream busy for a while
        x = torch.from_numpy(np.asarray(sc.x0, dtype=np.float64).copy()).pin_memory()
        r = s.advance(*pin, x=x)
        for t in pin:
            t.fill_(float("nan"))             # the caller reuses its buffers
        same(r, ref)
        assert np.array_equal(x.numpy(), x_ref)
        assert np.array_equal(s.get_velocity(), ref.v)


def test_advance_inside_a_stream_capture_is_refused():
    sc = scenes.terrain_lattice(dims=(40, 36, 6))
    stream = torch.cuda.Stream()
    with vfpi.Solver.from_scene(sc, theta_th=-1.0, l_max=4, force_path=1, stream=stream) as s:
        s.set_velocity(sc.v0)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.stream(stream):
            with pytest.raises(vfpi.VfpiError) as x:
                with torch.cuda.graph(g, stream=stream):
                    s.solve_async()
                    s.advance(v=sc.v0)
        assert x.value.status == vfpi.STATUS_CODES["VFPI_ERR_INVALID_ARG"]
        torch.cuda.synchronize()
        # the context still works after the refusal
        r = s.advance(v=sc.v0)
        assert r.iters == 4
