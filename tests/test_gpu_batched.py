"""Batched form: thousands of independent, uneven scenes in one persistent
launch (CTA-per-scene kernel), checked against per-scene solves and the
FP64 oracle; graph-captured time steps replay to the same numbers."""
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


def split(vec, sc_list, per):
    out, o = [], 0
    for s in sc_list:
        k = per(s)
        out.append(vec[o:o + k])
        o += k
    return out


@pytest.fixture(scope="module")
def lattices():
    return scenes.batched_lattices(96, seed=4321, side_range=(4, 9))


def test_batch_equals_per_scene_solves_bitwise(lattices):
    batch = scenes.concat_scenes(lattices)
    with vfpi.Solver.from_scene(batch, theta_th=1e-6, l_max=400, block_threads=128) as s:
        rb = s.solve(batch.v0)
    assert isinstance(rb.iters, np.ndarray) and len(rb.iters) == len(lattices)
    assert len(set(rb.iters.tolist())) > 1, "scenes should need different iteration counts"
    vs = split(rb.v, lattices, lambda q: q.n)
    ls = split(rb.lam, lattices, lambda q: 3 * q.n_c)
    for q in range(0, len(lattices), 7):
        sc = lattices[q]
        with vfpi.Solver.from_scene(sc, theta_th=1e-6, l_max=400, block_threads=128,
                                    force_path=2) as s1:
            r1 = s1.solve(sc.v0)
        assert r1.iters == rb.iters[q]
        assert r1.theta == rb.theta[q]
        assert np.array_equal(r1.v, vs[q])
        assert np.array_equal(r1.lam, ls[q])


def test_batch_against_oracle(lattices):
    batch = scenes.concat_scenes(lattices[:24])
    with vfpi.Solver.from_scene(batch, theta_th=0.0, l_max=25) as s:
        rb = s.solve(batch.v0)
    assert (rb.iters == 25).all()
    vs = split(rb.v, lattices[:24], lambda q: q.n)
    for q in range(0, 24, 5):
        sc = lattices[q]
        P = oracle_problem(sc)
        ref = ov.solve(P, ov.frobenius_w(P), sc.v0, theta_th=0.0, l_max=25)
        err = np.abs(vs[q] - ref.v).max() / np.abs(ref.v).max()
        assert err <= 1e-5, err


def test_batch_converged_scc_and_tolerance(lattices):
    sub = lattices[:12]
    batch = scenes.concat_scenes(sub)
    with vfpi.Solver.from_scene(batch, theta_th=1e-9, l_max=3000) as s:
        rb = s.solve(batch.v0)
    vs = split(rb.v, sub, lambda q: q.n)
    ls = split(rb.lam, sub, lambda q: 3 * q.n_c)
    for q, sc in enumerate(sub):
        P = oracle_problem(sc)
        ref = ov.solve(P, ov.frobenius_w(P), sc.v0, theta_th=1e-13, l_max=100000)
        assert np.linalg.norm(vs[q] - ref.v) <= 1e-5 * np.linalg.norm(ref.v)
        assert scc_residual(P, vs[q].astype(float), ls[q].astype(float).reshape(-1, 3)) <= 1e-6


def test_uneven_batch_with_d_contacts_f64():
    rng = np.random.default_rng(99)
    probs = [scenes.random_problem(rng, int(n), int(n) // 8, d_contacts=int(n) // 16,
                                   density=0.05, couple=0.4)
             for n in rng.integers(20, 140, size=10)]
    batch = scenes.concat_scenes(probs, dtype=np.float64)
    with vfpi.Solver.from_scene(batch, theta_th=0.0, l_max=15) as s:
        rb = s.solve(batch.v0)
    vs = split(rb.v, probs, lambda q: q.n)
    ls = split(rb.lam, probs, lambda q: 3 * q.n_c)
    for q, sc in enumerate(probs):
        P = oracle_problem(sc)
        ref = ov.solve(P, ov.frobenius_w(P), sc.v0, theta_th=0.0, l_max=15)
        assert np.allclose(vs[q], ref.v, rtol=1e-11, atol=1e-11 * np.abs(ref.v).max())
        assert np.allclose(ls[q].reshape(-1, 3), ref.lam, rtol=1e-10,
                           atol=1e-10 * max(np.abs(ref.lam).max(), 1e-300))


def test_cross_scene_block_is_rejected(lattices):
    a, b = lattices[0], lattices[1]
    batch = scenes.concat_scenes([a, b])
    # move one block of scene 0's last row onto a column of scene 1
    col = batch.col_idx.copy()
    last = batch.row_ptr[a.n_nodes] - 1
    col[last] = a.n_nodes  # first node of scene 1 (still sorted: larger than the row's others)
    with pytest.raises(vfpi.VfpiError) as e:
        vfpi.Solver(batch.row_ptr, col, batch.vals, batch.b, batch.node_i, batch.node_j,
                    batch.R, batch.mu, batch.phi, scene_ptr=batch.scene_ptr)
    assert e.value.status == -1 and "two scenes" in str(e.value)


def test_graph_captured_steps_replay_like_eager(lattices):
    sub = lattices[:32]
    batch = scenes.concat_scenes(sub)
    stream = torch.cuda.Stream()
    dev = torch.device("cuda")
    v0 = torch.from_numpy(batch.v0).to(dev)
    x_e = torch.from_numpy(batch.x0).to(dev)
    x_g = x_e.clone()
    with vfpi.Solver.from_scene(batch, theta_th=1e-6, l_max=300, stream=stream) as s:
        for _ in range(3):                       # eager reference
            s.set_velocity(v0)
            s.solve_async()
            s.integrate(x_e)
        it_e, th_e, _ = s.status()
        v_e = s.get_velocity()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.stream(stream):
            s.set_velocity(v0)                   # warm the path once outside capture
            torch.cuda.synchronize()
            with torch.cuda.graph(g, stream=stream):
                s.set_velocity(v0)
                s.solve_async()
                s.integrate(x_g)
        for _ in range(3):
            g.replay()
        torch.cuda.synchronize()
        it_g, th_g, _ = s.status()
        assert np.array_equal(it_g, it_e) and np.array_equal(th_g, th_e)
        assert np.array_equal(s.get_velocity(), v_e)
    assert torch.equal(x_g, x_e)
