"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on
identical seeded inputs.

Tolerances.  FP64 runs must agree to 1e-11 relative.  FP32 runs: a sweep
reads ~27 blocks per row, so one sweep carries a relative rounding error of a
few 1e-7 in ``A v - b``; the iteration is a contraction, so after k sweeps the
iterate differs from the FP64 one by at most a few 1e-6 of its norm.  The
ladder bound is therefore 1e-5 (norm-wise, and element-wise against the
largest entry).  The converged bar is the one the task fixes: relative
velocity error <= 1e-5 and scaled complementarity residual <= 1e-6.
"""
import numpy as np
import pytest

from oracle import vfpi as ov
from oracle.checks import dynamics_residual, mode_of, scc_residual
from paper_2201_09212_gb300 import scenes
from tests.conftest import oracle_problem

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2201_09212_gb300 import vfpi  # noqa: E402

F32_LADDER = 1e-5
F64_LADDER = 1e-11


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, float) - b) / max(np.linalg.norm(b), 1e-300))


def close(a, b, rtol):
    a = np.asarray(a, float)
    scale = max(np.abs(b).max(), 1e-300)
    return float(np.abs(a - b).max() / scale) <= rtol and rel(a, b) <= rtol


def ladder(sc, ks=(1, 2, 10), **kw):
    """Compare GPU and oracle iterates after each k in ks sweeps."""
    P = oracle_problem(sc)
    w = ov.frobenius_w(P)
    tol = F64_LADDER if sc.vals.dtype == np.float64 else F32_LADDER
    with vfpi.Solver.from_scene(sc, **kw) as s:
        wg = s.get_w()
        assert close(wg, w, 1e-12 if sc.vals.dtype == np.float64 else 1e-6)
        s.set_velocity(sc.v0)
        v = np.asarray(sc.v0, float)
        done = 0
        for k in ks:
            for _ in range(k - done):
                th_g = s.step()
                r = ov.sweep(P, w, v)
                v = r.v_next
            done = k
            vg = s.get_velocity()
            lg = s.get_lambda().reshape(-1, 3)
            assert close(vg, v, tol), (k, rel(vg, v))
            if P.n_c:
                assert close(lg, r.lam, 10 * tol), (k, rel(lg, r.lam))
            # theta is a difference of iterates: its error scales with ||v||
            assert abs(th_g - r.theta) <= 10 * tol * (r.theta + np.linalg.norm(v)), (th_g, r.theta)
    return P


# ----------------------------------------------------------------------------
# closed forms through the GPU
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_point_masses_one_sweep_matches_textbook(dtype):
    from tests.test_oracle_pins import single_node_cases, textbook_point_contact
    rng = np.random.default_rng(7)
    cases = single_node_cases(rng)
    N = len(cases) + 5
    masses = rng.uniform(0.5, 2.0, N)
    b = rng.normal(0, 1, 3 * N)
    Rs, mus, phis, nodes = [], [], [], []
    for q, (m_, b_, R_, mu_, phi_, _) in enumerate(cases):
        b[3 * q:3 * q + 3] = b_ * masses[q] / m_
        Rs.append(R_), mus.append(mu_), phis.append(phi_), nodes.append(q)
    npd = np.float64 if dtype == "f64" else np.float32
    vals = np.array([m * np.eye(3) for m in masses], dtype=npd)
    with vfpi.Solver(np.arange(N + 1), np.arange(N), vals, b.astype(npd), np.array(nodes),
                     None, np.array(Rs, dtype=npd), np.array(mus, dtype=npd),
                     np.array(phis, dtype=npd), dtype=dtype) as s:
        s.set_velocity(np.zeros(3 * N, dtype=npd))
        s.step()
        vg = s.get_velocity()
        lg = s.get_lambda().reshape(-1, 3)
    tol = 1e-12 if dtype == "f64" else 2e-6
    bq = b.astype(npd).astype(float)
    for q in range(N):
        sl = slice(3 * q, 3 * q + 3)
        if q < len(cases):
            v_ref, lam_ref, _ = textbook_point_contact(
                float(npd(masses[q])), bq[sl], np.array(Rs[q], dtype=npd).astype(float),
                float(npd(mus[q])), float(npd(phis[q])))
            assert np.allclose(lg[q], lam_ref, rtol=tol, atol=tol * np.abs(lam_ref).max())
        else:
            v_ref = bq[sl] / float(npd(masses[q]))
        assert np.allclose(vg[sl], v_ref, rtol=tol, atol=tol * np.abs(v_ref).max())


# ----------------------------------------------------------------------------
# per-iterate ladder
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("seed", range(3))
@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_ladder_random_s_and_d_contacts(seed, dtype):
    rng = np.random.default_rng(500 + seed)
    sc = scenes.random_problem(rng, 70, 12, d_contacts=6, density=0.08, couple=0.5,
                               dtype=dtype)
    ladder(sc)
    ladder(sc, force_path=1)
    ladder(sc, force_path=2, block_threads=64)


def test_ladder_small_lattice_f64():
    ladder(scenes.small_lattice(np.float64), ks=(1, 2, 10, 50))


def test_ladder_small_lattice_f32_both_paths():
    sc = scenes.small_lattice(np.float32)
    ladder(sc, ks=(1, 2, 10, 50))
    ladder(sc, ks=(1, 2, 10, 50), force_path=1, block_threads=128)


def test_ladder_fem_block_with_ragged_tail():
    # 13 x 11 x 5 cells: 14*12*6 = 1008 nodes, rows of 8..15 blocks, a partial last slice
    sc = scenes.fem_block_scene(13, 11, 5, seed=11, dtype=np.float32)
    ladder(sc, ks=(1, 3, 20), force_path=1)
    ladder(sc, ks=(1, 3, 20), force_path=2)


def test_ladder_terrain_lattice_medium():
    sc = scenes.terrain_lattice(dims=(40, 36, 6))
    ladder(sc, ks=(1, 5, 25), force_path=1)


# ----------------------------------------------------------------------------
# converged parity (task bar)
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("dtype,theta_th", [(np.float64, 1e-13), (np.float32, 1e-9)])
def test_converged_small_lattice(dtype, theta_th):
    sc = scenes.small_lattice(dtype)
    P = oracle_problem(sc)
    w = ov.frobenius_w(P)
    ref = ov.solve(P, w, sc.v0, theta_th=1e-13, l_max=100000)
    assert ref.converged
    with vfpi.Solver.from_scene(sc, theta_th=theta_th, l_max=4000) as s:
        r = s.solve(sc.v0)
    err = rel(r.v, ref.v)
    scc = scc_residual(P, np.asarray(r.v, float), np.asarray(r.lam, float).reshape(-1, 3))
    assert err <= (1e-10 if dtype == np.float64 else 1e-5), err
    assert scc <= 1e-6, scc
    if dtype == np.float64:
        assert r.converged and abs(r.iters - ref.iters) <= 2


def test_converged_random_with_d_contacts_matches_pgs_solution():
    from oracle.delassus import pgs
    rng = np.random.default_rng(42)
    sc = scenes.random_problem(rng, 40, 8, d_contacts=4, density=0.1, couple=0.3,
                               mu_range=(0.1, 0.6), dtype=np.float64)
    P = oracle_problem(sc)
    v_pgs, lam_pgs, _ = pgs(P)
    with vfpi.Solver.from_scene(sc, theta_th=1e-13, l_max=100000) as s:
        r = s.solve(sc.v0)
    assert r.converged
    assert rel(r.v, v_pgs) <= 1e-8
    assert dynamics_residual(P, r.v, r.lam) <= 1e-10


# ----------------------------------------------------------------------------
# other entry points
# ----------------------------------------------------------------------------

def test_matvec_integrate_and_device_pointers():
    sc = scenes.fem_block_scene(6, 5, 4, seed=3, dtype=np.float32)
    P = oracle_problem(sc)
    rng = np.random.default_rng(0)
    x = rng.normal(0, 1, P.n).astype(np.float32)
    with vfpi.Solver.from_scene(sc) as s:
        y = s.matvec(x)
        assert close(y, P.A @ x.astype(float), 1e-6)
        # device tensors in and out give the same numbers
        xd = torch.from_numpy(x).cuda()
        yd = torch.empty_like(xd)
        s.matvec(xd, out=yd)
        assert np.array_equal(yd.cpu().numpy(), y)
        s.set_velocity(sc.v0)
        s.solve()
        v = s.get_velocity()
        pos = sc.x0.copy()
        s.integrate(pos)
        assert np.allclose(pos, ov.integrate(sc.x0, v.astype(float), sc.h), rtol=0, atol=1e-15)
        posd = torch.from_numpy(sc.x0.copy()).cuda()
        s.integrate(posd)
        assert np.array_equal(posd.cpu().numpy(), pos)


def test_set_rhs_and_update_follow_new_data():
    sc = scenes.small_lattice(np.float64)
    rng = np.random.default_rng(5)
    b2 = sc.b * (1 + 0.1 * rng.standard_normal(sc.b.shape))
    phi2 = sc.phi + 0.05 * rng.standard_normal(sc.phi.shape)
    sc2 = scenes.dataclasses.replace(sc, b=b2, phi=phi2)
    P2 = oracle_problem(sc2)
    w = ov.frobenius_w(P2)
    ref = ov.solve(P2, w, sc.v0, theta_th=0.0, l_max=30)
    with vfpi.Solver.from_scene(sc, theta_th=0.0, l_max=30) as s:
        s.set_rhs(b2, phi2)
        r = s.solve(sc.v0)
    assert rel(r.v, ref.v) <= 1e-11
    # values update: scale A, b consistently -> same solution as the oracle on scaled data
    sc3 = scenes.dataclasses.replace(sc, vals=sc.vals * 2.0, b=sc.b * 2.0)
    P3 = oracle_problem(sc3)
    ref3 = ov.solve(P3, ov.frobenius_w(P3), sc.v0, theta_th=0.0, l_max=30)
    with vfpi.Solver.from_scene(sc, theta_th=0.0, l_max=30) as s:
        s.update(vals=sc3.vals, b=sc3.b)
        r3 = s.solve(sc.v0)
    assert rel(r3.v, ref3.v) <= 1e-11


def test_scalar_and_user_w():
    sc = scenes.small_lattice(np.float64)
    P = oracle_problem(sc)
    alpha = 0.9 * ov.optimal_alpha(P)
    ref = ov.solve(P, ov.scalar_w(P, alpha), sc.v0, theta_th=0.0, l_max=40)
    with vfpi.Solver.from_scene(sc, w_mode="scalar", alpha=alpha, theta_th=0.0, l_max=40) as s:
        assert np.array_equal(s.get_w(), np.full(P.n, alpha))
        r = s.solve(sc.v0)
    assert rel(r.v, ref.v) <= 1e-11
    wu = ov.frobenius_w(P) * 0.8
    ref = ov.solve(P, wu, sc.v0, theta_th=0.0, l_max=40)
    with vfpi.Solver.from_scene(sc, w_mode="user", w_user=wu, theta_th=0.0, l_max=40) as s:
        r = s.solve(sc.v0)
    assert rel(r.v, ref.v) <= 1e-11


def test_rms_norm_and_iteration_count():
    sc = scenes.small_lattice(np.float64)
    P = oracle_problem(sc)
    w = ov.frobenius_w(P)
    ref = ov.solve(P, w, sc.v0, theta_th=1e-6, l_max=1000, norm=ov.NORM_RMS)
    with vfpi.Solver.from_scene(sc, theta_th=1e-6, l_max=1000, norm="rms") as s:
        r = s.solve(sc.v0)
    assert r.iters == ref.iters and abs(r.theta - ref.theta) <= 1e-12 * ref.theta
    with vfpi.Solver.from_scene(sc, theta_th=0.0, l_max=7) as s:
        r = s.solve(sc.v0)
    assert r.iters == 7 and r.status == vfpi.VFPI_NOT_CONVERGED


def test_error_statuses():
    sc = scenes.small_lattice(np.float64)
    # a node in two contacts
    with pytest.raises(vfpi.VfpiError) as e:
        vfpi.Solver(sc.row_ptr, sc.col_idx, sc.vals, sc.b, np.array([0, 0]), None,
                    sc.R[:2], sc.mu[:2], sc.phi[:2], dtype="f64")
    assert e.value.status == -6
    # unsorted columns
    col = sc.col_idx.copy()
    col[[0, 1]] = col[[1, 0]]
    with pytest.raises(vfpi.VfpiError) as e:
        vfpi.Solver(sc.row_ptr, col, sc.vals, sc.b, sc.node_i, None, sc.R, sc.mu, sc.phi, dtype="f64")
    assert e.value.status == -1
    # non-finite b
    b = sc.b.copy()
    b[5] = np.nan
    with pytest.raises(vfpi.VfpiError) as e:
        vfpi.Solver(sc.row_ptr, sc.col_idx, sc.vals, b, sc.node_i, None, sc.R, sc.mu, sc.phi, dtype="f64")
    assert e.value.status == -2
    # a reflection is not a contact frame
    R = sc.R.copy()
    R[0, 2] *= -1
    with pytest.raises(vfpi.VfpiError) as e:
        vfpi.Solver(sc.row_ptr, sc.col_idx, sc.vals, sc.b, sc.node_i, None, R, sc.mu, sc.phi, dtype="f64")
    assert e.value.status == -1
    # divergent step size: NaN/Inf detected in the residual reduction, or l_max hit
    with vfpi.Solver.from_scene(sc, w_mode="scalar", alpha=1e6, theta_th=1e-12, l_max=3000) as s:
        with pytest.raises(vfpi.VfpiError) as e:
            s.solve(sc.v0)
        assert e.value.status == -2
    # NaN pushed through the unchecked per-step path is caught by the reduction
    with vfpi.Solver.from_scene(sc) as s:
        s.set_rhs(b=b)
        with pytest.raises(vfpi.VfpiError) as e:
            s.solve(sc.v0)
        assert e.value.status == -2


# ----------------------------------------------------------------------------
# full size, in the benchmark's launch configuration
# ----------------------------------------------------------------------------

@pytest.fixture(scope="module")
def terrain():
    return scenes.terrain_lattice()


def test_full_size_terrain_lattice_ladder(terrain):
    """1,572,864 DOF: GPU sweeps 1..10 against the oracle's, every entry."""
    sc = terrain
    P = oracle_problem(sc)
    w = ov.frobenius_w(P)
    with vfpi.Solver.from_scene(sc, theta_th=1e-5, l_max=200) as s:
        lay = s.layout()
        assert lay["path"] == 1 and lay["n_pad"] == sc.n_nodes
        assert close(s.get_w(), w, 1e-6)
        s.set_velocity(sc.v0)
        v = sc.v0.astype(float)
        for k in range(1, 11):
            s.step()
            r = ov.sweep(P, w, v)
            v = r.v_next
            if k in (1, 10):
                assert close(s.get_velocity(), v, F32_LADDER), k
                assert close(s.get_lambda().reshape(-1, 3), r.lam, 10 * F32_LADDER), k


def test_full_size_terrain_lattice_converged_properties(terrain):
    """Solve as the benchmark does; the returned iterate satisfies eq. (scc)
    (Prop. 4 makes that exact for every iterate) and the dynamics residual
    falls with the iteration count."""
    sc = terrain
    P = oracle_problem(sc)
    res = []
    with vfpi.Solver.from_scene(sc, theta_th=0.0, l_max=200) as s:
        for lm in (20, 200):
            s.set_velocity(sc.v0)
            it = 0
            while it < lm:
                s.step()
                it += 1
            v = s.get_velocity().astype(float)
            lam = s.get_lambda().astype(float).reshape(-1, 3)
            assert scc_residual(P, v, lam) <= 1e-6
            res.append(dynamics_residual(P, v, lam))
        r = s.solve(sc.v0)
        assert r.iters == 200
    assert res[1] < 0.5 * res[0]


def test_every_launch_variant_gives_identical_iterates():
    """Launch shapes only change which warp computes which row: the iterates
    are bitwise identical (theta may differ in its last bits, being reduced in
    a different grouping, so compare after a fixed number of sweeps)."""
    sc = scenes.terrain_lattice(dims=(40, 36, 6))
    ref = None
    with vfpi.Solver.from_scene(sc, theta_th=-1.0, l_max=12, force_path=1) as s:
        for var in list(range(16)) + [26, 27, 28, 29]:   # 12..15: symmetric storage; 26, 27:
            # 2-stage rings; 28, 29: symmetric blocks
            for grid in (0, 17):
                s.configure_launch(var, 0, grid)
                r = s.solve(sc.v0)
                out = (r.v.copy(), r.lam.copy())
                if ref is None:
                    ref = out
                assert np.array_equal(out[0], ref[0]), (var, grid)
                assert np.array_equal(out[1], ref[1]), (var, grid)


def test_tuner_picks_and_applies_a_shape(tmp_path):
    from paper_2201_09212_gb300 import tune
    sc = scenes.terrain_lattice(dims=(40, 36, 6))
    with vfpi.Solver.from_scene(sc, force_path=1) as s:
        res = tune.tune(s, sweeps=4, reps=1, cache=str(tmp_path / "t.json"))
        assert not res["cached"] and len(res["trials"]) >= 8
        lay = s.layout()
        assert lay["grid"] == res["grid"]
        again = tune.tune(s, cache=str(tmp_path / "t.json"))
        assert again["cached"] and again["kernel_variant"] == res["kernel_variant"]
        r = s.solve(sc.v0)
        assert np.isfinite(r.v).all()


def test_tma_and_register_shapes_agree_in_f64():
    sc = scenes.terrain_lattice(np.float64, dims=(40, 36, 6))
    ref = None
    with vfpi.Solver.from_scene(sc, theta_th=-1.0, l_max=12, force_path=1, dtype="f64") as s:
        for var in (0, 7, 8, 9, 10, 11, 12, 26, 27, 28, 29):
            s.configure_launch(var, 0, 0)
            r = s.solve(sc.v0)
            if ref is None:
                ref = (r.v.copy(), r.lam.copy())
            assert np.array_equal(r.v, ref[0]) and np.array_equal(r.lam, ref[1]), var
