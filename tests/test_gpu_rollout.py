"""Differentiable rollouts: torch autograd through the V-FPI solve (adjoint
kernel) against an FP64 dense reference gradient built from the oracle's
per-step dense adjoint, and against central differences (eps = 1e-4)."""
import numpy as np
import pytest

from oracle import vfpi as ov
from oracle.adjoint import adjoint as dense_adjoint
from paper_2201_09212_gb300 import scenes

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2201_09212_gb300 import vfpi  # noqa: E402
from paper_2201_09212_gb300.autograd import LatticeHarness, rollout  # noqa: E402

STEPS = 16


@pytest.fixture(scope="module")
def scene():
    return scenes.lattice_batch(2, seed=55, side_range=(4, 4), dtype=np.float64)


def oracle_rollout_grad(sc, steps):
    """FP64: forward with converged oracle solves, backward by chaining the dense
    per-step adjoints through b = M v + h M g - kappa (A - M)(x - x0), phi = z/h,
    x += h v_hat."""
    meta = sc.meta
    nq = meta["nodes"].astype(np.int64)
    dof_scene = np.repeat(np.arange(len(nq)), 3 * nq)
    comp = np.tile(np.arange(3), int(nq.sum()))
    h = sc.h
    m = sc.mass
    hg = h * m * meta["gravity"][dof_scene, comp]
    kap = (h * meta["k"] / meta["coef"])[dof_scene]
    zi = 3 * sc.node_i.astype(np.int64) + 2
    P = ov.make_problem(sc.row_ptr, sc.col_idx, sc.vals, sc.b, sc.node_i, sc.node_j, sc.R,
                        sc.mu, sc.phi)
    w = ov.frobenius_w(P)
    AmM = lambda u: P.A @ u - m * u
    x, v = sc.x0.copy(), sc.v0.astype(float).copy()
    tape = []
    for _ in range(steps):
        u = x - sc.x0
        P.b = m * v + hg - kap * AmM(u)
        P.phi = x[zi] / h
        r = ov.solve(P, w, v, theta_th=1e-14, l_max=200000)
        assert r.converged
        tape.append((P.b.copy(), P.phi.copy(), r.v.copy()))
        x = x + h * r.v
        v = r.v
    # L = sum over scenes of the mean z of the final positions
    xbar = np.zeros_like(x)
    for q in range(len(nq)):
        n0, n1 = sc.scene_ptr[q], sc.scene_ptr[q + 1]
        xbar[3 * n0 + 2:3 * n1:3] = 1.0 / (n1 - n0)
    vbar = np.zeros_like(v)
    mubar = np.zeros(sc.n_c)
    for k in reversed(range(steps)):
        b, phi, vhat = tape[k]
        P.b, P.phi = b, phi
        gvhat = vbar + h * xbar
        g_b, g_phi, g_mu, _ = dense_adjoint(P, w, vhat, gvhat)
        vbar = m * g_b
        xnew = xbar - kap * AmM(g_b)
        xnew[zi] += g_phi / h
        xbar = xnew
        mubar += g_mu
    return vbar, mubar, x


def gpu_rollout(sc, dtype, checkpoint=4, steps=STEPS, v0=None, mu=None, grad=True):
    dev = torch.device("cuda")
    td = torch.float64 if dtype == "f64" else torch.float32
    scd = sc if dtype == "f64" else sc.rounded(np.float32)
    th = 1e-14 if dtype == "f64" else 1e-8
    s = vfpi.Solver.from_scene(scd, dtype=dtype, theta_th=th, l_max=100000, norm="rms")
    H = LatticeHarness(scd, dev, dtype=td)
    v0 = torch.as_tensor(scd.v0 if v0 is None else v0, dtype=td, device=dev).clone()
    mu = torch.as_tensor(scd.mu if mu is None else mu, dtype=td, device=dev).clone()
    v0.requires_grad_(grad)
    mu.requires_grad_(grad)
    x0 = H.x_rest.clone()
    with torch.set_grad_enabled(grad):
        x, v = rollout(s, H, x0, v0, mu, steps, checkpoint=checkpoint)
        L = H.com_z(x).sum()
    if grad:
        L.backward()
        out = (float(L.detach()), v0.grad.cpu().numpy(), mu.grad.cpu().numpy(), x.detach().cpu().numpy())
    else:
        out = float(L)
    s.close()
    return out


def test_rollout_gradient_f64_matches_dense_reference(scene):
    vbar, mubar, x_ref = oracle_rollout_grad(scene, STEPS)
    L, g_v0, g_mu, x = gpu_rollout(scene, "f64")
    assert np.allclose(x, x_ref, rtol=0, atol=1e-12)
    assert np.abs(g_v0 - vbar).max() <= 1e-8 * np.abs(vbar).max()
    assert np.abs(g_mu - mubar).max() <= 1e-8 * max(np.abs(mubar).max(), 1e-300)
    assert np.abs(mubar).max() > 0, "no slipping contact: the mu gradient would be vacuous"


def test_rollout_gradient_f64_matches_central_differences(scene):
    L, g_v0, g_mu, _ = gpu_rollout(scene, "f64")
    eps = 1e-4
    rng = np.random.default_rng(0)
    for k in rng.choice(scene.n, 4, replace=False):
        vp, vm = scene.v0.copy(), scene.v0.copy()
        vp[k] += eps
        vm[k] -= eps
        fd = (gpu_rollout(scene, "f64", v0=vp, grad=False)
              - gpu_rollout(scene, "f64", v0=vm, grad=False)) / (2 * eps)
        assert abs(fd - g_v0[k]) <= 1e-5 * np.abs(g_v0).max() + 1e-6 * abs(fd)
    slipping = np.nonzero(np.abs(g_mu) > 1e-3 * np.abs(g_mu).max())[0]
    for m in slipping[:3]:
        mp, mm = scene.mu.copy(), scene.mu.copy()
        mp[m] += eps
        mm[m] -= eps
        fd = (gpu_rollout(scene, "f64", mu=mp, grad=False)
              - gpu_rollout(scene, "f64", mu=mm, grad=False)) / (2 * eps)
        assert abs(fd - g_mu[m]) <= 1e-3 * abs(fd) + 1e-6 * np.abs(g_mu).max()


def test_rollout_gradient_f32_against_fp64_reference(scene):
    vbar, mubar, _ = oracle_rollout_grad(scene.rounded(np.float32).as_f64(), STEPS)
    L, g_v0, g_mu, _ = gpu_rollout(scene, "f32")
    assert np.linalg.norm(g_v0 - vbar) <= 2e-3 * np.linalg.norm(vbar)
    assert np.linalg.norm(g_mu - mubar) <= 2e-2 * np.linalg.norm(mubar)


def test_checkpointing_does_not_change_the_gradient(scene):
    a = gpu_rollout(scene, "f32", checkpoint=4)
    b = gpu_rollout(scene, "f32", checkpoint=0)
    assert a[0] == b[0]
    assert np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2])


def test_autograd_solve_fails_loudly(scene):
    """A divergent step size (W = alpha I far above 2 / sigma_max) makes the
    forward residual non-finite: the differentiable solve raises VfpiError
    instead of returning the iterate.  A solve that reaches l_max warns with
    the scene indices (or raises on request), forward and adjoint alike."""
    from paper_2201_09212_gb300 import autograd as ag
    dev = torch.device("cuda")
    sc = scene
    H = LatticeHarness(sc, dev, dtype=torch.float64)
    v0 = torch.as_tensor(sc.v0, dtype=torch.float64, device=dev)
    mu = torch.as_tensor(sc.mu, dtype=torch.float64, device=dev).requires_grad_(True)
    b = torch.as_tensor(sc.b, dtype=torch.float64, device=dev).requires_grad_(True)
    phi = torch.as_tensor(sc.phi, dtype=torch.float64, device=dev)
    with vfpi.Solver.from_scene(sc, dtype="f64", w_mode="scalar", alpha=1e6, theta_th=1e-12,
                                l_max=3000) as s:
        with pytest.raises(vfpi.VfpiError) as e:
            ag.vfpi_solve(s, b, phi, mu, v0)
        assert e.value.status == vfpi.STATUS_CODES["VFPI_ERR_NONFINITE"]
    with vfpi.Solver.from_scene(sc, dtype="f64", theta_th=1e-14, l_max=3) as s:
        with pytest.warns(ag.VfpiNotConvergedWarning, match=r"forward solve: 2 scene\(s\)"):
            v = ag.vfpi_solve(s, b, phi, mu, v0)
        assert s.not_converged["forward"].tolist() == [0, 1]
        with pytest.raises(ag.VfpiNotConverged):
            ag.vfpi_solve(s, b, phi, mu, v0, on_not_converged="raise")
        s.set_tolerance(1e-13, 100000)
        v = ag.vfpi_solve(s, b, phi, mu, v0)
        assert s.not_converged["forward"].size == 0
        s.set_adjoint_tolerance(1e-14, 2, relative=True)
        with pytest.warns(ag.VfpiNotConvergedWarning, match=r"adjoint solve"):
            H.com_z(H.x_rest + sc.h * v).sum().backward()
        assert s.not_converged["adjoint"].tolist() == [0, 1]
