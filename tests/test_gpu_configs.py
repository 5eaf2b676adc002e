"""The remaining workload shapes as parity cases: the full-size tetrahedral FEM
block and a 100-step trajectory of the small lattice with A re-assembled every
step (Gauss-Newton springs at the current configuration)."""
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


def test_fem_block_full_size_ladder():
    """64x64x16-cell Kuhn-split block (215,475 DOF, 1,026,481 blocks, 4,225
    contacts), FP32: sweeps 1..10 against the FP64 oracle, every entry."""
    sc = scenes.fem_block()
    P = oracle_problem(sc)
    w = ov.frobenius_w(P)
    with vfpi.Solver.from_scene(sc, theta_th=0.0, l_max=10) as s:
        assert s.layout()["path"] == 1
        r = s.solve(sc.v0)
    ref = ov.solve(P, w, sc.v0, theta_th=0.0, l_max=10)
    assert np.abs(r.v - ref.v).max() <= 1e-5 * np.abs(ref.v).max()
    assert np.linalg.norm(r.v - ref.v) <= 1e-5 * np.linalg.norm(ref.v)
    assert scc_residual(P, np.asarray(r.v, float), np.asarray(r.lam, float).reshape(-1, 3)) <= 1e-6


def test_small_lattice_trajectory_f64():
    """100 steps of the 6x6x6 lattice falling on the ground (FP64): each step
    re-assembles A and b at the current positions, updates phi = z / h, solves
    to convergence and integrates x += h v_hat on the device; the GPU state
    tracks the oracle's step by step."""
    sc = scenes.small_lattice(np.float64)
    nx = ny = nz = 6
    meta = sc.meta
    x_rest = sc.x0.reshape(-1, 3).copy()
    x_g = sc.x0.copy()
    x_o = sc.x0.copy()
    v_g = sc.v0.copy()
    v_o = sc.v0.copy()
    bottom = sc.node_i
    worst = 0.0
    with vfpi.Solver.from_scene(sc, theta_th=1e-13, l_max=100000) as s:
        for k in range(100):
            rp, col, vals, b = scenes.lattice_system(nx, ny, nz, x_g.reshape(-1, 3), x_rest,
                                                     v_g, k=meta["k"], c=meta["c"], h=sc.h)
            phi = x_g[3 * bottom + 2] / sc.h
            s.update(vals=vals, b=b)
            s.set_rhs(phi=phi)
            r = s.solve(v_g)
            assert r.converged
            s.integrate(x_g)
            v_g = np.asarray(r.v, float)
            # oracle, on its own state
            rp, col, vals_o, b_o = scenes.lattice_system(nx, ny, nz, x_o.reshape(-1, 3), x_rest,
                                                         v_o, k=meta["k"], c=meta["c"], h=sc.h)
            P = ov.make_problem(rp, col, vals_o, b_o, sc.node_i, sc.node_j, sc.R, sc.mu,
                                x_o[3 * bottom + 2] / sc.h)
            ro = ov.solve(P, ov.frobenius_w(P), v_o, theta_th=1e-13, l_max=100000)
            x_o = ov.integrate(x_o, ro.v, sc.h)
            v_o = ro.v
            worst = max(worst, np.abs(v_g - v_o).max() / np.abs(v_o).max())
    assert worst <= 1e-8, worst
    assert np.abs(x_g - x_o).max() <= 1e-12
    # the lattice came to rest on the ground
    assert x_g[3 * bottom + 2].min() > -1e-4
