"""Virtual-node systems (eq. vnode; rigid bodies, S- and D-contacts through
virtual nodes) on the GPU against the FP64 oracle."""
import numpy as np
import pytest

from oracle import vfpi as ov
from paper_2201_09212_gb300 import scenes
from tests.conftest import oracle_problem
from tests.test_virtual_nodes import E_Z, box_on_ground

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2201_09212_gb300 import vfpi  # noqa: E402


def stacked_boxes(k_v):
    size = (0.2, 0.2, 0.1)
    body = scenes.rigid_boxes([dict(m=1.0, size=size, v=(0, 0, -0.1, 0, 0, 0)),
                               dict(m=0.5, size=size, v=(0.3, 0, -0.2, 0, 0, 0.5),
                                    force=(1.0, 0.0, 0.0))])
    sx, sy, sz = size
    corners = [np.array([ax * sx / 2, ay * sy / 2, 0.0]) for ax in (-1, 1) for ay in (-1, 1)]
    jv, vi, vj, p = [], [], [], 0
    for c in corners:
        jv += [(p, i, B) for (_, i, B) in scenes.point_jacobian(0, c + [0, 0, -sz / 2])]
        vi.append(p), vj.append(-1)
        p += 1
    for c in corners:
        jv += [(p, i, B) for (_, i, B) in scenes.point_jacobian(1, c + [0, 0, -sz / 2])]
        jv += [(p + 1, i, B) for (_, i, B) in scenes.point_jacobian(0, c + [0, 0, sz / 2])]
        vi.append(p), vj.append(p + 1)
        p += 2
    R = scenes.contact_frames(np.tile(E_Z, (8, 1)))
    nj = np.where(np.array(vj) >= 0, body.n_nodes + np.array(vj), -1)
    return scenes.add_virtual_nodes(body, jv, p, k_v, (body.n_nodes + np.array(vi), nj, R,
                                                       np.full(8, 0.4), np.zeros(8)))


@pytest.mark.parametrize("make", [lambda: box_on_ground(3.0)[0], lambda: stacked_boxes(3.0)])
@pytest.mark.parametrize("path", [1, 2])
def test_virtual_node_ladder_and_converged_f64(make, path):
    sc = make()
    P = oracle_problem(sc)
    w = ov.frobenius_w(P)
    with vfpi.Solver.from_scene(sc, theta_th=0.0, l_max=50, force_path=path) as s:
        r = s.solve(sc.v0)
        ref = ov.solve(P, w, sc.v0, theta_th=0.0, l_max=50)
        assert np.abs(r.v - ref.v).max() <= 1e-11 * np.abs(ref.v).max()
        s.set_tolerance(1e-13, 2_000_000)
        r = s.solve(sc.v0)
    ref = ov.solve(P, w, sc.v0, theta_th=1e-13, l_max=2_000_000)
    assert r.converged and abs(r.iters - ref.iters) <= 2
    assert np.abs(r.v - ref.v).max() <= 1e-9 * np.abs(ref.v).max()


@pytest.mark.parametrize("path", [1, 2])
def test_paper_box_rollout_f64(path):
    """The sliding box of Sec. V.B through the CUDA path in FP64 (k_v = 1 in
    the harness's units), ten time steps: each step's velocities and normal
    impulses are the oracle's V-FPI rollout's, the y error is mu times the z
    error, and the sinking is -h (sum of the normal impulses) / (4 k_v), the
    virtual-node perturbation of Sec. III.A."""
    from tests.test_virtual_nodes import PAPER_BOX, box_rollout

    def gpu(sc):
        with vfpi.Solver.from_scene(sc, theta_th=1e-12, l_max=3_000_000, force_path=path) as s:
            r = s.solve(sc.v0)
        assert r.converged
        return r.v, r.lam

    def cpu(sc):
        P = oracle_problem(sc)
        r = ov.solve(P, ov.frobenius_w(P), sc.v0, theta_th=1e-12, l_max=3_000_000)
        assert r.converged
        return r.v, r.lam

    k_v, mu, h = 1.0, PAPER_BOX["mu"], PAPER_BOX["h"]
    ex, ey, ez, lam_n = box_rollout(k_v, gpu, steps=10)
    rx, ry, rz, rlam = box_rollout(k_v, cpu, steps=10)
    assert ex.max() <= 1e-12
    assert np.allclose(ey, ry, rtol=1e-5, atol=0.0) and np.allclose(ez, rz, rtol=1e-5, atol=0.0)
    assert np.allclose(lam_n, rlam, rtol=1e-5, atol=0.0)
    assert np.allclose(ey / ez, mu, rtol=1e-5, atol=0.0)
    assert np.allclose(ez, h * lam_n / (4 * k_v), rtol=1e-5, atol=0.0)
