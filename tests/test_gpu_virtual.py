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
