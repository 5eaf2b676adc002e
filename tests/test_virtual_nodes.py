"""Virtual nodes (Sec. III.A, eq. vforce, eq. vnode): Prop. 1, Prop. 2 and an
analytic sliding box, on the FP64 oracle."""
import pathlib

import numpy as np
import pytest

from oracle import vfpi as ov
from oracle.delassus import pgs_general
from paper_2201_09212_gb300 import scenes
from tests.conftest import oracle_problem

E_Z = np.array([0.0, 0.0, 1.0])


def box_on_ground(k_v, F=8.0, m=1.0, size=(0.2, 0.2, 0.1), v=(0, 0, 0, 0, 0, 0), mu=0.5,
                  gap=0.0):
    """One rigid box resting on z = 0, contact at its four bottom corners
    through virtual nodes."""
    sx, sy, sz = size
    body = scenes.rigid_boxes([dict(m=m, size=size, v=v, force=(F, 0.0, 0.0))])
    corners = [np.array([ax * sx / 2, ay * sy / 2, -sz / 2]) for ax in (-1, 1) for ay in (-1, 1)]
    jv = []
    for p, r in enumerate(corners):
        jv += [(p, i, B) for (_, i, B) in scenes.point_jacobian(0, r)]
    R = scenes.contact_frames(np.tile(E_Z, (4, 1)))
    contacts = (np.arange(2, 6), -np.ones(4, int), R, np.full(4, mu), np.full(4, gap / body.h))
    return scenes.add_virtual_nodes(body, jv, 4, k_v, contacts), corners


def solve(sc, theta=1e-14):
    P = oracle_problem(sc)
    w = ov.frobenius_w(P)
    r = ov.solve(P, w, sc.v0, theta_th=theta, l_max=2_000_000)
    assert r.converged
    return r, P


@pytest.mark.parametrize("k_v", [1e-3, 1.0, 1e6])
def test_prop1_augmented_matrix_is_spd(k_v):
    sc, _ = box_on_ground(k_v)
    A = sc.dense_A()
    assert np.allclose(A, A.T)
    np.linalg.cholesky(A)


def test_prop2_virtual_node_contact_tends_to_the_original_one():
    """S-contacts at non-nodal points of a lattice (barycentric in a bottom
    cell): the virtual-node solution approaches the original contact problem
    (general Jacobian J_c = R J_v, solved by PGS) as k_v grows, error ~ 1/k_v."""
    rng = np.random.default_rng(3)
    base = scenes.lattice_scene(3, 3, 2, seed=8, v_down=0.3)
    base = scenes.dataclasses.replace(base, node_i=np.zeros(0, np.int32),
                                      node_j=np.zeros(0, np.int32), R=np.zeros((0, 3, 3)),
                                      mu=np.zeros(0), phi=np.zeros(0))
    # three contact points inside bottom cells, bilinear weights of the cell's 4 nodes
    cells = [(0, 0), (1, 0), (1, 1)]
    jv, J_rows = [], []
    for p, (cx, cy) in enumerate(cells):
        a, bb = rng.uniform(0.2, 0.8, 2)
        wts = {(cx, cy): (1 - a) * (1 - bb), (cx + 1, cy): a * (1 - bb),
               (cx, cy + 1): (1 - a) * bb, (cx + 1, cy + 1): a * bb}
        for (ix, iy), wgt in wts.items():
            jv.append((p, ix + 3 * iy, wgt * np.eye(3)))
    R = scenes.contact_frames(np.tile(E_Z, (3, 1)))
    mu = np.array([0.3, 0.6, 0.9])
    phi = np.array([-0.05, 0.0, 0.02])
    Jv = np.zeros((9, base.n))
    for p, i, B in jv:
        Jv[3 * p:3 * p + 3, 3 * i:3 * i + 3] += B
    Jc = np.zeros((9, base.n))
    for p in range(3):
        Jc[3 * p:3 * p + 3] = R[p] @ Jv[3 * p:3 * p + 3]
    v_ref, lam_ref = pgs_general(base.dense_A(), base.b, Jc, mu, phi)
    errs = []
    for k_v in (1e-2, 1e-1, 1.0):
        sc = scenes.add_virtual_nodes(base, jv, 3, k_v, (base.n_nodes + np.arange(3),
                                                         -np.ones(3, int), R, mu, phi))
        r, P = solve(sc)
        errs.append(np.linalg.norm(r.v[:base.n] - v_ref) / np.linalg.norm(v_ref))
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 2e-2 and errs[1] / errs[2] > 5 and errs[0] / errs[1] > 5


def test_prop2_with_d_contacts_between_two_bodies():
    """Two rigid boxes stacked; the top box's bottom corners touch the lower
    box's top face through pairs of virtual nodes (D-contacts); the lower box
    stands on the ground (S-contacts).  The original problem has the
    non-nodal Jacobian R (J_top - J_bottom)."""
    size = (0.2, 0.2, 0.1)
    body = scenes.rigid_boxes([dict(m=1.0, size=size, v=(0, 0, -0.1, 0, 0, 0)),
                               dict(m=0.5, size=size, v=(0.3, 0, -0.2, 0, 0, 0.5),
                                    force=(1.0, 0.0, 0.0))])
    sx, sy, sz = size
    corners = [np.array([ax * sx / 2, ay * sy / 2, 0.0]) for ax in (-1, 1) for ay in (-1, 1)]
    jv, vi, vj = [], [], []
    p = 0
    for c in corners:           # ground contacts of box 0 (its bottom corners)
        jv += [(p, i, B) for (_, i, B) in scenes.point_jacobian(0, c + [0, 0, -sz / 2])]
        vi.append(p)
        vj.append(-1)
        p += 1
    for c in corners:           # box 1 bottom corner against box 0 top face
        jv += [(p, i, B) for (_, i, B) in scenes.point_jacobian(1, c + [0, 0, -sz / 2])]
        jv += [(p + 1, i, B) for (_, i, B) in scenes.point_jacobian(0, c + [0, 0, sz / 2])]
        vi.append(p)
        vj.append(p + 1)
        p += 2
    nv = p
    R = scenes.contact_frames(np.tile(E_Z, (8, 1)))
    mu = np.full(8, 0.4)
    phi = np.zeros(8)
    Jv = np.zeros((3 * nv, body.n))
    for q, i, B in jv:
        Jv[3 * q:3 * q + 3, 3 * i:3 * i + 3] += B
    Jc = np.zeros((24, body.n))
    for m in range(8):
        Jm = Jv[3 * vi[m]:3 * vi[m] + 3] - (Jv[3 * vj[m]:3 * vj[m] + 3] if vj[m] >= 0 else 0.0)
        Jc[3 * m:3 * m + 3] = R[m] @ Jm
    v_ref, _ = pgs_general(body.dense_A(), body.b, Jc, mu, phi)
    errs = []
    # (the plain iteration slows down roughly in proportion to k_v, Sec. IV.C)
    for k_v in (3.0, 30.0):
        sc = scenes.add_virtual_nodes(
            body, jv, nv, k_v,
            (body.n_nodes + np.array(vi), np.where(np.array(vj) >= 0, body.n_nodes + np.array(vj), -1),
             R, mu, phi))
        r, P = solve(sc)
        errs.append(np.linalg.norm(r.v[:body.n] - v_ref) / np.linalg.norm(v_ref))
    assert errs[0] / errs[1] > 5 and errs[1] < 0.05


def test_sliding_box_matches_the_analytic_motion():
    """A box pushed by F > mu m g slides with a = F/m - mu g (backward Euler is
    exact for constant forces).  The virtual-node compliance lets the corners
    sink a little and lightens the normal (hence friction) impulse; both the
    sliding-velocity error and the penetration shrink like 1/k_v -- the trend
    of the paper's box experiment (Sec. V.B)."""
    F, m, mu, g = 8.0, 1.0, 0.5, scenes.GRAVITY
    h = 1e-3
    steps = 10
    pen, verr = [], []
    for k_v in (0.3, 3.0, 30.0):
        v = np.zeros(6)
        z = 0.0
        deepest, worst = 0.0, 0.0
        for k in range(steps):
            sc, corners = box_on_ground(k_v, F=F, m=m, v=v, mu=mu, gap=z)
            r, P = solve(sc, theta=1e-13)
            v = r.v[:6]
            z += h * v[2]
            deepest = min(deepest, z)
            worst = max(worst, abs(v[0] - (k + 1) * h * (F / m - mu * g)))
        pen.append(-deepest)
        verr.append(worst)
    assert pen[0] > pen[1] > pen[2] > 0
    assert 5 < pen[0] / pen[1] < 20 and 5 < pen[1] / pen[2] < 20
    assert verr[0] > verr[1] > verr[2] and verr[1] / verr[2] > 5
    assert verr[2] < 0.05 * (steps * h * (F / m - mu * g))


GOLDEN_BOX = pathlib.Path(__file__).parent / "golden" / "box_sliding_errors.txt"
PAPER_BOX = dict(m=0.5, side=0.2, mu=0.2, h=0.01)


def paper_box(k_v, v, z, F=2.0):
    """The sliding box of Sec. V.B: a cube of side 0.2 m and mass 0.5 kg on
    z = 0, friction coefficient 0.2, contacts at the four bottom vertices
    through virtual nodes, a constant force F along y, time step 10 ms.  The
    paper does not print its force; 2 N exceeds the friction limit
    (0.98 N), so the box slides from the first step.  ``z`` is the current
    height of the centre (its sinking), which sets the gap phi = z / h."""
    m, L, mu, h = PAPER_BOX["m"], PAPER_BOX["side"], PAPER_BOX["mu"], PAPER_BOX["h"]
    body = scenes.rigid_boxes([dict(m=m, size=(L, L, L), v=v, force=(0.0, F, 0.0))], h=h)
    corners = [np.array([ax * L / 2, ay * L / 2, -L / 2]) for ax in (-1, 1) for ay in (-1, 1)]
    jv = []
    for p, r in enumerate(corners):
        jv += [(p, i, B) for (_, i, B) in scenes.point_jacobian(0, r)]
    R = scenes.contact_frames(np.tile(E_Z, (4, 1)))
    return scenes.add_virtual_nodes(body, jv, 4, k_v, (np.arange(2, 6), -np.ones(4, int), R,
                                                       np.full(4, mu), np.full(4, z / h)))


def pgs_box_solve(sc):
    """The augmented contact problem (eq. vnode) solved through its Delassus
    operator: contacts act on the virtual nodes (J_c rows R_m at node 2 + m)."""
    A = sc.dense_A()
    J = np.zeros((3 * sc.n_c, A.shape[0]))
    for q in range(sc.n_c):
        J[3 * q:3 * q + 3, 3 * sc.node_i[q]:3 * sc.node_i[q] + 3] = sc.R[q]
    v, lam = pgs_general(A, sc.b, J, sc.mu, sc.phi)
    return v, lam.reshape(-1, 3)


def box_rollout(k_v, solve, steps, F=2.0):
    """Per-step position errors against the analytic motion (backward Euler of
    a = F/m - mu g along y, no motion along x or z) and the summed normal
    impulse of the four contacts."""
    m, mu, h, g = PAPER_BOX["m"], PAPER_BOX["mu"], PAPER_BOX["h"], scenes.GRAVITY
    v = np.zeros(6)
    pos = np.zeros(3)
    va = ya = 0.0
    ex, ey, ez, lam_n = [], [], [], []
    for _ in range(steps):
        v, lam = solve(paper_box(k_v, v, pos[2], F))
        v = np.asarray(v, float)[:6]
        pos = pos + h * v[:3]
        va += h * (F / m - mu * g)
        ya += h * va
        ex.append(abs(pos[0]))
        ey.append(abs(pos[1] - ya))
        ez.append(abs(pos[2]))
        lam_n.append(float(np.asarray(lam, float).reshape(-1, 3)[:, 0].sum()))
    return np.array(ex), np.array(ey), np.array(ez), np.array(lam_n)


def test_paper_box_table_trend_on_the_oracle():
    """The paper's table (tests/golden/box_sliding_errors.txt) shows, to its
    printed rounding, no error along x, a y error of mu times the z error and
    errors falling tenfold per decade of k_v.  The oracle's box shows the same,
    and its sinking is the virtual-node perturbation of Sec. III.A: the SCC
    hold on the virtual nodes, whose velocity differs from the contact point's
    by k_v^-1 lambda, so with all four corners in contact
    z_k = -h (sum of the normal impulses) / (4 k_v) at every step."""
    rows = np.loadtxt(GOLDEN_BOX)
    half = 0.5e-4                                     # four printed decimals
    mu = PAPER_BOX["mu"]
    for k_v, exm, eym, ezm in rows:
        assert exm == 0.0
        assert (eym - half) / (ezm + half) <= mu <= (eym + half) / (ezm - half), k_v
    for (k0, _, _, z0), (k1, _, _, z1) in zip(rows[:-1], rows[1:]):
        assert k1 == 10 * k0
        assert abs(z0 / z1 - 10.0) <= 0.01 * 10.0 + 10.0 * half * (1 / z1 + 1 / z0)
    h = PAPER_BOX["h"]
    means = []
    for k_v in (1.0, 10.0):                           # the harness's k_v (A in impulse units)
        ex, ey, ez, lam_n = box_rollout(k_v, pgs_box_solve, steps=20)
        assert ex.max() <= 1e-15
        assert np.allclose(ey / ez, mu, rtol=1e-7, atol=0.0)
        assert np.allclose(ez, h * lam_n / (4 * k_v), rtol=1e-9, atol=0.0)
        means.append(ez.mean())
    assert abs(means[0] / means[1] - 10.0) <= 0.01 * 10.0
