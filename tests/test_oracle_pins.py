"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each pin checks the oracle against something other than itself: textbook
point-mass Coulomb contact, brute-force minimisation, an independent solver
(projected Gauss-Seidel on the Delassus operator), exhaustive active-set
enumeration, exact invariants stated by the paper (Prop. 3, Prop. 4, the
consistency remark, Lemma 2), and central finite differences.
"""
import math

import numpy as np
import pytest
import scipy.optimize as so

from oracle import vfpi as ov
from oracle.adjoint import adjoint, strict_jacobian
from oracle.checks import contact_velocity, dynamics_residual, scc_residual, mode_of
from oracle.delassus import pgs
from oracle.enumerate import enumerate_scc
from paper_2201_09212_gb300 import scenes
from tests.conftest import oracle_problem


# ----------------------------------------------------------------------------
# helpers building tiny problems directly
# ----------------------------------------------------------------------------

def point_masses(masses, b, R, mu, phi, contact_nodes):
    """Independent point masses (block-diagonal A = m_i I), S-contacts on some nodes."""
    N = len(masses)
    vals = np.array([m * np.eye(3) for m in masses])
    return ov.make_problem(np.arange(N + 1), np.arange(N), vals, b,
                           np.asarray(contact_nodes), -np.ones(len(contact_nodes), int),
                           R, mu, phi)


def textbook_point_contact(m, b, R, mu, phi):
    """Point mass ``m`` with momentum ``b`` hitting a contact frame ``R``:
    impulse-momentum balance plus Coulomb's law (open / stick / slide)."""
    v_free = b / m
    u = R @ v_free
    u[0] += phi
    if u[0] >= 0.0:
        return v_free, np.zeros(3), "open"
    ln = -m * u[0]                      # stop the approach
    ut = u[1:]
    if m * np.linalg.norm(ut) <= mu * ln:
        lt = -m * ut                    # stop the sliding
        mode = "stick"
    else:
        lt = -mu * ln * ut / np.linalg.norm(ut)   # kinetic friction opposes sliding
        mode = "slip"
    lam = np.concatenate([[ln], lt])
    return v_free + R.T @ lam / m, lam, mode


def single_node_cases(rng):
    """(m, b, R, mu, phi, expected_mode) covering open, stick and slip."""
    cases = []
    for mode in ("open", "stick", "slip"):
        for _ in range(4):
            m = rng.uniform(0.5, 3.0)
            R = scenes.random_rotations(rng, 1)[0]
            mu = rng.uniform(0.2, 1.0)
            phi = rng.uniform(-0.3, 0.3)
            if mode == "open":
                u = np.array([rng.uniform(0.1, 1.0), *rng.normal(0, 1, 2)])
            elif mode == "stick":
                un = -rng.uniform(0.5, 1.5)
                ut = rng.normal(0, 1, 2)
                ut *= 0.5 * mu * (-un) / np.linalg.norm(ut)
                u = np.array([un, *ut])
            else:
                un = -rng.uniform(0.5, 1.5)
                ut = rng.normal(0, 1, 2)
                ut *= 3.0 * mu * (-un) / np.linalg.norm(ut)
                u = np.array([un, *ut])
            u_free = u.copy()
            u_free[0] -= phi
            b = m * (R.T @ u_free)
            cases.append((m, b, R, mu, phi, mode))
    return cases


# ----------------------------------------------------------------------------
# ProjectFC (eq. operator)
# ----------------------------------------------------------------------------

def test_strict_projection_is_disk_projection(rng):
    """Normal part clamped at 0; tangential part is the nearest point of the disk
    of radius mu*lambda_n (checked against dense sampling of the disk)."""
    for _ in range(200):
        ls = rng.normal(0, 1, 3)
        mu = rng.uniform(0, 1.5)
        lam = ov.project_strict(ls[None], np.array([mu]))[0]
        assert lam[0] == max(ls[0], 0.0)
        radius = mu * lam[0]
        r = np.sqrt(rng.uniform(0, 1, 4000)) * radius
        a = rng.uniform(0, 2 * np.pi, 4000)
        pts = np.stack([r * np.cos(a), r * np.sin(a)], 1)
        best = np.linalg.norm(pts - ls[1:], axis=1).min()
        assert np.linalg.norm(lam[1:] - ls[1:]) <= best + 1e-12
        assert np.hypot(*lam[1:]) <= radius * (1 + 1e-12) + 1e-300


def test_strict_projection_tie_cases():
    mu = np.array([0.5])
    assert np.array_equal(ov.project_strict(np.array([[0.0, 1.0, 0.0]]), mu), np.zeros((1, 3)))
    assert np.array_equal(ov.project_strict(np.array([[-1.0, 1.0, 2.0]]), mu), np.zeros((1, 3)))
    # on the cone boundary both branches coincide
    on = np.array([[2.0, 0.6, 0.8]])
    assert np.allclose(ov.project_strict(on, mu), on, rtol=0, atol=1e-15)
    # mu = 0: frictionless, tangential impulse vanishes
    assert np.array_equal(ov.project_strict(np.array([[1.0, 3.0, 4.0]]), np.array([0.0])),
                          np.array([[1.0, 0.0, 0.0]]))


def test_proximal_projection_is_euclidean_cone_projection(rng):
    """Nearest point of the friction cone (eq. genfc): the result lies in the cone,
    no sampled cone point is closer, and the variational inequality
    (x - p)^T (y - p) <= 0 (the normal-cone property used in Lemma 3) holds."""
    for _ in range(100):
        x = rng.normal(0, 1, 3)
        mu = rng.uniform(0.1, 1.5)
        p = ov.project_proximal(x[None], np.array([mu]))[0]
        assert p[0] >= 0 and np.hypot(p[1], p[2]) <= mu * p[0] * (1 + 1e-12) + 1e-15
        yn = rng.uniform(0, 3, 20000)
        ang = rng.uniform(0, 2 * np.pi, 20000)
        rad = np.sqrt(rng.uniform(0, 1, 20000)) * mu * yn
        ys = np.stack([yn, rad * np.cos(ang), rad * np.sin(ang)], 1)
        assert np.linalg.norm(x - p) <= np.linalg.norm(ys - x, axis=1).min() + 1e-12
        assert ((ys - p) @ (x - p)).max() <= 1e-12
    # inside: unchanged; polar cone: apex
    assert np.array_equal(ov.project_proximal(np.array([[2.0, 0.1, 0.1]]), np.array([0.5])),
                          np.array([[2.0, 0.1, 0.1]]))
    assert np.array_equal(ov.project_proximal(np.array([[-2.0, 0.1, 0.1]]), np.array([0.5])),
                          np.zeros((1, 3)))


def test_lemma2_slip_derivative_norm_is_mu(rng):
    """Lemma 2: in slip, ||d lambda_t / d lambda*_n|| = mu (finite differences)."""
    for _ in range(50):
        mu = rng.uniform(0.1, 1.2)
        ln = rng.uniform(0.5, 2.0)
        t = rng.normal(0, 1, 2)
        t *= rng.uniform(1.5, 4.0) * mu * ln / np.linalg.norm(t)
        ls = np.array([ln, *t])
        eps = 1e-6
        d = (ov.project_strict((ls + [eps, 0, 0])[None], np.array([mu]))[0]
             - ov.project_strict((ls - [eps, 0, 0])[None], np.array([mu]))[0]) / (2 * eps)
        assert abs(np.linalg.norm(d[1:]) - mu) < 1e-7
        Pp, dmu = strict_jacobian(ls, mu)
        assert np.allclose(Pp[:, 0], d, atol=1e-7)
        # the full Jacobian by columns
        for k in range(3):
            e = np.zeros(3)
            e[k] = eps
            col = (ov.project_strict((ls + e)[None], np.array([mu]))[0]
                   - ov.project_strict((ls - e)[None], np.array([mu]))[0]) / (2 * eps)
            assert np.allclose(Pp[:, k], col, atol=1e-7)
        dm = (ov.project_strict(ls[None], np.array([mu + eps]))[0]
              - ov.project_strict(ls[None], np.array([mu - eps]))[0]) / (2 * eps)
        assert np.allclose(dmu, dm, atol=1e-7)


# ----------------------------------------------------------------------------
# W (Sec. IV.C) and Prop. 3
# ----------------------------------------------------------------------------

def test_frobenius_w_is_the_tied_minimiser(rng):
    """frobenius_w minimises ||I - W A||_F over diagonal W with the Prop. 3 tying
    (brute-force numerical minimisation of the dense norm)."""
    sc = scenes.random_problem(rng, 5, 1, d_contacts=1, density=0.6)
    P = oracle_problem(sc)
    A = P.A.toarray()
    w = ov.frobenius_w(P)
    groups = [list(range(3 * sc.node_i[0], 3 * sc.node_i[0] + 3)),
              list(range(3 * sc.node_i[1], 3 * sc.node_i[1] + 3))
              + list(range(3 * sc.node_j[1], 3 * sc.node_j[1] + 3))]
    tied = set(sum(groups, []))
    free = [r for r in range(P.n) if r not in tied]

    def expand(p):
        ww = np.zeros(P.n)
        for g, val in zip(groups, p[:len(groups)]):
            ww[g] = val
        ww[free] = p[len(groups):]
        return ww

    f = lambda p: np.sum((np.eye(P.n) - np.diag(expand(p)) @ A) ** 2)
    res = so.minimize(f, np.full(len(groups) + len(free), 0.1), method="BFGS",
                      options=dict(gtol=1e-12, maxiter=10000))
    assert np.allclose(expand(res.x), w, rtol=1e-6, atol=1e-9)
    assert f(np.concatenate([[w[g[0]] for g in groups], w[free]])) <= res.fun + 1e-12
    # the paper's closed form on the untied rows: w_rr = a_rr / ||A_r*||^2
    for r in free:
        assert math.isclose(w[r], A[r, r] / np.sum(A[r] ** 2), rel_tol=1e-14)


def test_prop3_surrogate_delassus_is_diagonal(rng):
    """Prop. 3: with tied W, J_c W J_c^T = diag(gamma_m I3), gamma = w_i (S) or
    w_i + w_j (D) -- checked on the dense product."""
    sc = scenes.random_problem(rng, 9, 3, d_contacts=2)
    P = oracle_problem(sc)
    w = ov.frobenius_w(P)
    J = P.Jc.toarray()
    Gam = J @ np.diag(w) @ J.T
    for m in range(P.n_c):
        gi = w[3 * sc.node_i[m]]
        g = gi + (w[3 * sc.node_j[m]] if sc.node_j[m] >= 0 else 0.0)
        for k in range(P.n_c):
            blk = Gam[3 * m:3 * m + 3, 3 * k:3 * k + 3]
            assert np.allclose(blk, g * np.eye(3) if k == m else 0.0, atol=1e-14)
    assert np.allclose(ov.gamma_blocks(P, w), [Gam[3 * m:3 * m + 3, 3 * m:3 * m + 3]
                                               for m in range(P.n_c)], atol=1e-14)


# ----------------------------------------------------------------------------
# sweep and solve against closed forms
# ----------------------------------------------------------------------------

def test_single_point_mass_matches_textbook_coulomb(rng):
    """With W = A^{-1} (= the Frobenius W for A = m I) one sweep lands on the
    textbook point-mass solution and the next sweep does not move (theta = 0)."""
    seen = set()
    for m, b, R, mu, phi, mode in single_node_cases(rng):
        P = point_masses([m], b, R[None], [mu], [phi], [0])
        w = ov.frobenius_w(P)
        assert np.allclose(w, 1.0 / m, rtol=1e-15)
        v_ref, lam_ref, mode_ref = textbook_point_contact(m, b, R, mu, phi)
        assert mode_ref == mode
        seen.add(mode)
        res = ov.solve(P, w, rng.normal(0, 1, 3), theta_th=1e-300, l_max=2)
        r1 = ov.sweep(P, w, rng.normal(0, 1, 3))
        assert np.allclose(r1.v_next, v_ref, rtol=1e-13, atol=1e-13)
        assert np.allclose(r1.lam[0], lam_ref, rtol=1e-13, atol=1e-13)
        assert res.thetas[1] <= 1e-14 * max(1.0, np.abs(v_ref).max())
        assert scc_residual(P, r1.v_next, r1.lam) < 1e-12
    assert seen == {"open", "stick", "slip"}


def test_independent_point_masses_one_sweep(rng):
    """Block-diagonal A with random masses, a subset of nodes in contact: every
    node independently matches the textbook solution after one sweep."""
    N = 12
    masses = rng.uniform(0.5, 2.0, N)
    contact_nodes = rng.permutation(N)[:7]
    cases = single_node_cases(rng)
    b = rng.normal(0, 1, 3 * N)
    Rs, mus, phis = [], [], []
    for q, node in enumerate(contact_nodes):
        m_, b_, R_, mu_, phi_, _ = cases[q]
        b[3 * node:3 * node + 3] = b_ * masses[node] / m_
        Rs.append(R_), mus.append(mu_), phis.append(phi_)
    P = point_masses(masses, b, np.array(Rs), mus, phis, contact_nodes)
    w = ov.frobenius_w(P)
    r = ov.sweep(P, w, np.zeros(3 * N))
    for node in range(N):
        sl = slice(3 * node, 3 * node + 3)
        if node in contact_nodes:
            q = list(contact_nodes).index(node)
            v_ref, lam_ref, _ = textbook_point_contact(masses[node], b[sl], Rs[q], mus[q], phis[q])
            assert np.allclose(r.lam[q], lam_ref, rtol=1e-12, atol=1e-12)
        else:
            v_ref = b[sl] / masses[node]
        assert np.allclose(r.v_next[sl], v_ref, rtol=1e-12, atol=1e-12)


def test_iterates_satisfy_surrogate_scc_exactly(rng):
    """Prop. 4: every iterate's (J v^{l+1} + phi, lambda) solves the surrogate
    contact problem exactly, i.e. satisfies eq. (scc) to rounding, and
    J v^{l+1} = Gamma lambda + eta (eq. subp)."""
    sc = scenes.random_problem(rng, 14, 5, d_contacts=2)
    P = oracle_problem(sc)
    w = ov.frobenius_w(P)
    v = sc.v0.astype(float)
    for _ in range(6):
        r = ov.sweep(P, w, v)
        Jv = (P.Jc @ r.v_next).reshape(-1, 3)
        gam = ov.gamma_blocks(P, w)
        assert np.allclose(Jv, np.einsum("mab,mb->ma", gam, r.lam) + r.eta, atol=1e-12)
        assert scc_residual(P, r.v_next, r.lam) < 1e-11
        v = r.v_next


def test_theta_is_two_norm_of_the_update(rng):
    sc = scenes.random_problem(rng, 10, 3)
    P = oracle_problem(sc)
    w = ov.frobenius_w(P)
    r = ov.sweep(P, w, sc.v0)
    dv = (r.v_next - sc.v0).astype(np.longdouble)
    assert math.isclose(r.theta, float(np.sqrt(np.sum(dv * dv))), rel_tol=1e-15)
    r2 = ov.sweep(P, w, sc.v0, norm=ov.NORM_RMS)
    assert math.isclose(r2.theta, r.theta / math.sqrt(P.n), rel_tol=1e-15)


def test_solve_counts_iterations_like_alg1(rng):
    sc = scenes.random_problem(rng, 8, 2)
    P = oracle_problem(sc)
    w = ov.frobenius_w(P)
    r = ov.solve(P, w, sc.v0, theta_th=0.0, l_max=7)
    assert r.iters == 7 and len(r.thetas) == 7 and not r.converged
    r = ov.solve(P, w, sc.v0, theta_th=1e300, l_max=7)
    assert r.iters == 1 and r.converged
    r1 = ov.solve(P, w, sc.v0, theta_th=0.0, l_max=1)
    assert np.array_equal(r1.v, ov.sweep(P, w, sc.v0).v_next)


def textbook_two_body(mi, mj, vi, vj, R, mu, phi):
    """Two point masses meeting at a contact with frame ``R`` (normal from j to i):
    relative velocity ``u = R (v_i - v_j) + phi e_n``, effective mass
    ``m_i m_j / (m_i + m_j)``, Coulomb's law, equal and opposite impulses."""
    me = mi * mj / (mi + mj)
    u = R @ (vi - vj)
    u[0] += phi
    if u[0] >= 0.0:
        lam = np.zeros(3)
    else:
        ln = -me * u[0]
        ut = u[1:]
        lt = -me * ut if me * np.linalg.norm(ut) <= mu * ln else -mu * ln * ut / np.linalg.norm(ut)
        lam = np.concatenate([[ln], lt])
    return vi + R.T @ lam / mi, vj - R.T @ lam / mj, lam


@pytest.mark.parametrize("equal", [True, False])
def test_two_point_masses_d_contact_match_textbook_impact(rng, equal):
    """D-contact (eq. jcnode with +R on node i and -R on node j) between two free
    point masses reproduces the textbook two-body impact with friction; with
    equal masses the tied W equals A^{-1} and one sweep suffices."""
    modes = set()
    for q in range(24):
        mi = rng.uniform(0.5, 2.0)
        mj = mi if equal else rng.uniform(0.5, 2.0)
        R = scenes.random_rotations(rng, 1)[0]
        mu = rng.uniform(0.2, 1.0)
        phi = rng.uniform(-0.2, 0.2)
        vi, vj = rng.normal(0, 1, 3), rng.normal(0, 1, 3)
        b = np.concatenate([mi * vi, mj * vj])
        vals = np.array([mi * np.eye(3), mj * np.eye(3)])
        P = ov.make_problem(np.arange(3), np.arange(2), vals, b, [0], [1], R[None], [mu], [phi])
        w = ov.frobenius_w(P)
        ri, rj, lam = textbook_two_body(mi, mj, vi, vj, R, mu, phi)
        modes.add(int(mode_of(lam[None], np.array([mu]))[0]) if np.any(lam) else 0)
        if equal:
            r = ov.sweep(P, w, np.zeros(6))
        else:
            r = ov.solve(P, w, np.zeros(6), theta_th=1e-15, l_max=100000)
            assert r.converged
        v = r.v_next if equal else r.v
        assert np.allclose(v, np.concatenate([ri, rj]), rtol=1e-10, atol=1e-10)
        assert np.allclose(r.lam[0], lam, rtol=1e-9, atol=1e-10)
    assert modes == {0, 1, 2}


def test_gamma_blocks_are_the_dense_product_for_any_diagonal_w(rng):
    """Gamma_{c,m} = J_{c,m} W J_{c,m}^T (eq. subp) for an untied diagonal W too."""
    sc = scenes.random_problem(rng, 9, 3, d_contacts=2)
    P = oracle_problem(sc)
    w = rng.uniform(0.1, 2.0, P.n)
    J = P.Jc.toarray()
    Gam = J @ np.diag(w) @ J.T
    assert np.allclose(ov.gamma_blocks(P, w), [Gam[3 * m:3 * m + 3, 3 * m:3 * m + 3]
                                               for m in range(P.n_c)], atol=1e-14)


# ----------------------------------------------------------------------------
# converged V-FPI against independent solvers
# ----------------------------------------------------------------------------

def _converged(P, w, v0):
    r = ov.solve(P, w, v0, theta_th=1e-13, l_max=200000)
    assert r.converged
    return r


@pytest.mark.parametrize("seed", range(6))
def test_fixed_point_consistency_and_pgs_agreement(seed):
    """Consistency remark: the fixed point satisfies A v = b + J^T lambda and
    eq. (scc); it agrees with projected Gauss-Seidel on the Delassus operator."""
    rng = np.random.default_rng(100 + seed)
    sc = scenes.random_problem(rng, 10, 4, mu_range=(0.1, 0.6), couple=0.3)
    P = oracle_problem(sc)
    w = ov.frobenius_w(P)
    r = _converged(P, w, sc.v0)
    assert dynamics_residual(P, r.v, r.lam) < 1e-10
    assert scc_residual(P, r.v, r.lam) < 1e-10
    v_pgs, lam_pgs, _ = pgs(P)
    assert scc_residual(P, v_pgs, lam_pgs) < 1e-10
    assert dynamics_residual(P, v_pgs, lam_pgs) < 1e-12
    assert np.linalg.norm(r.v - v_pgs) <= 1e-8 * np.linalg.norm(v_pgs)


# seeds chosen to cover open, stick+slip, slip+slip, stick+stick and mixed triples
@pytest.mark.parametrize("n_c,seed", [(1, 0), (1, 1), (2, 2), (2, 4), (2, 17), (2, 52),
                                      (3, 4), (3, 12), (3, 21), (3, 29), (3, 73)])
def test_fixed_point_is_in_enumerated_scc_set(n_c, seed):
    """Brute force: the V-FPI fixed point is one of the exhaustively enumerated
    open/stick/slip solutions of eq. (scc)."""
    rng = np.random.default_rng(200 + seed)
    sc = scenes.random_problem(rng, 5, n_c, mu_range=(0.2, 0.9), couple=0.5, phi_scale=1.0)
    P = oracle_problem(sc)
    w = ov.frobenius_w(P)
    r = _converged(P, w, sc.v0)
    sols = enumerate_scc(P)
    assert sols, "enumeration found no SCC solution"
    err = min(np.linalg.norm(s["v"] - r.v) / np.linalg.norm(s["v"]) for s in sols)
    assert err < 1e-7
    for s in sols:
        assert scc_residual(P, s["v"], s["lam"]) < 1e-7


def test_enumeration_reproduces_textbook_single_contact(rng):
    for m, b, R, mu, phi, mode in single_node_cases(rng):
        P = point_masses([m], b, R[None], [mu], [phi], [0])
        v_ref, lam_ref, _ = textbook_point_contact(m, b, R, mu, phi)
        sols = enumerate_scc(P)
        assert len(sols) == 1
        assert np.allclose(sols[0]["v"], v_ref, rtol=1e-9, atol=1e-12)
        assert sols[0]["modes"] == ({"open": 0, "stick": 1, "slip": 2}[mode],)


def test_small_lattice_converges_and_matches_pgs():
    """6x6x6 lattice on the ground (648 DOF, 36 contacts, FP64)."""
    sc = scenes.small_lattice()
    P = oracle_problem(sc)
    w = ov.frobenius_w(P)
    A = P.A.toarray()
    rho = np.abs(np.linalg.eigvals(np.eye(P.n) - np.diag(w) @ A)).max()
    assert rho < 1.0
    r = ov.solve(P, w, sc.v0, theta_th=1e-14, l_max=100000)
    assert r.converged
    assert dynamics_residual(P, r.v, r.lam) < 1e-9
    assert scc_residual(P, r.v, r.lam) < 1e-9
    v_pgs, lam_pgs, _ = pgs(P, tol=1e-13)
    assert np.linalg.norm(r.v - v_pgs) <= 1e-7 * np.linalg.norm(v_pgs)
    modes = mode_of(r.lam, P.mu)
    assert (modes > 0).sum() > 0


# ----------------------------------------------------------------------------
# adjoint
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("seed", range(4))
def test_dense_adjoint_matches_central_differences(seed):
    """Implicit-function adjoint vs central differences of the converged solve,
    on problems whose active set does not change under the perturbation."""
    rng = np.random.default_rng(300 + seed)
    sc = scenes.random_problem(rng, 8, 3, mu_range=(0.2, 0.8), couple=0.3, phi_scale=1.0)
    P = oracle_problem(sc)
    w = ov.frobenius_w(P)
    base = _converged(P, w, sc.v0)
    c = rng.normal(0, 1, P.n)
    g_b, g_phi, g_mu, _ = adjoint(P, w, base.v, c)
    eps = 1e-6
    modes0 = mode_of(base.lam, P.mu)

    def loss_with(field, k, delta):
        import copy
        Q = copy.copy(P)
        arr = getattr(P, field).copy()
        arr[k] += delta
        setattr(Q, field, arr)
        r = _converged(Q, w, base.v)
        assert np.array_equal(mode_of(r.lam, Q.mu), modes0)
        return c @ r.v

    for k in rng.permutation(P.n)[:6]:
        fd = (loss_with("b", k, eps) - loss_with("b", k, -eps)) / (2 * eps)
        assert abs(fd - g_b[k]) <= 1e-6 * max(1.0, abs(fd))
    for m in range(P.n_c):
        fd = (loss_with("phi", m, eps) - loss_with("phi", m, -eps)) / (2 * eps)
        assert abs(fd - g_phi[m]) <= 1e-6 * max(1.0, abs(fd))
        fd = (loss_with("mu", m, eps) - loss_with("mu", m, -eps)) / (2 * eps)
        assert abs(fd - g_mu[m]) <= 1e-6 * max(1.0, abs(fd))


def test_integrate_is_explicit_position_update(rng):
    x = rng.normal(0, 1, 30)
    v = rng.normal(0, 1, 30)
    assert np.array_equal(ov.integrate(x, v, 1e-3), x + 1e-3 * v)


def test_without_contacts_the_fixed_point_is_the_linear_solve():
    """With no contact the V-FPI fixed point of eq. (pgd1) is v = A^{-1} b
    (W is positive and diagonal): Alg. 1 must reach the direct solution, for
    the Frobenius W and for W = alpha I with alpha below 2 / lambda_max(A)."""
    from paper_2201_09212_gb300 import scenes
    from tests.conftest import oracle_problem
    sc = scenes.random_problem(np.random.default_rng(41), 40, 0, density=0.1, couple=0.5)
    P = oracle_problem(sc)
    x = np.linalg.solve(P.A.toarray(), P.b)
    for w in (ov.frobenius_w(P), np.full(P.n, 1.0 / np.linalg.eigvalsh(P.A.toarray()).max())):
        r = ov.solve(P, w, sc.v0, theta_th=1e-13, l_max=100000)
        assert r.converged
        assert np.linalg.norm(r.v - x) <= 1e-11 * np.linalg.norm(x)
