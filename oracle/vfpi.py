"""Plain FP64 V-FPI (Alg. 1 with Alg. 2), written out in the paper's order.

Test infrastructure only (see the package docstring).

Notation follows the paper: ``A v = b + J_c^T lambda_c`` (eq. lindyn), nodal
contact Jacobian rows ``J_{c,m} = [.. R_m .. -R_m ..]`` (eq. jcnode, the ``-R``
block only for a D-contact), diagonal step matrix ``W``, surrogate step
``v* = v - W (A v - b)`` (eq. pgd1), surrogate contact problem
``lambda_c = SOL(eta_c, Gamma_c)`` with ``Gamma_c = J_c W J_c^T`` and
``eta_c = J_c v*`` (eq. subp), one-shot solve (Alg. 2, eq. operator) and update
``v^{l+1} = v* + W J_c^T lambda_c`` (eq. vup).  The residual
``theta = ||v^{l+1} - v^l||`` and the stop test follow Alg. 1.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
import scipy.sparse as sp

STRICT = "strict"
PROXIMAL = "proximal"
NORM_ABS = "abs"      # theta = ||dv||_2 (Alg. 1)
NORM_RMS = "rms"      # theta = ||dv||_2 / sqrt(n)


@dataclasses.dataclass
class Problem:
    """The data of one V-FPI problem, promoted to float64."""

    A: sp.spmatrix            # n x n, SPD
    b: np.ndarray             # [n]
    node_i: np.ndarray        # [n_c]
    node_j: np.ndarray        # [n_c], -1 for an S-contact
    R: np.ndarray             # [n_c, 3, 3], rows n, t1, t2
    mu: np.ndarray            # [n_c]
    phi: np.ndarray           # [n_c]
    Jc: sp.spmatrix           # 3 n_c x n, eq. (jcnode)

    @property
    def n(self) -> int:
        return self.A.shape[0]

    @property
    def n_c(self) -> int:
        return self.node_i.shape[0]


def make_problem(row_ptr, col_idx, vals, b, node_i, node_j, R, mu, phi) -> Problem:
    """Assemble ``A`` (BSR, 3x3 blocks) and ``J_c`` (eq. jcnode) in float64."""
    vals = np.asarray(vals, dtype=np.float64).reshape(-1, 3, 3)
    N = len(row_ptr) - 1
    A = sp.bsr_matrix((vals, np.asarray(col_idx), np.asarray(row_ptr)), shape=(3 * N, 3 * N))
    node_i = np.asarray(node_i, dtype=np.int64)
    node_j = np.asarray(node_j, dtype=np.int64)
    R = np.asarray(R, dtype=np.float64).reshape(-1, 3, 3)
    n_c = node_i.shape[0]
    rows, cols, data = [], [], []
    for sign, nodes, keep in ((1.0, node_i, np.ones(n_c, bool)), (-1.0, node_j, node_j >= 0)):
        m = np.nonzero(keep)[0]
        r = 3 * m[:, None, None] + np.arange(3)[None, :, None]
        c = 3 * nodes[m][:, None, None] + np.arange(3)[None, None, :]
        rows.append(np.broadcast_to(r, (len(m), 3, 3)).ravel())
        cols.append(np.broadcast_to(c, (len(m), 3, 3)).ravel())
        data.append((sign * R[m]).ravel())
    Jc = sp.csr_matrix((np.concatenate(data), (np.concatenate(rows), np.concatenate(cols))),
                       shape=(3 * n_c, 3 * N))
    return Problem(A=A, b=np.asarray(b, dtype=np.float64).copy(), node_i=node_i, node_j=node_j,
                   R=R, mu=np.asarray(mu, dtype=np.float64).copy(),
                   phi=np.asarray(phi, dtype=np.float64).copy(), Jc=Jc)


# ----------------------------------------------------------------------------
# Choice of W (Sec. IV.C)
# ----------------------------------------------------------------------------

def frobenius_w(P: Problem) -> np.ndarray:
    """Diagonal W minimising ``||I - W A||_F`` under the tying of Prop. 3.

    Row by row, ``||I - W A||_F^2 = sum_r (1 - 2 w_r a_rr + w_r^2 ||A_r*||^2)``,
    so a group of DOFs sharing one value ``w`` takes
    ``w = sum a_rr / sum ||A_r*||^2`` (Sec. IV.C; the three DOFs of a node in
    contact form one group, the six DOFs of a D-contact's two nodes form one
    group) and every other DOF takes ``w_rr = a_rr / ||A_r*||^2``.
    """
    A = P.A.tocsr()
    d = A.diagonal().astype(np.float64)
    s = np.asarray(A.multiply(A).sum(axis=1)).ravel()
    w = d / s
    for m in range(P.n_c):
        nodes = [P.node_i[m]] + ([P.node_j[m]] if P.node_j[m] >= 0 else [])
        dofs = np.concatenate([np.arange(3 * q, 3 * q + 3) for q in nodes])
        w[dofs] = d[dofs].sum() / s[dofs].sum()
    return w


def scalar_w(P: Problem, alpha: float) -> np.ndarray:
    """``W = alpha I`` (Sec. IV.C)."""
    return np.full(P.n, float(alpha))


def optimal_alpha(P: Problem) -> float:
    """``alpha = 2 / (sigma_min(A) + sigma_max(A))`` (Sec. IV.C), dense eigenvalues."""
    ev = np.linalg.eigvalsh(P.A.toarray())
    return 2.0 / (ev[0] + ev[-1])


# ----------------------------------------------------------------------------
# ProjectFC (eq. operator)
# ----------------------------------------------------------------------------

def project_strict(lam_star: np.ndarray, mu: np.ndarray) -> np.ndarray:
    """Strict operator: ``lambda_n = max(lambda*_n, 0)``, then the tangential part
    is projected onto the disk of radius ``mu lambda_n`` (the cross-section of the
    friction cone at ``lambda_n``)."""
    lam_star = np.asarray(lam_star, dtype=np.float64).reshape(-1, 3)
    lam = np.empty_like(lam_star)
    lam[:, 0] = np.maximum(lam_star[:, 0], 0.0)
    t = lam_star[:, 1:]
    rho = np.sqrt(t[:, 0] ** 2 + t[:, 1] ** 2)
    radius = mu * lam[:, 0]
    inside = rho <= radius
    scale = np.where(inside, 1.0, radius / np.where(inside, 1.0, rho))
    lam[:, 1:] = t * scale[:, None]
    return lam


def project_strict_elliptic(lam_star: np.ndarray, mu1: np.ndarray, mu2: np.ndarray) -> np.ndarray:
    """Strict operator for the elliptic (anisotropic) cone
    ``lambda_n^2 >= lambda_t1^2 / mu1^2 + lambda_t2^2 / mu2^2`` (Sec. III.E):
    ``lambda_n = max(lambda*_n, 0)``, then ``lambda_t`` is the nearest point of
    the ellipse with semi-axes ``mu1 lambda_n, mu2 lambda_n`` -- the maximal
    dissipation solution (Prop. 6).  Outside the ellipse the nearest point is
    ``t_k = a_k^2 t*_k / (a_k^2 + nu)`` with the multiplier ``nu > 0`` the root
    of ``sum_k (a_k t*_k / (a_k^2 + nu))^2 = 1`` (found with brentq)."""
    import scipy.optimize as so
    lam_star = np.asarray(lam_star, dtype=np.float64).reshape(-1, 3)
    lam = np.zeros_like(lam_star)
    for m in range(lam_star.shape[0]):
        ln = max(lam_star[m, 0], 0.0)
        lam[m, 0] = ln
        t = lam_star[m, 1:]
        a = np.array([mu1[m], mu2[m]]) * ln
        if ln == 0.0 or not np.any(a > 0):
            continue
        if (t[0] / a[0]) ** 2 + (t[1] / a[1]) ** 2 <= 1.0:
            lam[m, 1:] = t
            continue
        g = lambda nu: np.sum((a * t / (a * a + nu)) ** 2) - 1.0
        hi = np.sqrt(np.sum(a * a)) * np.linalg.norm(t)
        nu = so.brentq(g, 0.0, hi, xtol=1e-300, rtol=4 * np.finfo(float).eps, maxiter=500)
        lam[m, 1:] = a * a * t / (a * a + nu)
    return lam


def project_proximal(lam_star: np.ndarray, mu: np.ndarray) -> np.ndarray:
    """Proximal operator: Euclidean projection onto the cone
    ``{lambda_n >= 0, ||lambda_t|| <= mu lambda_n}`` (eq. operator, eq. genfc)."""
    lam_star = np.asarray(lam_star, dtype=np.float64).reshape(-1, 3)
    a = lam_star[:, 0]
    t = lam_star[:, 1:]
    r = np.sqrt(t[:, 0] ** 2 + t[:, 1] ** 2)
    lam = np.zeros_like(lam_star)
    inside = r <= mu * a
    polar = mu * r <= -a
    edge = ~inside & ~polar
    lam[inside] = lam_star[inside]
    ln = (a[edge] + mu[edge] * r[edge]) / (1.0 + mu[edge] ** 2)
    lam[edge, 0] = ln
    lam[edge, 1:] = (mu[edge] * ln / r[edge])[:, None] * t[edge]
    return lam


# ----------------------------------------------------------------------------
# One sweep and the loop (Alg. 1, Alg. 2)
# ----------------------------------------------------------------------------

def gamma_blocks(P: Problem, w: np.ndarray) -> np.ndarray:
    """Diagonal 3x3 blocks ``Gamma_{c,m} = J_{c,m} W J_{c,m}^T`` of eq. (subp)."""
    G = np.zeros((P.n_c, 3, 3))
    for sign_nodes in (P.node_i, P.node_j):
        m = np.nonzero(sign_nodes >= 0)[0]
        Wn = w.reshape(-1, 3)[sign_nodes[m]]                   # [k, 3]
        G[m] += np.einsum("kab,kb,kcb->kac", P.R[m], Wn, P.R[m])
    return G


@dataclasses.dataclass
class SweepResult:
    v_next: np.ndarray
    v_star: np.ndarray
    eta: np.ndarray           # [n_c, 3]
    lam_star: np.ndarray      # [n_c, 3]
    lam: np.ndarray           # [n_c, 3]
    theta: float


def sweep(P: Problem, w: np.ndarray, v: np.ndarray, operator: str = STRICT,
          norm: str = NORM_ABS, omega: np.ndarray | None = None,
          mu2: np.ndarray | None = None) -> SweepResult:
    """One V-FPI iteration from ``v = v^l``.

    ``omega`` (optional, [n_c, 3, 3]) is added to ``Gamma_c`` as in the
    invertible-contact extension (eq. invt); ``mu2`` (optional, [n_c]) makes the
    friction cone elliptic with coefficients ``mu`` along t1 and ``mu2`` along t2
    (strict operator only, Prop. 6).
    """
    v = np.asarray(v, dtype=np.float64)
    # eq. (pgd1): gradient / surrogate-splitting step
    v_star = v - w * (P.A @ v - P.b)
    # eq. (subp): eta_c = J_c v*, Gamma_c = J_c W J_c^T (block diagonal, Prop. 3)
    eta = (P.Jc @ v_star).reshape(-1, 3)
    Gam = gamma_blocks(P, w)
    if omega is not None:
        Gam = Gam + omega
    # Alg. 2: lambda*_m = -Gamma_m^{-1} (eta_m + phi_m), phi_m = [phi_n; 0; 0]
    rhs = eta.copy()
    rhs[:, 0] += P.phi
    lam_star = -np.linalg.solve(Gam, rhs[:, :, None])[:, :, 0] if P.n_c else rhs
    if mu2 is not None:
        assert operator == STRICT
        lam = project_strict_elliptic(lam_star, P.mu, mu2)
    else:
        lam = (project_strict if operator == STRICT else project_proximal)(lam_star, P.mu)
    # eq. (vup): v^{l+1} = v* + W J_c^T lambda_c
    v_next = v_star + w * (P.Jc.T @ lam.ravel())
    dv = v_next - v
    theta = math.sqrt(math.fsum(dv * dv))
    if norm == NORM_RMS:
        theta /= math.sqrt(P.n)
    return SweepResult(v_next, v_star, eta, lam_star, lam, theta)


@dataclasses.dataclass
class SolveResult:
    v: np.ndarray
    lam: np.ndarray
    lam_star: np.ndarray
    iters: int
    theta: float
    converged: bool
    thetas: list


def solve(P: Problem, w: np.ndarray, v0: np.ndarray, theta_th: float, l_max: int,
          operator: str = STRICT, norm: str = NORM_ABS, omega=None, mu2=None) -> SolveResult:
    """Alg. 1 inner loop: sweep, residual, break on ``theta < theta_th`` or ``l = l_max``."""
    v = np.asarray(v0, dtype=np.float64).copy()
    thetas = []
    l = 1
    while True:
        r = sweep(P, w, v, operator, norm, omega, mu2)
        thetas.append(r.theta)
        if r.theta < theta_th or l == l_max:
            break
        v = r.v_next
        l += 1
    return SolveResult(r.v_next, r.lam, r.lam_star, l, r.theta, r.theta < theta_th, thetas)


def integrate(x: np.ndarray, v: np.ndarray, h: float) -> np.ndarray:
    """State update ``x_{k+1} = x_k + h v_hat`` (eq. disc_dyn, backward-Euler reading)."""
    return np.asarray(x, dtype=np.float64) + h * np.asarray(v, dtype=np.float64)


# ----------------------------------------------------------------------------
# Chebyshev acceleration (Alg. 3)
# ----------------------------------------------------------------------------

def chebyshev_nu(l: int, l_s: int, rho: float, nu_prev: float) -> float:
    """The weight nu_{l+1} of Alg. 3: 1 before the slow start ``l_s``,
    ``2 / (2 - rho^2)`` at ``l = l_s`` and ``4 / (4 - rho^2 nu_l)`` after."""
    if l < l_s:
        return 1.0
    if l == l_s:
        return 2.0 / (2.0 - rho * rho)
    return 4.0 / (4.0 - rho * rho * nu_prev)


def solve_chebyshev(P: Problem, w: np.ndarray, v0: np.ndarray, theta_th: float, l_max: int,
                    l_s: int = 10, u: float = 0.9, operator: str = STRICT,
                    norm: str = NORM_ABS, rho_fixed: float | None = None) -> SolveResult:
    """Alg. 3: the V-FPI step gives ``v**`` (eq. pgd1, Alg. 2, eq. vup); then
    ``v^{l+1} = nu (u (v** - v^l) + v^l - v^{l-1}) + v^{l-1}`` (eq. chebyup with
    the under-relaxation ``u`` of the text; ``u = 1`` is the printed update),
    ``theta = ||v^{l+1} - v^l||``, and after the stop test
    ``rho = min(||v^l - v^{l-1}|| / ||v^{l-1} - v^{l-2}||, 1)`` (eq. varrho, taken
    with the current l).  The loop starts from ``v^1`` (the warm start), so
    that ratio first exists after the stop test of ``l = 3`` and is first used
    by the weight of ``l = 4``: hence ``l_s >= 4``.  ``rho_fixed`` replaces the
    estimate by a given spectral radius (then ``l_s >= 2``)."""
    if l_s < (2 if rho_fixed is not None else 4):
        raise ValueError("l_s too small")
    v = np.asarray(v0, dtype=np.float64).copy()
    v_prev = v.copy()
    thetas, nu, rho = [], 1.0, (0.0 if rho_fixed is None else float(rho_fixed))
    l = 1
    while True:
        r = sweep(P, w, v, operator, norm)
        nu = chebyshev_nu(l, l_s, rho, nu)
        v_next = nu * (u * (r.v_next - v) + v - v_prev) + v_prev
        dv = v_next - v
        theta = math.sqrt(math.fsum(dv * dv))
        if norm == NORM_RMS:
            theta /= math.sqrt(P.n)
        thetas.append(theta)
        if theta < theta_th or l == l_max:
            break
        if l >= 3 and rho_fixed is None:
            rho = min(thetas[l - 2] / thetas[l - 3], 1.0) if thetas[l - 3] > 0 else 1.0
        v_prev, v = v, v_next
        l += 1
    return SolveResult(v_next, r.lam, r.lam_star, l, theta, theta < theta_th, thetas)


# ----------------------------------------------------------------------------
# Barzilai-Borwein step size (Sec. IV.C)
# ----------------------------------------------------------------------------

def bb_alpha(s: np.ndarray, z: np.ndarray, rule: str, alpha_prev: float) -> float:
    """``alpha_bb1 = s^T s / s^T z`` or ``alpha_bb2 = s^T z / z^T z`` with
    ``s = v^l - v^{l-1}`` and ``z = A s``; keeps the previous value when the
    quotient is not a positive finite number (curvature s^T z <= 0)."""
    ss = math.fsum(s * s)
    sz = math.fsum(s * z)
    zz = math.fsum(z * z)
    a = ss / sz if rule == "bb1" else (sz / zz if zz > 0 else float("nan"))
    return a if (sz > 0 and math.isfinite(a) and a > 0) else alpha_prev


def solve_bb(P: Problem, v0: np.ndarray, theta_th: float, l_max: int, alpha0: float,
             rule: str = "bb1", norm: str = NORM_ABS) -> SolveResult:
    """Alg. 1 with the step matrix re-determined every iteration as
    ``W = alpha_l I`` by the Barzilai-Borwein rule (``"bb1"``, ``"bb2"`` or
    ``"alt"``, alternating bb1 on odd and bb2 on even l); ``alpha_1 = alpha0``.
    A scalar W satisfies the tying of Prop. 3, so Alg. 2 stays one-shot."""
    v = np.asarray(v0, dtype=np.float64).copy()
    v_prev = r_prev = None
    alpha = float(alpha0)
    thetas = []
    l = 1
    while True:
        r_l = P.A @ v - P.b
        if v_prev is not None:
            this = rule if rule != "alt" else ("bb1" if l % 2 == 1 else "bb2")
            alpha = bb_alpha(v - v_prev, r_l - r_prev, this, alpha)
        res = sweep(P, np.full(P.n, alpha), v, STRICT, norm)
        thetas.append(res.theta)
        if res.theta < theta_th or l == l_max:
            break
        v_prev, r_prev, v = v, r_l, res.v_next
        l += 1
    return SolveResult(res.v_next, res.lam, res.lam_star, l, res.theta, res.theta < theta_th, thetas)
