"""Dense implicit-function adjoint of the V-FPI fixed point (test infrastructure only).

The V-FPI map of Sec. IV is ``f(v) = v* + W J_c^T lambda_c(v*)`` with
``v* = (I - W A) v + W b`` and ``lambda_c = ProjectFC(-Gamma_c^{-1}(J_c v* + phi))``
(Alg. 2).  Holding the active set of the projection fixed at the converged
point, ``df/dv = (I - S)(I - W A)`` with
``S = W J_c^T diag(P'_m Gamma_m^{-1}) J_c`` and ``P'_m`` the Jacobian of the
strict operator (eq. operator) at ``lambda*_m``.  The fixed point ``v = f(v)``
then gives, for a loss ``L(v)`` with ``g_v = dL/dv``,
``(I - D)^T g_bar = g_v`` and

* ``dL/db = W (I - S)^T g_bar``
* ``dL/dphi_m = -g_bar^T W J_m^T P'_m Gamma_m^{-1} e_n``
* ``dL/dmu_m = g_bar^T W J_m^T dProjectFC/dmu``.

The paper gives the map and, in Lemma 2, the slip derivative
``||d lambda_t / d lambda*_n|| = mu``; the implicit-function step is standard
calculus on that map.  Dense: small problems only.
"""
from __future__ import annotations

import numpy as np

from .vfpi import PROXIMAL, STRICT, gamma_blocks, sweep


def strict_jacobian(lam_star: np.ndarray, mu: float):
    """``(P', dP/dmu)`` of the strict operator at one ``lambda*`` (3-vector).

    open (``lambda*_n <= 0``): zero.  stick (``||lambda*_t|| <= mu lambda*_n``):
    identity.  slip: ``dlambda_n/dlambda*_n = 1``,
    ``dlambda_t/dlambda*_n = mu t``, ``dlambda_t/dlambda*_t = (mu lambda_n / rho)(I - t t^T)``
    with ``rho = ||lambda*_t||``, ``t = lambda*_t / rho``; ``dlambda_t/dmu = lambda_n t``.
    """
    ln = float(lam_star[0])
    Pp = np.zeros((3, 3))
    dmu = np.zeros(3)
    if ln <= 0.0:
        return Pp, dmu
    rho = float(np.hypot(lam_star[1], lam_star[2]))
    if rho <= mu * ln:
        return np.eye(3), dmu
    t = np.asarray(lam_star[1:], dtype=np.float64) / rho
    Pp[0, 0] = 1.0
    Pp[1:, 0] = mu * t
    Pp[1:, 1:] = (mu * ln / rho) * (np.eye(2) - np.outer(t, t))
    dmu[1:] = ln * t
    return Pp, dmu


def proximal_jacobian(lam_star: np.ndarray, mu: float):
    """``(P', dP/dmu)`` of the proximal operator (Euclidean projection onto the
    friction cone, eq. operator) at one ``lambda*``.  Inside the cone: identity;
    in its polar cone: zero; otherwise, with ``r = ||lambda*_t||``, ``t = lambda*_t / r``
    and ``lambda_n = (lambda*_n + mu r) / (1 + mu^2)``:
    ``dlambda_n = (d lambda*_n + mu t . d lambda*_t) / (1 + mu^2)``,
    ``dlambda_t = mu t dlambda_n + mu (lambda_n / r)(I - t t^T) d lambda*_t``."""
    a = float(lam_star[0])
    r = float(np.hypot(lam_star[1], lam_star[2]))
    Pp = np.zeros((3, 3))
    dmu = np.zeros(3)
    if r <= mu * a:
        return np.eye(3), dmu
    if mu * r <= -a:
        return Pp, dmu
    t = np.asarray(lam_star[1:], dtype=np.float64) / r
    k = 1.0 + mu * mu
    ln = (a + mu * r) / k
    dln = np.concatenate([[1.0], mu * t]) / k                     # d lambda_n / d lambda*
    Pp[0] = dln
    Pp[1:] = mu * np.outer(t, dln)
    Pp[1:, 1:] += mu * (ln / r) * (np.eye(2) - np.outer(t, t))
    dln_dmu = (r * k - 2.0 * mu * (a + mu * r)) / (k * k)
    dmu[0] = dln_dmu
    dmu[1:] = (ln + mu * dln_dmu) * t
    return Pp, dmu


def adjoint(P, w: np.ndarray, v: np.ndarray, g_v: np.ndarray, operator: str = STRICT,
            omega: np.ndarray | None = None):
    """Dense adjoint at the converged ``v``; returns ``(g_b, g_phi, g_mu, g_bar)``.
    ``omega`` ([n_c] scalars, the regularisation ``Omega_m = omega_m I`` of
    eq. invt) enters through ``Gamma_m + Omega_m``."""
    om = None if omega is None else np.asarray(omega, float)[:, None, None] * np.eye(3)
    r = sweep(P, w, v, operator, omega=om)
    n = P.n
    Gam = gamma_blocks(P, w)
    if om is not None:
        Gam = Gam + om
    n_c = P.n_c
    B = np.zeros((3 * n_c, 3 * n_c))
    dmu = np.zeros((n_c, 3))
    jac = strict_jacobian if operator == STRICT else proximal_jacobian
    for m in range(n_c):
        Pp, dm = jac(r.lam_star[m], P.mu[m])
        B[3 * m:3 * m + 3, 3 * m:3 * m + 3] = Pp @ np.linalg.inv(Gam[m])
        dmu[m] = dm
    J = P.Jc.toarray()
    W = np.diag(w)
    A = P.A.toarray()
    S = W @ J.T @ B @ J
    D = (np.eye(n) - S) @ (np.eye(n) - W @ A)
    g_bar = np.linalg.solve((np.eye(n) - D).T, np.asarray(g_v, dtype=np.float64))
    g_b = W @ (np.eye(n) - S).T @ g_bar
    WJT = W @ J.T                                   # n x 3n_c
    h = WJT.T @ g_bar                               # 3n_c: J W g_bar
    g_phi = np.array([-(h[3 * m:3 * m + 3] @ B[3 * m:3 * m + 3, 3 * m]) for m in range(n_c)])
    g_mu = np.array([h[3 * m:3 * m + 3] @ dmu[m] for m in range(n_c)])
    return g_b, g_phi, g_mu, g_bar
