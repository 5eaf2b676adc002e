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

from .vfpi import STRICT, gamma_blocks, sweep


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


def adjoint(P, w: np.ndarray, v: np.ndarray, g_v: np.ndarray):
    """Dense adjoint at the converged ``v``; returns ``(g_b, g_phi, g_mu, g_bar)``."""
    r = sweep(P, w, v, STRICT)
    n = P.n
    Gam = gamma_blocks(P, w)
    n_c = P.n_c
    B = np.zeros((3 * n_c, 3 * n_c))
    dmu = np.zeros((n_c, 3))
    for m in range(n_c):
        Pp, dm = strict_jacobian(r.lam_star[m], P.mu[m])
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
