"""Projected Gauss-Seidel on the dense Delassus operator (test infrastructure only).

This is the impulse-space fixed-point iteration (I-FPI) the paper compares
against (Sec. V.C, baselines; eq. delassus): factor ``A``, form
``G = J_c A^{-1} J_c^T`` and ``c = J_c A^{-1} b``, then sweep the contacts in
order, replacing ``lambda_m`` by ``ProjectFC(lambda_m - u_m / g_m)`` with
``u_m = sum_k G_mk lambda_k + c_m + phi_m e_n`` and the scalar
``g_m = lambda_max(G_mm)``.  Any fixed point of that map satisfies eq. (scc)
(the argument of Prop. 4 applies unchanged to a scalar step), so it is an
independent route to the same solution set as V-FPI.  Dense: small problems
only.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

from .vfpi import project_proximal, project_strict


def delassus(P):
    """``(G, c, chol)`` with ``G = J A^{-1} J^T``, ``c = J A^{-1} b`` (eq. delassus)."""
    A = P.A.toarray()
    chol = sla.cho_factor(A)
    J = P.Jc.toarray()
    AinvJT = sla.cho_solve(chol, J.T)
    G = J @ AinvJT
    c = J @ sla.cho_solve(chol, P.b)
    return G, c, chol


def pgs(P, tol: float = 1e-14, max_sweeps: int = 200000, relax: float = 1.0):
    """Projected Gauss-Seidel; returns ``(v, lambda [n_c, 3], sweeps)``."""
    G, c, chol = delassus(P)
    n_c = P.n_c
    g = np.array([np.linalg.eigvalsh(G[3 * m:3 * m + 3, 3 * m:3 * m + 3]).max()
                  for m in range(n_c)])
    lam = np.zeros(3 * n_c)
    phi_vec = np.zeros(3 * n_c)
    phi_vec[0::3] = P.phi
    sweeps = 0
    for sweeps in range(1, max_sweeps + 1):
        change = 0.0
        scale = 0.0
        for m in range(n_c):
            s = slice(3 * m, 3 * m + 3)
            u = G[s] @ lam + c[s] + phi_vec[s]
            new = project_strict(lam[s] - relax * u / g[m], P.mu[m:m + 1])[0]
            change = max(change, float(np.abs(new - lam[s]).max()))
            lam[s] = new
            scale = max(scale, float(np.abs(new).max()))
        if change <= tol * max(scale, 1e-300):
            break
    v = sla.cho_solve(chol, P.b + P.Jc.T @ lam)
    return v, lam.reshape(-1, 3), sweeps


def ccp_apgd(P, omega=None, iters: int = 200000, tol: float = 1e-15):
    """The convex contact problem (eq. ccp, with eq. invt's regularisation):
    ``min 1/2 lambda^T (G + Omega) lambda + lambda^T (c + phi e_n)`` over the
    product of friction cones, by accelerated projected gradient (Nesterov /
    FISTA with the Euclidean cone projection and step 1 / L, L the largest
    eigenvalue of G + Omega).  Returns ``(v, lambda [n_c, 3], iterations)``."""
    G, c, chol = delassus(P)
    n_c = P.n_c
    H = G.copy()
    if omega is not None:
        H += np.kron(np.diag(np.asarray(omega, float)), np.eye(3))
    q = c.copy()
    q[0::3] += P.phi
    L = np.linalg.eigvalsh(H).max()
    lam = np.zeros(3 * n_c)
    y = lam.copy()
    tk = 1.0
    it = 0
    for it in range(1, iters + 1):
        new = project_proximal(y - (H @ y + q) / L, P.mu).ravel()
        tk1 = 0.5 * (1.0 + np.sqrt(1.0 + 4.0 * tk * tk))
        y = new + ((tk - 1.0) / tk1) * (new - lam)
        done = np.abs(new - lam).max() <= tol * max(np.abs(new).max(), 1e-300)
        lam, tk = new, tk1
        if done:
            break
    v = sla.cho_solve(chol, P.b + P.Jc.T @ lam)
    return v, lam.reshape(-1, 3), it


def pgs_general(A, b, J, mu, phi, tol: float = 1e-14, max_sweeps: int = 200000):
    """Projected Gauss-Seidel for ``A v = b + J^T lambda`` with an arbitrary
    (not nodal) contact Jacobian ``J`` [3 n_c x n]: the original contact problem
    that virtual nodes stand in for (Sec. III.A).  Dense."""
    A = np.asarray(A, float)
    J = np.asarray(J, float)
    chol = sla.cho_factor(A)
    G = J @ sla.cho_solve(chol, J.T)
    c = J @ sla.cho_solve(chol, np.asarray(b, float))
    n_c = J.shape[0] // 3
    mu = np.asarray(mu, float)
    g = np.array([np.linalg.eigvalsh(G[3 * m:3 * m + 3, 3 * m:3 * m + 3]).max() for m in range(n_c)])
    lam = np.zeros(3 * n_c)
    ph = np.zeros(3 * n_c)
    ph[0::3] = phi
    for _ in range(max_sweeps):
        change = scale = 0.0
        for m in range(n_c):
            s = slice(3 * m, 3 * m + 3)
            u = G[s] @ lam + c[s] + ph[s]
            new = project_strict(lam[s] - u / g[m], mu[m:m + 1])[0]
            change = max(change, float(np.abs(new - lam[s]).max()))
            lam[s] = new
            scale = max(scale, float(np.abs(new).max()))
        if change <= tol * max(scale, 1e-300):
            break
    v = sla.cho_solve(chol, np.asarray(b, float) + J.T @ lam)
    return v, lam.reshape(-1, 3)
