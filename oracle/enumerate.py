"""Brute-force active-set enumeration of eq. (scc) for 1-3 contacts
(test infrastructure only).

Every assignment of the three cases of Fig. complementarity -- open, stick,
slip -- is solved directly in impulse space, ``u = G lambda + c + phi e_n``
with the dense Delassus operator of eq. (delassus):

* open:  ``lambda_m = 0``, then require ``u_n >= 0``;
* stick: ``u_m = 0``, then require ``lambda_n >= 0`` and ``||lambda_t|| <= mu lambda_n``;
* slip:  ``u_n = 0`` and ``u_t = -s lambda_t`` with a slip parameter ``s > 0``
  (friction opposes sliding, third line of eq. scc), then require
  ``||lambda_t|| = mu lambda_n`` -- a scalar equation per slipping contact,
  solved for ``s`` by a grid scan plus root polishing.

For fixed ``s`` each assignment is a square linear system, so the search is
exhaustive over the assignments and over the grid of ``s``.  The result is the
set of SCC solutions (``v``, ``lambda``) found; V-FPI's fixed point must lie in
it.
"""
from __future__ import annotations

import itertools

import numpy as np
import scipy.linalg as sla
import scipy.optimize as so

from .delassus import delassus

OPEN, STICK, SLIP = 0, 1, 2


def _system(G, cp, modes, s_vals):
    n3 = G.shape[0]
    M = np.zeros((n3, n3))
    r = np.zeros(n3)
    k = 0
    for m, mode in enumerate(modes):
        a = 3 * m
        if mode == OPEN:
            M[a:a + 3, a:a + 3] = np.eye(3)
        elif mode == STICK:
            M[a:a + 3] = G[a:a + 3]
            r[a:a + 3] = -cp[a:a + 3]
        else:
            M[a:a + 3] = G[a:a + 3]
            M[a + 1, a + 1] += s_vals[k]
            M[a + 2, a + 2] += s_vals[k]
            r[a:a + 3] = -cp[a:a + 3]
            k += 1
    return M, r


def _lam(G, cp, modes, s_vals):
    M, r = _system(G, cp, modes, s_vals)
    return np.linalg.solve(M, r)


def _cone_gap(lam, mu, slips):
    lam = lam.reshape(-1, 3)
    return np.array([np.hypot(lam[m, 1], lam[m, 2]) - mu[m] * lam[m, 0] for m in slips])


def _feasible(lam, u, mu, modes, tol):
    lam = lam.reshape(-1, 3)
    u = u.reshape(-1, 3)
    Ls = max(np.abs(lam).max(), 1e-300)
    Us = max(np.abs(u).max(), 1e-300)
    for m, mode in enumerate(modes):
        lt = np.hypot(lam[m, 1], lam[m, 2])
        if mode == OPEN:
            if u[m, 0] < -tol * Us:
                return False
        elif mode == STICK:
            if lam[m, 0] < -tol * Ls or lt > mu[m] * lam[m, 0] + tol * Ls:
                return False
        else:
            if lam[m, 0] < -tol * Ls or abs(lt - mu[m] * lam[m, 0]) > tol * Ls:
                return False
            # sliding must oppose the friction impulse: u_t . lambda_t <= 0
            if u[m, 1] * lam[m, 1] + u[m, 2] * lam[m, 2] > tol * Ls * Us:
                return False
    return True


def enumerate_scc(P, tol: float = 1e-8, grid: int | None = None):
    """All SCC solutions found; list of dicts with ``v``, ``lam``, ``modes``."""
    G, c, chol = delassus(P)
    cp = c.copy()
    cp[0::3] += P.phi
    n_c = P.n_c
    assert 1 <= n_c <= 3, "brute force is for 1-3 contacts"
    s_scale = float(np.mean(np.diag(G)))
    sols = []

    def add(lam, modes):
        u = G @ lam + cp
        if not _feasible(lam, u, P.mu, modes, tol):
            return
        for q in sols:
            if np.abs(q["lam"].ravel() - lam).max() <= 1e-7 * max(np.abs(lam).max(), 1e-300):
                return
        v = sla.cho_solve(chol, P.b + P.Jc.T @ lam)
        sols.append(dict(v=v, lam=lam.reshape(-1, 3).copy(), modes=tuple(modes)))

    for modes in itertools.product((OPEN, STICK, SLIP), repeat=n_c):
        slips = [m for m in range(n_c) if modes[m] == SLIP]
        ns = len(slips)
        if ns == 0:
            try:
                add(_lam(G, cp, modes, []), modes)
            except np.linalg.LinAlgError:
                pass
            continue

        def F(tau):
            s = s_scale * np.exp(np.clip(tau, -60.0, 60.0))
            lam = _lam(G, cp, modes, s)
            return _cone_gap(lam, P.mu, slips) / max(np.abs(lam).max(), 1e-300)

        k = grid or {1: 400, 2: 48, 3: 16}[ns]
        axis = np.linspace(np.log(1e-8), np.log(1e8), k)
        pts = np.array(list(itertools.product(axis, repeat=ns)))
        vals = []
        for p in pts:
            try:
                vals.append(F(p))
            except np.linalg.LinAlgError:
                vals.append(np.full(ns, np.inf))
        vals = np.array(vals)
        starts = []
        if ns == 1:
            f = vals[:, 0]
            for q in range(k - 1):
                if np.isfinite(f[q]) and np.isfinite(f[q + 1]) and f[q] * f[q + 1] <= 0:
                    try:
                        t = so.brentq(lambda x: F(np.array([x]))[0], axis[q], axis[q + 1],
                                      xtol=1e-14, rtol=1e-14, maxiter=400)
                        starts.append(np.array([t]))
                    except ValueError:
                        pass
        else:
            order = np.argsort(np.linalg.norm(vals, axis=1))
            starts = [pts[q] for q in order[:40]]
        for t0 in starts:
            if ns > 1:
                sol = so.root(F, t0, method="hybr", options=dict(xtol=1e-14))
                if not sol.success or np.abs(F(sol.x)).max() > 1e-9:
                    continue
                t0 = sol.x
            s = s_scale * np.exp(t0)
            try:
                add(_lam(G, cp, modes, s), modes)
            except np.linalg.LinAlgError:
                pass
    return sols
