"""Residual checkers (test infrastructure only).

``dynamics_residual`` measures eq. (lindyn); ``scc_residual`` measures the
Signorini-Coulomb conditions of eq. (scc) with the friction cone of eq. (genfc)
in a scaled, dimensionless form (the paper states the conditions but no
residual; the scaling below is this project's reading).
"""
from __future__ import annotations

import numpy as np


def contact_velocity(P, v: np.ndarray) -> np.ndarray:
    """``u_m = J_{c,m} v + phi_m e_n`` for every contact, shape [n_c, 3]."""
    u = (P.Jc @ np.asarray(v, dtype=np.float64)).reshape(-1, 3)
    u[:, 0] += P.phi
    return u


def dynamics_residual(P, v, lam) -> float:
    """``||A v - b - J_c^T lambda|| / ||b||`` (eq. lindyn)."""
    r = P.A @ v - P.b - P.Jc.T @ np.asarray(lam, dtype=np.float64).ravel()
    return float(np.linalg.norm(r) / max(np.linalg.norm(P.b), 1e-300))


def scc_terms(u: np.ndarray, lam: np.ndarray, mu: np.ndarray, v_scale: float):
    """Per-contact violations of eq. (scc), scaled by ``Lambda = max |lambda|``
    and ``V = v_scale``:

    * normal complementarity ``|min(lambda_n / Lambda, u_n / V)|``
    * cone feasibility ``max(0, ||lambda_t|| - mu lambda_n) / Lambda``
    * slip complementarity ``|min((mu lambda_n - ||lambda_t||) / Lambda, ||u_t|| / V)|``
    * maximal dissipation ``|| ||u_t|| lambda_t + ||lambda_t|| u_t || / (Lambda V)``
    """
    lam = np.asarray(lam, dtype=np.float64).reshape(-1, 3)
    u = np.asarray(u, dtype=np.float64).reshape(-1, 3)
    Lam = float(np.abs(lam).max()) if lam.size else 0.0
    V = max(float(v_scale), 1e-300)
    if Lam == 0.0:
        # all contacts open: only the gap condition remains
        return np.maximum(0.0, -u[:, 0] / V)[:, None]
    lt = np.linalg.norm(lam[:, 1:], axis=1)
    ut = np.linalg.norm(u[:, 1:], axis=1)
    t1 = np.abs(np.minimum(lam[:, 0] / Lam, u[:, 0] / V))
    t2 = np.maximum(0.0, lt - mu * lam[:, 0]) / Lam
    t3 = np.abs(np.minimum((mu * lam[:, 0] - lt) / Lam, ut / V))
    t4 = np.linalg.norm(ut[:, None] * lam[:, 1:] + lt[:, None] * u[:, 1:], axis=1) / (Lam * V)
    return np.stack([t1, t2, t3, t4], axis=1)


def scc_residual(P, v, lam) -> float:
    """Largest scaled violation of eq. (scc) over all contacts (0 for none)."""
    if P.n_c == 0:
        return 0.0
    u = contact_velocity(P, v)
    v_scale = max(np.abs(u).max(), np.abs(v).max())
    return float(scc_terms(u, lam, P.mu, v_scale).max())


def mode_of(lam: np.ndarray, mu: np.ndarray, rel: float = 1e-9) -> np.ndarray:
    """0 = open, 1 = stick, 2 = slip for each contact impulse (eq. scc cases)."""
    lam = np.asarray(lam).reshape(-1, 3)
    scale = max(np.abs(lam).max(), 1e-300)
    lt = np.linalg.norm(lam[:, 1:], axis=1)
    mode = np.where(lam[:, 0] <= rel * scale, 0, 1)
    mode = np.where((mode == 1) & (lt >= mu * lam[:, 0] * (1 - 1e-9)) & (lt > rel * scale), 2, mode)
    return mode
