"""Pins of the residual checkers (oracle/checks.py) on hand-built violations.

The Signorini-Coulomb conditions of eq. (scc), with the friction cone of
eq. (genfc), split into four cases that a solution must satisfy per contact:
a normal impulse only where the gap velocity is zero (``0 <= lambda_n _|_ u_n
>= 0``), an impulse inside the cone, the cone's boundary whenever the contact
slides, and a sliding friction that points against the sliding velocity
(maximal dissipation).  Each case below breaks exactly one of them (with
numbers chosen so that the scaled violation can be worked out by hand) and
checks that the checker reports it in its own column; valid open, stick and
slip contacts give zero.  The dynamics residual of eq. (lindyn) is checked on a
diagonal system against its hand value.

The functions are called through the module so that planted mistakes in it
(tests/test_oracle_mutants.py) are seen here.
"""
import math

import numpy as np

from oracle import checks as oc
from oracle import vfpi as ov

MU = 0.5
V_SCALE = 1.0

# (name, lambda = [n, t1, t2], u = [n, t1, t2], expected scaled terms [t1..t4])
# Lambda = max |lambda| = 2 over the whole set (the reference contacts), V = 1.
CASES = [
    # valid contacts: stick (inside the cone, no sliding), slip on the cone
    # boundary against the sliding direction, open (no impulse, separating)
    ("stick_ok", [2.0, 0.5, 0.0], [0.0, 0.0, 0.0], [0.0, 0.0, 0.0, 0.0]),
    ("slip_ok", [2.0, -0.6, -0.8], [0.0, 0.3, 0.4], [0.0, 0.0, 0.0, 0.0]),
    ("open_ok", [0.0, 0.0, 0.0], [0.7, 0.1, -0.2], [0.0, 0.0, 0.0, 0.0]),
    # penetration (u_n < 0) with no impulse: |min(0 / 2, -0.3 / 1)| = 0.3
    ("penetrating_free", [0.0, 0.0, 0.0], [-0.3, 0.0, 0.0], [0.3, 0.0, 0.0, 0.0]),
    # impulse on a separating contact: min(0.8 / 2, 0.25 / 1) = 0.25
    ("pulling_apart", [0.8, 0.0, 0.0], [0.25, 0.0, 0.0], [0.25, 0.0, 0.0, 0.0]),
    # outside the cone: ||lambda_t|| = 1 > mu lambda_n = 0.5 gives (1 - 0.5) / 2
    # for feasibility, and the slip-complementarity term |min(-0.25, 0)| too
    ("outside_cone", [1.0, 0.6, 0.8], [0.0, 0.0, 0.0], [0.0, 0.25, 0.25, 0.0]),
    # strictly inside the cone (0.2 < 1.0) while sliding at 0.5, friction
    # against the sliding: min((1.0 - 0.2) / 2, 0.5 / 1) = 0.4
    ("stick_while_sliding", [2.0, -0.12, -0.16], [0.0, 0.3, 0.4], [0.0, 0.0, 0.4, 0.0]),
    # on the boundary, sliding along t2 with friction along t1:
    # || 0.5 (1, 0) + 1 (0, 0.5) || / (2 * 1) = sqrt(0.5) / 2
    ("friction_sideways", [2.0, 1.0, 0.0], [0.0, 0.0, 0.5], [0.0, 0.0, 0.0, math.sqrt(0.5) / 2]),
    # on the boundary, friction along the sliding: || 0.5 (1, 0) + 1 (0.5, 0) || / 2
    ("friction_along_sliding", [2.0, 1.0, 0.0], [0.0, 0.5, 0.0], [0.0, 0.0, 0.0, 0.5]),
]


def _arrays(cases):
    lam = np.array([c[1] for c in cases], dtype=np.float64)
    u = np.array([c[2] for c in cases], dtype=np.float64)
    mu = np.full(len(cases), MU)
    return lam, u, mu


def test_scc_terms_flag_each_violation_in_its_column():
    lam, u, mu = _arrays(CASES)
    terms = oc.scc_terms(u, lam, mu, V_SCALE)
    assert terms.shape == (len(CASES), 4)
    for (name, _, _, want), got in zip(CASES, terms):
        assert np.allclose(got, want, rtol=1e-12, atol=1e-15), (name, got, want)


def _point_mass_problem(lam, u):
    """Independent unit point masses with S-contacts in the identity frame and
    no gap term, so that ``u_m = v_m``; ``b = v - lambda`` makes the dynamics
    exact, leaving only the contact conditions to check."""
    n_c = len(lam)
    vals = np.array([np.eye(3)] * n_c)
    b = (u - lam).ravel()
    return ov.make_problem(np.arange(n_c + 1), np.arange(n_c), vals, b, np.arange(n_c),
                           -np.ones(n_c, int), np.array([np.eye(3)] * n_c), np.full(n_c, MU),
                           np.zeros(n_c))


def test_scc_residual_is_zero_on_valid_and_at_least_the_violation_on_each_case():
    valid = [c for c in CASES if c[0].endswith("_ok")]
    lam, u, _ = _arrays(valid)
    P = _point_mass_problem(lam, u)
    assert oc.dynamics_residual(P, u.ravel(), lam) <= 1e-15
    assert oc.scc_residual(P, u.ravel(), lam) <= 1e-15
    for case in CASES:
        if case[0].endswith("_ok"):
            continue
        # the reference contacts fix Lambda = 2; V = max |u| <= 1 here, so the
        # u-scaled terms can only grow compared with the hand values at V = 1
        lam, u, _ = _arrays(valid + [case])
        P = _point_mass_problem(lam, u)
        r = oc.scc_residual(P, u.ravel(), lam)
        assert r >= max(case[3]) * (1 - 1e-12), (case[0], r)


def test_scc_residual_scales_with_the_gap_term():
    """``u_n`` includes ``phi_m`` (eq. scc's gap term): a resting contact with a
    negative gap is penetrating.  Unit mass, v = 0, lambda = 0, phi = -0.25:
    only the gap condition remains (``Lambda = 0``), ``|u_n| / V = 1``."""
    P = ov.make_problem(np.arange(2), np.arange(1), np.eye(3)[None], np.zeros(3), [0], [-1],
                        np.eye(3)[None], [MU], [-0.25])
    assert np.allclose(oc.contact_velocity(P, np.zeros(3)), [[-0.25, 0.0, 0.0]])
    assert oc.scc_residual(P, np.zeros(3), np.zeros(3)) == 1.0
    P.phi[:] = 0.25
    assert oc.scc_residual(P, np.zeros(3), np.zeros(3)) == 0.0


def test_contact_velocity_uses_the_frame_and_the_d_contact_sign():
    """``u_m = R_m (v_i - v_j) + phi_m e_n`` (eq. jcnode) with rows n, t1, t2."""
    R = np.array([[0.0, 0.0, 1.0], [1.0, 0.0, 0.0], [0.0, 1.0, 0.0]])  # n = e_z
    P = ov.make_problem(np.arange(3), np.arange(2), np.array([np.eye(3)] * 2), np.zeros(6),
                        [0], [1], R[None], [MU], [0.1])
    v = np.array([1.0, 2.0, 3.0, 0.5, 0.25, 4.0])
    # v_i - v_j = (0.5, 1.75, -1); in the frame: (n, t1, t2) = (-1, 0.5, 1.75)
    assert np.allclose(oc.contact_velocity(P, v), [[-1.0 + 0.1, 0.5, 1.75]], atol=1e-15)


def test_dynamics_residual_hand_value():
    """Diagonal A = diag(2, 3, 4), one S-contact with R = I on the node:
    r = A v - b - J^T lambda = (2 - 1 - 1, 3 - 0 - 0.5, 4 - 2 - 0) = (0, 2.5, 2),
    ||r|| / ||b|| = sqrt(10.25) / sqrt(5)."""
    P = ov.make_problem(np.arange(2), np.arange(1), np.diag([2.0, 3.0, 4.0])[None],
                        np.array([1.0, 0.0, 2.0]), [0], [-1], np.eye(3)[None], [MU], [0.0])
    got = oc.dynamics_residual(P, np.ones(3), np.array([1.0, 0.5, 0.0]))
    assert abs(got - math.sqrt(10.25) / math.sqrt(5.0)) <= 1e-15


def test_mode_of_classifies_open_stick_slip():
    """Eq. (scc)'s three cases from the impulse alone: zero normal impulse is
    open, inside the cone is stick, on its boundary is slip."""
    lam = np.array([[0.0, 0.0, 0.0],      # open
                    [2.0, 0.5, 0.0],      # stick: 0.5 < mu * 2 = 1
                    [2.0, -0.6, -0.8],    # slip: ||lambda_t|| = 1 = mu * 2
                    [2e-12, 0.0, 0.0],    # a rounding-level normal impulse is open
                    [1.0, 0.0, 0.0]])     # normal only: stick
    assert oc.mode_of(lam, np.full(5, MU)).tolist() == [0, 1, 2, 0, 1]
