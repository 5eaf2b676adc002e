"""Host logic of the differentiable solve (paper_2201_09212_gb300/autograd.py)
against a fake solver on the CPU: failures of the forward or adjoint solve
raise, scenes that reach l_max are reported per the chosen policy and
recorded on the solver.  The fake does none of the method's arithmetic; it
only plays back the statuses the library would return."""
import warnings

import numpy as np
import pytest
import torch

from paper_2201_09212_gb300 import autograd as ag
from paper_2201_09212_gb300 import vfpi

NOT_CONVERGED = vfpi.VFPI_NOT_CONVERGED
NONFINITE = vfpi.STATUS_CODES["VFPI_ERR_NONFINITE"]
TIMEOUT = vfpi.STATUS_CODES["VFPI_ERR_TIMEOUT"]


class FakeSolver:
    """Stands in for vfpi.Solver: three scenes, one DOF block each."""

    n_scenes, n, n_c = 3, 9, 3

    def __init__(self, forward=(0, 0, 0), adjoint=(0, 0, 0)):
        self.outcomes = {"forward": np.array(forward, np.int32),
                         "adjoint": np.array(adjoint, np.int32)}
        self.phase = "forward"

    def _code(self):
        st = self.outcomes[self.phase]
        if (st < 0).any():
            return int(st[st < 0][0])
        return NOT_CONVERGED if (st == NOT_CONVERGED).any() else 0

    # the calls autograd makes ----------------------------------------------
    def set_rhs(self, b, phi):
        pass

    def set_friction(self, mu):
        pass

    def set_velocity(self, v):
        self.v = v.clone()

    def solve_async(self):
        self.phase = "forward"

    def status(self):
        code = self._code()
        if code < 0:        # what vfpi.Solver.status() does with a failure code
            raise vfpi.VfpiError(code, "fake failure")
        return np.zeros(3, np.int32), np.zeros(3), code

    def scene_status(self):
        return self.outcomes[self.phase].copy()

    def get_velocity(self, out):
        out.copy_(self.v)
        return out

    def get_lambda_star(self, out):
        out.zero_()
        return out

    def adjoint(self, g_v, lambda_star=None, out_b=None, out_phi=None, out_mu=None):
        self.phase = "adjoint"
        code = self._code()
        if code < 0:
            raise vfpi.VfpiError(code, "fake adjoint failure")
        out_b.copy_(g_v)
        out_phi.zero_()
        out_mu.zero_()


def _run(solver, policy="warn", backward=True):
    b = torch.ones(9, requires_grad=True)
    phi = torch.zeros(3)
    mu = torch.full((3,), 0.5, requires_grad=True)
    v0 = torch.zeros(9)
    v = ag.vfpi_solve(solver, b, phi, mu, v0, on_not_converged=policy)
    if backward:
        v.sum().backward()
    return v


def test_converged_solves_report_nothing():
    s = FakeSolver()
    with warnings.catch_warnings():
        warnings.simplefilter("error")
        _run(s)
    assert s.not_converged["forward"].size == 0 and s.not_converged["adjoint"].size == 0


@pytest.mark.parametrize("which", ["forward", "adjoint"])
@pytest.mark.parametrize("code", [NONFINITE, TIMEOUT])
def test_failed_solves_raise(which, code):
    st = [0, code, 0]
    s = FakeSolver(**{which: st})
    with pytest.raises(vfpi.VfpiError) as e:
        _run(s, policy="ignore")
    assert e.value.status == code


def test_forward_not_converged_warns_with_the_scene_indices():
    s = FakeSolver(forward=[NOT_CONVERGED, 0, NOT_CONVERGED])
    with pytest.warns(ag.VfpiNotConvergedWarning, match=r"forward solve: 2 scene\(s\).*scenes 0, 2"):
        _run(s, backward=False)
    assert s.not_converged["forward"].tolist() == [0, 2]


def test_adjoint_not_converged_warns_with_the_scene_indices():
    s = FakeSolver(adjoint=[0, NOT_CONVERGED, 0])
    with pytest.warns(ag.VfpiNotConvergedWarning, match=r"adjoint solve: 1 scene\(s\).*scenes 1"):
        _run(s)
    assert s.not_converged["forward"].size == 0
    assert s.not_converged["adjoint"].tolist() == [1]


def test_raise_policy_raises_and_ignore_only_records():
    s = FakeSolver(forward=[0, 0, NOT_CONVERGED])
    with pytest.raises(ag.VfpiNotConverged) as e:
        _run(s, policy="raise")
    assert e.value.scenes.tolist() == [2]
    s = FakeSolver(adjoint=[NOT_CONVERGED, 0, 0])
    with warnings.catch_warnings():
        warnings.simplefilter("error")
        _run(s, policy="ignore")
    assert s.not_converged["adjoint"].tolist() == [0]
    with pytest.raises(ValueError):
        _run(FakeSolver(), policy="sometimes")
