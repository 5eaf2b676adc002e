"""PyTorch autograd for the V-FPI solve and checkpointed rollouts.

``vfpi_solve(solver, b, phi, mu, v_warm)`` returns the converged ``v_hat`` of
the solver's problem with right-hand side ``b``, penetration terms ``phi`` and
friction ``mu``; its backward runs the library's adjoint kernel
(``vfpi_adjoint``) at the active set of that forward solve (the forward saves
its ``lambda*``), so it stays correct when a checkpointed segment is
recomputed.  ``matvec(solver, x)`` is ``A x`` (backward ``A g``: the system
matrix of the method is symmetric, Sec. II.A).

Failures are loud: a forward or adjoint solve that ends on a non-finite
residual or a timed-out wait raises ``VfpiError`` (the iterate is invalid and
no gradient is formed from it).  A solve that reaches ``l_max`` before its stop
test still returns its last iterate (Alg. 1's second exit), but its scenes are
reported: ``on_not_converged="warn"`` (default) issues a
``VfpiNotConvergedWarning`` naming them, ``"raise"`` raises
``VfpiNotConverged``, ``"ignore"`` only records them; either way the indices
are left in ``solver.not_converged`` (``{"forward": ..., "adjoint": ...}``,
arrays of scene indices of the latest such solve).

``rollout`` integrates a rest-linearised lattice scene (or a batch of them)
for ``steps`` time steps -- ``b_k = M v_k + h M g - kappa (A - M)(x_k - x_0)``,
``phi_k = z_k / h`` on the ground contacts, ``v_{k+1} = v_hat_k``,
``x_{k+1} = x_k + h v_hat_k`` -- recomputing every ``checkpoint`` steps in the
backward pass instead of storing them.  The dynamics harness is plain tensor
algebra; every solve and every product with A runs in the library's kernels.
"""
from __future__ import annotations

import warnings

import numpy as np
import torch
import torch.utils.checkpoint as ckpt

from .vfpi import VFPI_NOT_CONVERGED

POLICIES = ("warn", "raise", "ignore")


class VfpiNotConvergedWarning(RuntimeWarning):
    """Some scenes of a solve reached l_max before the stop test."""


class VfpiNotConverged(RuntimeError):
    """Raised instead of the warning with ``on_not_converged="raise"``."""

    def __init__(self, msg, scenes):
        super().__init__(msg)
        self.scenes = scenes


def _check_outcome(solver, which, policy):
    """Read how the last solve ended.  ``solver.status()`` raises ``VfpiError``
    on a non-finite residual or a timed-out wait; scenes that reached l_max are
    recorded in ``solver.not_converged[which]`` and reported per ``policy``."""
    if policy not in POLICIES:
        raise ValueError(f"on_not_converged must be one of {POLICIES}")
    _, _, st = solver.status()
    bad = np.zeros(0, dtype=np.int64)
    if st == VFPI_NOT_CONVERGED:
        bad = np.nonzero(np.asarray(solver.scene_status()) == VFPI_NOT_CONVERGED)[0]
    rec = getattr(solver, "not_converged", None)
    if not isinstance(rec, dict):
        rec = {}
        solver.not_converged = rec
    rec[which] = bad
    if bad.size and policy != "ignore":
        shown = ", ".join(str(int(q)) for q in bad[:16]) + (", ..." if bad.size > 16 else "")
        msg = (f"{which} solve: {bad.size} scene(s) reached l_max before the stop test "
               f"(scenes {shown}); their last iterate is used")
        if policy == "raise":
            raise VfpiNotConverged(msg, bad)
        warnings.warn(msg, VfpiNotConvergedWarning, stacklevel=3)
    return bad


class _Solve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, solver, b, phi, mu, v_warm, policy):
        solver.set_rhs(b.detach().contiguous(), phi.detach().contiguous())
        solver.set_friction(mu.detach().contiguous())
        v = v_warm.detach().clone().contiguous()
        solver.set_velocity(v)
        solver.solve_async()
        _check_outcome(solver, "forward", policy)
        solver.get_velocity(out=v)
        lam_star = torch.empty(3 * solver.n_c, dtype=b.dtype, device=b.device)
        solver.get_lambda_star(out=lam_star)
        ctx.solver = solver
        ctx.policy = policy
        ctx.save_for_backward(lam_star)
        return v

    @staticmethod
    def backward(ctx, g_v):
        (lam_star,) = ctx.saved_tensors
        s = ctx.solver
        g_b = torch.empty(s.n, dtype=g_v.dtype, device=g_v.device)
        g_phi = torch.empty(s.n_c, dtype=g_v.dtype, device=g_v.device)
        g_mu = torch.empty(s.n_c, dtype=g_v.dtype, device=g_v.device)
        s.adjoint(g_v.contiguous(), lambda_star=lam_star, out_b=g_b, out_phi=g_phi, out_mu=g_mu)
        _check_outcome(s, "adjoint", ctx.policy)
        return None, g_b, g_phi, g_mu, None, None


class _Matvec(torch.autograd.Function):
    @staticmethod
    def forward(ctx, solver, x):
        y = torch.empty_like(x)
        solver.matvec(x.detach().contiguous(), out=y)
        ctx.solver = solver
        return y

    @staticmethod
    def backward(ctx, g):
        y = torch.empty_like(g)
        ctx.solver.matvec(g.contiguous(), out=y)
        return None, y


def vfpi_solve(solver, b, phi, mu, v_warm, on_not_converged="warn"):
    """Differentiable V-FPI solve (see the module docstring for the failure
    policy ``on_not_converged``)."""
    return _Solve.apply(solver, b, phi, mu, v_warm, on_not_converged)


def matvec(solver, x):
    return _Matvec.apply(solver, x)


class LatticeHarness:
    """Per-DOF constants of rest-linearised lattice scenes (see module docstring)."""

    def __init__(self, scene, device, dtype=torch.float32):
        meta = scene.meta
        h = scene.h
        if meta.get("kind") == "lattice_batch":
            nq = meta["nodes"].astype(np.int64)
            dof_scene = np.repeat(np.arange(len(nq)), 3 * nq)
            g = meta["gravity"][dof_scene, np.tile(np.arange(3), int(nq.sum()))]
            kappa = (h * meta["k"] / meta["coef"])[dof_scene]
            self.scene_ptr = scene.scene_ptr
        else:
            coef = h * meta["c"] + h * h * meta["k"]
            g = np.tile(np.asarray(meta["gravity"]), scene.n_nodes)
            kappa = np.full(scene.n, h * meta["k"] / coef)
            self.scene_ptr = np.array([0, scene.n_nodes], dtype=np.int32)
        T = lambda a, dt=dtype: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=device)
        self.h = h
        self.mass = T(scene.mass)
        self.hg = T(h * scene.mass * g)
        self.kappa = T(kappa)
        self.x_rest = T(scene.x0, torch.float64)
        self.zi = T(3 * scene.node_i.astype(np.int64) + 2, torch.int64)
        self.dtype = dtype

    def rhs(self, solver, x, v):
        u = (x - self.x_rest).to(self.dtype)
        b = self.mass * v + self.hg - self.kappa * (matvec(solver, u) - self.mass * u)
        phi = x.index_select(0, self.zi).to(self.dtype) / self.h
        return b, phi

    def com_z(self, x):
        """Height of each scene's centre of mass, [n_scenes] (a fixed-order
        reduction: prefix sums differenced at the scene boundaries)."""
        z = x[2::3]
        ptr = torch.as_tensor(self.scene_ptr, device=x.device, dtype=torch.int64)
        c = torch.cat([torch.zeros(1, dtype=z.dtype, device=z.device), torch.cumsum(z, 0)])
        return (c[ptr[1:]] - c[ptr[:-1]]) / (ptr[1:] - ptr[:-1]).to(z.dtype)


def rollout(solver, harness, x0, v0, mu, steps, checkpoint=8, on_not_converged="warn"):
    """Positions and velocities after ``steps`` time steps, differentiable in
    ``v0`` and ``mu``; ``checkpoint`` <= 0 stores every step instead."""

    def segment(x, v, mu_, n):
        for _ in range(n):
            b, phi = harness.rhs(solver, x, v)
            v = vfpi_solve(solver, b, phi, mu_, v, on_not_converged)
            x = x + harness.h * v.to(x.dtype)
        return x, v

    x, v = x0, v0
    k = 0
    while k < steps:
        n = min(checkpoint, steps - k) if checkpoint > 0 else steps - k
        if checkpoint > 0 and torch.is_grad_enabled():
            x, v = ckpt.checkpoint(segment, x, v, mu, n, use_reentrant=False)
        else:
            x, v = segment(x, v, mu, n)
        k += n
    return x, v
