"""Gradients through PCEXP steps with torch.autograd (argument marshalling only).

``PCEXPStep.apply(u_n, theta, solver, dt, m)`` runs one PCEXP step (Eq. s9, s10) of the CUDA
library with the free-stream parameters theta = (Mach number, flow angle in degrees) and, in
backward, its exact reverse (``pcexp_step_backward``): the step is recomputed from the saved
u_n (per-step checkpointing), the Krylov bases are rebuilt, and the adjoints of u_n and of
theta come back from the library.  ``ProjectedState.apply(theta, solver, kind, params)`` is
the projected initial state (``pcexp_project_state``) with its exact adjoint;
``WallForce.apply(u, solver, kind)`` the slip-wall pressure force and ``VortexError.apply(u,
solver, params)`` the L2 error against the translated vortex, each with its gradient from
the library.  ``adjoint_rollout`` chains N steps without autograd and returns the functional
and its gradients with respect to the initial state, (Mach, alpha) and the vortex strength.

States are CUDA float64 tensors of K coefficients in the context's basis; theta is a float64
tensor of 2 entries.  Every derivative is computed by the library; this module only moves
arguments and results.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import torch

from . import capi


def _free_with(solver_free, theta):
    return dataclasses.replace(solver_free, mach=float(theta[0]), alpha_deg=float(theta[1]))


class PCEXPStep(torch.autograd.Function):
    @staticmethod
    def forward(ctx, u, theta, solver, free, dt, m):
        u = u.detach().contiguous()
        fr = _free_with(free, theta.detach().cpu())
        solver.set_physics(fr)
        solver.set_state(u)
        solver.step(capi.PCEXP_SCHEME_PCEXP, capi.PCEXP_DT_GIVEN, float(dt), int(m), info=False)
        out = solver.get_state(torch.empty_like(u))
        ctx.save_for_backward(u, theta.detach())
        ctx.solver, ctx.free, ctx.dt, ctx.m = solver, free, float(dt), int(m)
        return out

    @staticmethod
    def backward(ctx, g):
        u, theta = ctx.saved_tensors
        ctx.solver.set_physics(_free_with(ctx.free, theta.cpu()))
        ub, th = ctx.solver.step_backward(u, ctx.dt, ctx.m, g.contiguous(), with_theta=True)
        return ub, torch.tensor(th, dtype=theta.dtype, device=theta.device), None, None, None, None


class ProjectedState(torch.autograd.Function):
    """u_0 = projection of the analytic state `kind` with params, under free stream theta."""

    @staticmethod
    def forward(ctx, theta, solver, free, kind, params):
        solver.set_physics(_free_with(free, theta.detach().cpu()))
        solver.project_state(kind, params)
        u0 = solver.get_state(torch.empty(solver.K, dtype=torch.float64, device="cuda"))
        ctx.save_for_backward(theta.detach())
        ctx.solver, ctx.free, ctx.kind, ctx.params = solver, free, kind, list(params)
        return u0

    @staticmethod
    def backward(ctx, g):
        (theta,) = ctx.saved_tensors
        ctx.solver.set_physics(_free_with(ctx.free, theta.cpu()))
        th = ctx.solver.project_state_adjoint(ctx.kind, ctx.params, g.contiguous())
        return torch.tensor(th[:2], dtype=theta.dtype, device=theta.device), None, None, None, None


class WallForce(torch.autograd.Function):
    @staticmethod
    def forward(ctx, u, solver, kind=capi.PCEXP_FUNC_WALL_FX):
        u = u.detach().contiguous()
        grad = torch.empty_like(u)
        val, _ = solver.functional(kind, u, grad)
        ctx.save_for_backward(grad)
        return torch.tensor(val, dtype=u.dtype, device=u.device)

    @staticmethod
    def backward(ctx, g):
        (grad,) = ctx.saved_tensors
        return g * grad, None, None


class VortexError(torch.autograd.Function):
    @staticmethod
    def forward(ctx, u, solver, params):
        u = u.detach().contiguous()
        grad = torch.empty_like(u)
        val, _ = solver.functional(capi.PCEXP_FUNC_VORTEX_L2, u, grad, params=params)
        ctx.save_for_backward(grad)
        return torch.tensor(val, dtype=u.dtype, device=u.device)

    @staticmethod
    def backward(ctx, g):
        (grad,) = ctx.saved_tensors
        return g * grad, None, None


def rollout(u0, theta, solver, free, dt, m, steps):
    """u_N after ``steps`` PCEXP steps, differentiable with respect to u0 and theta."""
    u = u0
    for _ in range(steps):
        u = PCEXPStep.apply(u, theta, solver, free, dt, m)
    return u


@dataclasses.dataclass
class AdjointResult:
    value: float
    grad_u0: torch.Tensor
    grad_params: dict


def adjoint_rollout(solver, u0, dt, m, steps, kind=capi.PCEXP_FUNC_WALL_FX, functional_params=None,
                    initial=None):
    """Value and gradients of J(u_N), u_{n+1} = PCEXP(u_n; theta), theta = (Mach, alpha).

    Forward steps keep their checkpoints u_n; the reverse sweep calls pcexp_step_backward
    per step, which returns ubar_n and the step's adjoint of theta.  grad_params holds
      mach, alpha_deg:  sum_n theta_bar_n (+ the initial state's and the functional's share),
      eps (vortex functional and vortex initial state): the initial state's share plus the
           functional's partial at fixed u_N.
    ``initial`` = (kind, params) of the projected initial state u0 (its adjoint then
    contributes); None leaves u0 as given.  ``functional_params`` are passed to the
    functional (PCEXP_FUNC_VORTEX_L2)."""
    checkpoints = [u0.detach().contiguous()]
    u = checkpoints[0]
    for _ in range(steps):
        solver.set_state(u)
        solver.step(capi.PCEXP_SCHEME_PCEXP, capi.PCEXP_DT_GIVEN, float(dt), int(m), info=False)
        u = solver.get_state(torch.empty_like(u))
        checkpoints.append(u)
    grad = torch.empty_like(u)
    value, _ = solver.functional(kind, u, grad, params=functional_params)
    theta = np.zeros(2)
    ub = grad
    for n in range(steps - 1, -1, -1):
        ub, th = solver.step_backward(checkpoints[n], float(dt), int(m), ub.contiguous(), with_theta=True)
        theta += th
    gp = {}
    dJ = solver.functional_param_grad(kind, u, functional_params)
    theta += dJ[:2]
    eps = dJ[2]
    if initial is not None:
        t0 = solver.project_state_adjoint(initial[0], initial[1], ub.contiguous())
        theta += t0[:2]
        if len(t0) > 2:
            eps += t0[2]
    gp["mach"], gp["alpha_deg"] = float(theta[0]), float(theta[1])
    if kind == capi.PCEXP_FUNC_VORTEX_L2 or (initial is not None and initial[0] == capi.PCEXP_PROJ_VORTEX):
        gp["eps"] = float(eps)
    return AdjointResult(value=value, grad_u0=ub, grad_params=gp)
