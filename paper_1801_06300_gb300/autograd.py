"""Gradients through PCEXP steps with torch.autograd (argument marshalling only).

``PCEXPStep.apply(u_n, solver, dt, m)`` runs one PCEXP step (Eq. s9, s10) of the CUDA
library and, in backward, its exact reverse (``pcexp_step_backward``): the step is
recomputed from the saved u_n (per-step checkpointing) and the Krylov bases are rebuilt.
``WallForce.apply(u, solver, kind)`` is the slip-wall pressure force and its gradient;
``VortexError.apply(u, solver, params)`` the L2 error against the translated vortex.
``adjoint_rollout`` chains N steps and returns the functional, its gradient with respect
to the initial state and, optionally, with respect to free-stream parameters and to
parameters of the initial state and the functional (the vortex strength).

States are CUDA float64 tensors of K coefficients in the context's basis.
"""
from __future__ import annotations

import dataclasses

import torch

from . import capi


class PCEXPStep(torch.autograd.Function):
    @staticmethod
    def forward(ctx, u, solver, dt, m):
        u = u.detach().contiguous()
        solver.set_state(u)
        solver.step(capi.PCEXP_SCHEME_PCEXP, capi.PCEXP_DT_GIVEN, float(dt), int(m), info=False)
        out = solver.get_state(torch.empty_like(u))
        ctx.save_for_backward(u)
        ctx.solver, ctx.dt, ctx.m = solver, float(dt), int(m)
        return out

    @staticmethod
    def backward(ctx, g):
        (u,) = ctx.saved_tensors
        ub = ctx.solver.step_backward(u, ctx.dt, ctx.m, g.contiguous())
        return ub, None, None, None


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


def rollout(u0, solver, dt, m, steps):
    """u_N after ``steps`` PCEXP steps, differentiable with respect to u0."""
    u = u0
    for _ in range(steps):
        u = PCEXPStep.apply(u, solver, dt, m)
    return u


@dataclasses.dataclass
class AdjointResult:
    value: float
    grad_u0: torch.Tensor
    grad_params: dict


def adjoint_rollout(solver, u0, dt, m, steps, kind=capi.PCEXP_FUNC_WALL_FX, params=None, initial_state=None,
                    h=1e-6, functional_params=None, case_params=None):
    """Value and gradients of J(u_N), u_{n+1} = PCEXP(u_n; theta).

    grad_u0 is exact (reverse of every step).  For each free-stream parameter name in
    ``params`` (attributes of the Freestream passed as ``params[name] = freestream``),
    dJ/dtheta = sum_n ubar_{n+1} . dF/dtheta (u_n) + ubar_0 . du_0/dtheta, where the
    partial of one step (and of the initial state ``initial_state(free)``) with respect
    to theta is taken by a central difference of width h at fixed u_n.

    ``functional_params`` are passed to the functional (PCEXP_FUNC_VORTEX_L2).
    ``case_params`` = {name: (theta, init(theta) -> u0, fparams(theta) -> functional
    parameters)} lists parameters that enter the initial state and the functional but
    not the step map (the vortex strength): dJ/dtheta = ubar_0 . du_0/dtheta +
    dJ/dtheta at fixed u_N, both partials by central differences of width h (relative
    to max(1, |theta|)).
    """
    checkpoints = [u0.detach().contiguous()]
    u = checkpoints[0]
    for _ in range(steps):
        solver.set_state(u)
        solver.step(capi.PCEXP_SCHEME_PCEXP, capi.PCEXP_DT_GIVEN, float(dt), int(m), info=False)
        u = solver.get_state(torch.empty_like(u))
        checkpoints.append(u)
    grad = torch.empty_like(u)
    value, _ = solver.functional(kind, u, grad, params=functional_params)
    ubars = [None] * (steps + 1)
    ubars[steps] = grad
    for n in range(steps - 1, -1, -1):
        ubars[n] = solver.step_backward(checkpoints[n], float(dt), int(m), ubars[n + 1].contiguous())
    gp = {}
    if params:
        base_free = params["free"]
        for name in params["names"]:
            theta = getattr(base_free, name)
            total = 0.0
            for n in range(steps):
                outs = []
                for sgn in (1.0, -1.0):
                    solver.set_physics(dataclasses.replace(base_free, **{name: theta + sgn * h}))
                    solver.set_state(checkpoints[n])
                    solver.step(capi.PCEXP_SCHEME_PCEXP, capi.PCEXP_DT_GIVEN, float(dt), int(m), info=False)
                    outs.append(solver.get_state(torch.empty_like(u)))
                total += float(torch.dot(ubars[n + 1], (outs[0] - outs[1]) / (2 * h)))
            if initial_state is not None:
                up = initial_state(dataclasses.replace(base_free, **{name: theta + h}))
                um = initial_state(dataclasses.replace(base_free, **{name: theta - h}))
                total += float(torch.dot(ubars[0], (up - um) / (2 * h)))
            solver.set_physics(base_free)
            gp[name] = total
    for name, (theta, init, fparams) in (case_params or {}).items():
        hh = h * max(1.0, abs(theta))
        du0 = (init(theta + hh) - init(theta - hh)) / (2 * hh)
        jp, _ = solver.functional(kind, u, None, params=fparams(theta + hh))
        jm, _ = solver.functional(kind, u, None, params=fparams(theta - hh))
        gp[name] = float(torch.dot(ubars[0], du0)) + (jp - jm) / (2 * hh)
    return AdjointResult(value=value, grad_u0=ubars[0], grad_params=gp)
