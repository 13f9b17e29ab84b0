"""The reduced objective of variable projection as a differentiable torch
function.

J(c) = min over h of ||S[c] h - d||^2 + alpha ||A h||^2 (eqn:esis): the
source subproblem solved for a velocity model c, as a function of c alone
(eqn:esi and the paragraph after eqn:esis). Its gradient is the gradient of
the subproblem's objective in c at the minimiser (the objective is
stationary in h there), which ``ssx_velocity_gradient`` computes by the
discrete adjoint state method with checkpoints. The inner problem is solved
by conjugate gradients on its normal equation (SSX_MODE_CG), whose
minimiser is the one of this Euclidean objective.

Every step runs in the CUDA library; this module only marshals tensors.
"""
from __future__ import annotations

import torch

from . import ssx


class ReducedObjective(torch.autograd.Function):
    """forward(vel, d, context, rho, alpha, maxit, rtol, checkpoint_every) -> J
    (0-d float64 tensor); backward gives dJ/dvel (the same shape and dtype
    as vel). The context's model is set to vel; its geometry and grid stay."""

    @staticmethod
    def forward(fctx, vel, d, context, rho, alpha, maxit, rtol, checkpoint_every):
        context.set_velocity_model(vel.detach().to(torch.float32).contiguous(), float(rho))
        h, _, iters, status = context.solve(d, alpha, maxit, rtol, ssx.MODE_CG)
        g, phi = context.velocity_gradient(h, d, alpha, checkpoint_every)
        fctx.save_for_backward(g)
        fctx.vel_dtype = vel.dtype
        fctx.inner = (iters, status)
        return torch.tensor(phi, dtype=torch.float64, device=vel.device)

    @staticmethod
    def backward(fctx, grad_out):
        (g,) = fctx.saved_tensors
        return (grad_out * g).to(fctx.vel_dtype), None, None, None, None, None, None, None


def reduced_objective(vel, d, context, rho=1.0, alpha=0.0, maxit=30, rtol=1e-6,
                      checkpoint_every=50):
    """J(vel) for one shot (see ReducedObjective); sum over shots' contexts
    for a survey."""
    return ReducedObjective.apply(vel, d, context, rho, alpha, maxit, rtol, checkpoint_every)
