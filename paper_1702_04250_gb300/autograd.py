"""PPPM energy as a differentiable torch function.

``PPPMEnergy.apply(x, q, plan)`` returns the PPPM k-space energy (the energy
pppm_compute reports: mesh energy minus the self and neutralising-background
terms).  Its gradients are hand-written CUDA, not autograd of an expression:
one pppm_energy_grad call builds the mesh potential phi of the plan's
influence function and interpolates it back with the charge-assignment
stencil -- the transpose of make_rho -- giving

    dE/dq_i = C phi(x_i) - 2 C g q_i / sqrt(pi) - C pi Q / (g^2 V)
    dE/dx_i = C q_i sum_p dW(p - u_i)/dx phi(p)

which are the exact derivatives of the PPPM energy (for ad plans dE/dx is
minus the force before the self-force correction; for ik plans it differs
from the ik force at the discretisation level).  The forward pass computes
them together with the energy and the backward pass scales them by the
incoming gradient.
"""
from __future__ import annotations

import torch


class PPPMEnergy(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, q, plan):
        dEdx, dEdq, ev = plan.energy_grad(x, q)
        ctx.save_for_backward(dEdx, dEdq)
        ctx.x_dtype = x.dtype
        ctx.q_dtype = q.dtype
        return ev[0].clone()

    @staticmethod
    def backward(ctx, gE):
        dEdx, dEdq = ctx.saved_tensors
        gx = gq = None
        if ctx.needs_input_grad[0]:
            gx = (gE * dEdx.double()).to(ctx.x_dtype)
        if ctx.needs_input_grad[1]:
            gq = (gE * dEdq.double()).to(ctx.q_dtype)
        return gx, gq, None


def pppm_energy(x, q, plan):
    """Differentiable PPPM k-space energy of charges q at positions x."""
    return PPPMEnergy.apply(x, q, plan)
