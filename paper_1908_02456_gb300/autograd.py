"""Gradient of the absorbed probability with respect to the potential, as a
torch.autograd.Function over the native adjoint (``abc_adjoint_run``).

J(V) = sum_j (1 - h^3 |phi_j(T)|^2): the probability that left the box through the
absorbing boundary after ``nsteps`` steps from ``psi0`` in the static potential V.
The forward pass runs the native forward sweep (with checkpoints every
``ckpt_every`` steps) and the discrete adjoint of the Horner stages in one call;
backward scales the stored dJ/dV.
"""
from __future__ import annotations

import torch


class AbsorbedProbability(torch.autograd.Function):
    @staticmethod
    def forward(fctx, V, psi0, context, dt, nsteps, ckpt_every):
        J, g = context.adjoint(psi0.contiguous(), V.contiguous(), dt, nsteps, ckpt_every)
        fctx.save_for_backward(g)
        return torch.tensor(J, dtype=torch.float64, device=V.device)

    @staticmethod
    def backward(fctx, grad_J):
        (g,) = fctx.saved_tensors
        return grad_J.to(g.dtype) * g, None, None, None, None, None


def absorbed_probability(V, psi0, context, dt, nsteps, ckpt_every=50):
    """J(V); differentiable in V (psi0 and the context are constants)."""
    return AbsorbedProbability.apply(V, psi0, context, dt, nsteps, ckpt_every)
