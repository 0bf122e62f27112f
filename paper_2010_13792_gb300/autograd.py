"""Differentiable force evaluation: a ``torch.autograd.Function`` whose
backward is libgrav's hand-written adjoint kernel (``grav_eval_backward``).

Forward returns the accelerations a_i at every element and the potential
energy W = 1/2 sum_i m_i Phi_i; backward takes dL/da and dL/dW and returns
dL/dx and dL/dm.  Pair terms are recomputed in the backward pass, nothing
per pair is stored.  The paper has no adjoint; the sums are the derivatives
of Eq. 4's acceleration and of the softened potential (see
``include/grav.h``).
"""
from __future__ import annotations

import torch

from . import grav


class GravityForce(torch.autograd.Function):
    """(pos [n,3], mass [n], vel [n,3]) -> (acc [n,3], W scalar)."""

    @staticmethod
    def forward(ctx, pos, mass, vel, h: float, G: float = 1.0, precision: int = grav.MIXED):
        n = mass.numel()
        pos = pos.contiguous()
        mass = mass.contiguous()
        vel = vel.contiguous()
        acc = torch.empty(n, 3, dtype=torch.float64, device=pos.device)
        jerk = torch.empty_like(acc)
        tidal = torch.empty(n, 6, dtype=torch.float64, device=pos.device)
        pot = torch.empty(n, dtype=torch.float64, device=pos.device)
        p = grav.params(G=G, h=h, precision=precision, want_pot=True)
        grav.eval_active(p, pos, vel, mass, None, None, n, acc, jerk, tidal, pot, None)
        W = 0.5 * torch.dot(mass, pot)
        ctx.save_for_backward(pos, mass, acc, tidal, pot)
        ctx.h, ctx.G, ctx.precision = h, G, precision
        return acc, W

    @staticmethod
    def backward(ctx, g_acc, g_W):
        pos, mass, acc, tidal, pot = ctx.saved_tensors
        n = mass.numel()
        a_bar = None if g_acc is None else g_acc.contiguous().to(torch.float64)
        w_bar = 0.0 if g_W is None else float(g_W.item())
        pos_bar = torch.empty(n, 3, dtype=torch.float64, device=pos.device)
        mass_bar = torch.empty(n, dtype=torch.float64, device=pos.device)
        p = grav.params(G=ctx.G, h=ctx.h, precision=ctx.precision)
        grav.eval_backward(p, pos, mass, a_bar, w_bar, acc, tidal, pot, pos_bar, mass_bar)
        return pos_bar, mass_bar, None, None, None, None


def gravity(pos, mass, vel=None, *, h: float, G: float = 1.0, precision: int = grav.MIXED):
    """Accelerations and potential energy, differentiable in pos and mass."""
    if vel is None:
        vel = torch.zeros_like(pos)
    return GravityForce.apply(pos, mass, vel, h, G, precision)
