"""The MERA energy as a torch.autograd.Function.

Forward evaluates only the energy per bottom site (ascending maps and the
scale-invariant fixed point, ``mera_energy``).  Backward re-enters the
library for the reverse pass of every layer (``mera_energy_grad``), whose
conjugated-leaf adjoints are the u/w environments; the forward
intermediates are recomputed there (warm-started from the forward's fixed
point) instead of being kept by autograd.

Gradient convention: for real tensors the library's partial derivative
D_v = 2 dC/d conj(v) (Sec. 2.3) equals the ordinary gradient dC/dv, which is
what torch expects, so backward returns grad_output * D_v (unprojected; the
Riemannian gradient is its tangent projection, ``Mera.project``).
"""
from __future__ import annotations

import torch

from . import mera as gm


class MeraEnergy(torch.autograd.Function):
    @staticmethod
    def forward(ctx, problem: "gm.Mera", *tensors):
        pts = [t.detach().to(torch.float64).contiguous() for t in tensors]
        problem.set_tensors(pts)
        e = problem.energy_only()
        ctx.problem = problem
        ctx.save_for_backward(*pts)
        return torch.tensor(e, dtype=torch.float64, device=tensors[0].device)

    @staticmethod
    def backward(ctx, grad_out):
        pts = ctx.saved_tensors
        problem = ctx.problem
        problem.set_tensors(list(pts))
        _, _, D = problem.energy_grad(device=pts[0].is_cuda, deriv=True)
        g = grad_out.to(torch.float64)
        return (None,) + tuple(g * d.to(pts[0].device) for d in D)


def mera_energy(problem: "gm.Mera", tensors):
    """Differentiable energy per bottom site of the MERA given by ``tensors``
    ([u_0, w_0, ..., u_L, w_L]) under ``problem``'s Hamiltonian."""
    return MeraEnergy.apply(problem, *tensors)
