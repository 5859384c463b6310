"""The MERA energy as a torch.autograd.Function.

Forward evaluates only the energy per bottom site (ascending maps and the
scale-invariant fixed point, ``mera_energy``).  Backward re-enters the
library for the reverse pass of every layer (``mera_energy_grad``), whose
conjugated-leaf adjoints are the u/w environments; the forward
intermediates are recomputed there (warm-started from the forward's fixed
point) instead of being kept by autograd.

Gradient convention: the library's partial derivative is
D_v = 2 dC/d conj(v) (Sec. 2.3).  For real tensors that is the ordinary
gradient dC/dv.  For complex tensors torch's gradient of a real function is
also 2 dC/d conj(v) (it returns 2 z for |z|^2), so in both cases backward
returns grad_output * D_v, unscaled and unprojected (the Riemannian
gradient is its tangent projection, ``Mera.project``).  Complex tensors need
a problem created with dtype MERA_C128; their first-order change is
dC = Re sum conj(grad) dW.
"""
from __future__ import annotations

import torch

from . import mera as gm


class MeraEnergy(torch.autograd.Function):
    @staticmethod
    def forward(ctx, problem: "gm.Mera", *tensors):
        pts = [t.detach().to(torch.complex128 if t.is_complex() else torch.float64).contiguous()
               for t in tensors]
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
