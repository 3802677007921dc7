"""torch.autograd bindings of the element kernels.

The paper differentiates the total potential automatically: the residual is
the gradient of Psi_h (its Eq. 1, via reverse mode) and the tangent acts as
the forward-mode derivative of the residual (Eq. 3).  Here the derivatives are
the hand-written kernels instead:

* ``Energy``:   forward = fem_energy (Eq. 2); backward = the residual kernel.
* ``Residual``: forward = fem_residual; backward = the HVP kernel (K(u) is
  symmetric, so the vector-Jacobian product is K(u) g).
* ``Hvp``:      forward = fem_hvp; backward in v = K(u) g again.  Its
  derivative in u is a third derivative of Psi, which no kernel provides, so
  asking for it raises.

Double backward of the energy (a Hessian-vector product through
``torch.autograd.grad(..., create_graph=True)``) therefore runs the HVP
kernel.  All results are unmasked (the full gradient and Hessian); Dirichlet
conditions are the caller's business.
"""
from __future__ import annotations

import torch

from .fem import Mesh


class Energy(torch.autograd.Function):
    @staticmethod
    def forward(ctx, u: torch.Tensor, mesh: Mesh) -> torch.Tensor:
        ctx.mesh = mesh
        ctx.save_for_backward(u)
        return mesh.energy(u)[0].clone()

    @staticmethod
    def backward(ctx, g):
        (u,) = ctx.saved_tensors
        r = Residual.apply(u, ctx.mesh)
        return g.to(r.dtype) * r, None


class Residual(torch.autograd.Function):
    @staticmethod
    def forward(ctx, u: torch.Tensor, mesh: Mesh) -> torch.Tensor:
        ctx.mesh = mesh
        ctx.save_for_backward(u)
        return mesh.residual(u, mask_out=False)

    @staticmethod
    def backward(ctx, g):
        (u,) = ctx.saved_tensors
        return Hvp.apply(u, g.contiguous().to(u.dtype), ctx.mesh), None


class Hvp(torch.autograd.Function):
    @staticmethod
    def forward(ctx, u: torch.Tensor, v: torch.Tensor, mesh: Mesh) -> torch.Tensor:
        ctx.mesh = mesh
        ctx.save_for_backward(u)
        return mesh.hvp(u, v, mask_in=False, mask_out=False)

    @staticmethod
    def backward(ctx, g):
        (u,) = ctx.saved_tensors
        if ctx.needs_input_grad[0]:
            raise NotImplementedError("the derivative of K(u) v in u (a third derivative of Psi) "
                                      "has no kernel")
        return None, Hvp.apply(u, g.contiguous().to(u.dtype), ctx.mesh), None


def energy(u: torch.Tensor, mesh: Mesh) -> torch.Tensor:
    """Psi_h(u) as a differentiable FP64 scalar."""
    return Energy.apply(u, mesh)


def residual(u: torch.Tensor, mesh: Mesh) -> torch.Tensor:
    """grad Psi_h(u) (unmasked), differentiable once more through the HVP."""
    return Residual.apply(u, mesh)
