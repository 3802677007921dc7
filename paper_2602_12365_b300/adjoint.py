"""Adjoint design gradient of the compliance with respect to per-element moduli.

Under pure displacement loading the work done by the prescribed displacements
u_c is the compliance c = u_c^T r_c(u*), r = grad Psi_h at the converged state
u* (free residual r_f(u*) = 0).  Differentiating with r_f(u*(mu), mu) = 0
fixed:

    dc/dmu = u_c^T dr_c/dmu - lam^T dr_f/dmu,   K_ff lam = K_fc u_c,

i.e. dc/dmu_e = a^T dr_e/dmu_e with a = (-lam on free DOFs, u_c on prescribed
ones).  The moduli are tied as lambda_e = ratio * mu_e, so
d/dmu_e = d/dmu_e + ratio d/dlambda_e, which fem_param_vjp returns per element
as (g_mu, g_lam).  K_fc u_c is one masked HVP with u_c as the direction, and
the adjoint solve is fem_tangent_solve (block-Jacobi PCG on the HVP kernel).
The state u* is the checkpoint of the last converged load step: the material
is hyperelastic, so the gradient depends on the final state only.
"""
from __future__ import annotations

import torch

from .fem import Mesh


def compliance(mesh: Mesh, u: torch.Tensor, uc: torch.Tensor) -> float:
    """c = u_c^T r(u) over the prescribed DOFs (uc is zero elsewhere), FP64."""
    r = mesh.residual(u, mask_out=False)
    return float(torch.dot(uc, r))


def prescribed_part(mesh: Mesh, u: torch.Tensor) -> torch.Tensor:
    """u on prescribed DOFs, 0 on free ones."""
    return torch.where(mesh.dirichlet_mask(u.device), u, torch.zeros_like(u))


def compliance_gradient(mesh: Mesh, u: torch.Tensor, ratio: float = 10.0, rtol: float = 1e-10,
                        cg_dtype=torch.float64, vjp_dtype=torch.float64):
    """Return (c, dc/dmu [n_elems] FP64, adjoint CG iterations) at the
    converged FP64 state u.  ``cg_dtype`` float32 runs the adjoint PCG in FP32
    with FP64 dot products; ``vjp_dtype`` is the element pass's arithmetic."""
    uc = prescribed_part(mesh, u)
    c = compliance(mesh, u, uc)
    # K_fc u_c: the HVP with u_c as the direction, output masked to free DOFs
    rhs = mesh.hvp(u, uc, mask_in=False, mask_out=True)
    lam, iters = mesh.tangent_solve(u, rhs, rtol=rtol, cg_dtype=cg_dtype)
    a = uc - lam  # lam vanishes on prescribed DOFs
    if vjp_dtype == torch.float64:
        g_mu, g_lam = mesh.param_vjp(u, a)
    else:
        g_mu, g_lam = mesh.param_vjp(u.to(vjp_dtype), a.to(vjp_dtype))
    return c, g_mu + ratio * g_lam, iters
