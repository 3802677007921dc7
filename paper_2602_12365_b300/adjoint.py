"""Adjoint design gradient of the compliance with respect to per-element moduli.

Under pure displacement loading the work done by the prescribed displacements
u_c is the compliance c = u_c^T r_c(u*), r = grad Psi_h at the converged state
u* (free residual r_f(u*) = 0).  Differentiating with r_f(u*(mu), mu) = 0
fixed:

    dc/dmu = u_c^T dr_c/dmu - lam^T dr_f/dmu,   K_ff lam = K_fc u_c,

i.e. dc/dmu_e = a^T dr_e/dmu_e with a = (-lam on free DOFs, u_c on prescribed
ones).  The moduli are tied as lambda_e = ratio * mu_e, so
d/dmu_e = d/dmu_e + ratio d/dlambda_e.  Every step (c, the right-hand side
K_fc u_c as one HVP, the adjoint PCG, a, the per-element pass and the tied
sum) runs in the library's fem_compliance_gradient; this module only
marshals arguments.  The state u* is the checkpoint of the last converged load
step: the material is hyperelastic, so the gradient depends on the final state
only.
"""
from __future__ import annotations

import torch

from .fem import Mesh


def compliance_gradient(mesh: Mesh, u: torch.Tensor, ratio: float = 10.0, rtol: float = 1e-10,
                        cg_dtype=torch.float64, vjp_dtype=torch.float64):
    """Return (c, dc/dmu [n_elems] FP64, adjoint CG iterations) at the
    converged FP64 state u.  ``cg_dtype`` float32 runs the adjoint PCG in FP32
    with FP64 dot products; ``vjp_dtype`` is the element pass's arithmetic."""
    c, g, iters = mesh.compliance_gradient(u, ratio=ratio, rtol=rtol, cg_dtype=cg_dtype, vjp_dtype=vjp_dtype)
    return float(c.item()), g, iters
