"""The adjoint design gradient at full size, and in-place moduli updates.

The compliance gradient dc/dmu_e of the 128^3 Q1 hex benchmark mesh
(2,097,152 elements, lognormal moduli from seed 0, lambda = 10 mu, base
clamped, top sheared by 0.1) is checked against central differences of the
compliance on 32 random elements: each perturbed problem (mu_e +- h, lambda_e
tied) is re-solved from the converged state by a Newton load step with a zero
load increment, and c = u_c . r(u) is evaluated from the library's FP64
residual by the test itself.  The moduli are changed in place with
fem_mesh_set_moduli, whose results must equal those of a mesh created with
the new moduli, bit for bit.
"""
import numpy as np
import pytest
import torch

from paper_2602_12365_b300 import meshgen as mg
from paper_2602_12365_b300.fem import Mesh

pytestmark = pytest.mark.gpu

SHEAR = (0.1, 0.0, 0.0)


def _states(m):
    u = torch.as_tensor(mg.smooth_state(m, 0.5).ravel(), device="cuda")
    v = torch.as_tensor(mg.random_direction(m, 1).ravel(), device="cuda")
    return u, v


@pytest.mark.parametrize("kind", ["tet", "hex"])
def test_set_moduli_equals_a_fresh_mesh(kind):
    base = mg.workload_tet(6, seed=3, random_moduli=4) if kind == "tet" else mg.workload_hex(6, seed=4)
    rng = np.random.default_rng(9)
    mu2 = base.mu_e() * np.exp(0.3 * rng.standard_normal(base.n_el))
    lam2 = 10.0 * mu2
    gm = Mesh(base.elem_type, base.coords, base.conn, base.mu_e(), base.lam_e(), dirichlet=base.dirichlet,
              tile_elems=64)
    gm.set_moduli(mu2, lam2)
    fresh = Mesh(base.elem_type, base.coords, base.conn, mu2, lam2, dirichlet=base.dirichlet, tile_elems=64)
    u, v = _states(base)
    for dt in (torch.float64, torch.float32):
        a, b = u.to(dt), v.to(dt)
        assert torch.equal(gm.energy(a), fresh.energy(a))
        assert torch.equal(gm.residual(a), fresh.residual(a))
        assert torch.equal(gm.hvp(a, b), fresh.hvp(a, b))
        assert torch.equal(gm.block_diag(a), fresh.block_diag(a))
    assert gm.sync_status() == 0


def test_set_moduli_rejects_bad_input():
    from paper_2602_12365_b300._lib import FemError
    m = mg.workload_tet(3, seed=1, random_moduli=2)
    gm = Mesh.from_fixture(m)
    u, _ = _states(m)
    before = gm.residual(u).clone()
    bad = m.mu_e().copy()
    bad[5] = -1.0
    with pytest.raises(FemError, match="mu > 0"):
        gm.set_moduli(bad, m.lam_e())
    assert torch.equal(gm.residual(u), before)  # nothing changed
    scalar = Mesh.from_fixture(mg.workload_tet(3, seed=1))
    with pytest.raises(FemError, match="scalar moduli"):
        scalar.set_moduli(m.mu_e(), m.lam_e())


def test_adjoint_gradient_128_matches_central_differences():
    m = mg.workload_hex(128, seed=0)
    assert m.n_el == 2_097_152
    mu, lam = m.mu.copy(), m.lam.copy()
    gm = Mesh(m.elem_type, m.coords, m.conn, mu, lam, dirichlet=m.dirichlet)
    ubar = torch.as_tensor(m.ubar.ravel(), dtype=torch.float64, device="cuda")
    u = torch.zeros(m.n_nodes * 3, dtype=torch.float64, device="cuda")
    s_prev = 0.0
    for s in (0.5, 1.0):  # the final state of the load path (hyperelastic: path independent)
        assert gm.newton_step(u, ubar, s_prev, s, cg_dtype=torch.float32)["status"] == 0
        s_prev = s
    # the checkpoint polished by a zero increment, so that the perturbed
    # problems below start from a residual far below their own
    st = gm.newton_step(u, ubar, 1.0, 1.0, cg_dtype=torch.float32, newton_rtol=1e-3, max_bisect=0, eta_max=1e-4)
    assert st["status"] == 0
    c, grad, iters = gm.compliance_gradient(u, rtol=1e-10, cg_dtype=torch.float32)
    grad = grad.cpu().numpy()
    assert iters > 0 and np.all(np.isfinite(grad))
    uc = torch.where(gm.dirichlet_mask(u.device), u, torch.zeros_like(u))
    assert float(c.item()) == pytest.approx(float(torch.dot(uc, gm.residual(u, mask_out=False))), rel=1e-12)
    rng = np.random.default_rng(2024)
    els = rng.choice(m.n_el, size=32, replace=False)
    # What limits the check is the FD quotient, not the adjoint: the perturbed
    # solves stop at 1e-6 of their own initial residual, which scales with h,
    # so their error moves the quotient by an amount that does not shrink
    # with h.  Measured: |FD - adjoint| up to ~4e-14 (3.5e-7 of the largest
    # gradient, random in sign), the same with h tripled, while an adjoint
    # solved to 1e-12 instead of 1e-10 moved only in the tenth digit.  On the
    # sampled elements (gradients ~2e-9) that is up to ~2e-5 of their own
    # gradient, hence a 5e-5 bar; gradients under 1 % of the largest are
    # compared relative to that 1 %.
    floor = 1e-2 * np.abs(grad).max()
    worst = 0.0
    for e in els:
        h = 1e-3 * mu[e]
        rs = []
        for sgn in (1.0, -1.0):
            mp = mu.copy()
            mp[e] += sgn * h
            gm.set_moduli(mp, 10.0 * mp)
            up = u.clone()
            # linear solves to 1e-4 (eta_max); the step stops once the residual
            # is under 1e-6 of the perturbation's initial residual (~5e-9)
            st = gm.newton_step(up, ubar, 1.0, 1.0, cg_dtype=torch.float32, newton_rtol=1e-6, max_bisect=0,
                                newton_max=20, eta_max=1e-4)
            assert st["status"] == 0
            rs.append(gm.residual(up, mask_out=False))
        # c(+) - c(-) = u_c . (r(+) - r(-)): the difference first, so that the
        # two compliances' common part cancels exactly
        fd = float(torch.dot(uc, rs[0] - rs[1])) / (2 * h)
        err = abs(fd - grad[e]) / max(abs(grad[e]), floor)
        print(f"element {e}: adjoint {grad[e]:.10e} FD {fd:.10e} |diff| {abs(fd - grad[e]):.3e} rel {err:.2e}")
        worst = max(worst, err)
        assert err <= 5e-5, (e, fd, grad[e])
    gm.set_moduli(mu, lam)
    print(f"128^3 adjoint vs central differences on 32 elements: worst relative error {worst:.2e}, "
          f"max |dc/dmu| {np.abs(grad).max():.3e}, floor {floor:.3e}")
