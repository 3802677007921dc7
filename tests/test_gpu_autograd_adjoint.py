"""torch.autograd bindings and the adjoint compliance gradient on the GPU.

Autograd: the energy's backward is the residual kernel and its double
backward the HVP kernel (bitwise the same calls), both checked against
central finite differences and torch.autograd.gradcheck / gradgradcheck.

Adjoint: dc/dmu_e at the converged state against (i) the oracle's own
adjoint -- its load steps, then K_ff lam = K_fc u_c by CG on the oracle HVP
-- and (ii) central differences of re-solved compliances on sampled
elements.
"""
import numpy as np
import pytest
import torch
from scipy.sparse.linalg import LinearOperator, cg

import oracle
from paper_2602_12365_b300 import autograd as fa
from paper_2602_12365_b300 import meshgen as mg
from paper_2602_12365_b300.adjoint import compliance_gradient
from paper_2602_12365_b300.fem import Mesh

pytestmark = pytest.mark.gpu


def _state(m, dtype, s=0.5, amp=0.02):
    return torch.as_tensor(mg.smooth_state(m, s, amp).ravel(), dtype=dtype, device="cuda")


def _dir(m, seed, dtype=torch.float64):
    return torch.as_tensor(mg.random_direction(m, seed).ravel(), dtype=dtype, device="cuda")


@pytest.mark.parametrize("kind", ["tri", "tet", "hex"])
def test_energy_backward_is_the_residual_kernel(kind):
    m = {"tri": lambda: mg.workload_tri(10), "tet": lambda: mg.workload_tet(5, seed=1),
         "hex": lambda: mg.workload_hex(4, seed=2)}[kind]()
    gm = Mesh.from_fixture(m)
    u = _state(m, torch.float64).requires_grad_(True)
    (g,) = torch.autograd.grad(fa.energy(u, gm), u)
    assert torch.equal(g, gm.residual(u.detach(), mask_out=False))
    # central differences of the energy along a random direction
    v = _dir(m, 3)
    h = 1e-6  # truncation O(h^2 |grad v|^3) stays below 1e-8 relative
    with torch.no_grad():
        ep = gm.energy(u.detach() + h * v)[0].item()
        em = gm.energy(u.detach() - h * v)[0].item()
    fd = (ep - em) / (2 * h)
    assert fd == pytest.approx(torch.dot(g, v).item(), rel=1e-7)


@pytest.mark.parametrize("kind", ["tri", "tet", "hex"])
def test_double_backward_is_the_hvp_kernel(kind):
    m = {"tri": lambda: mg.workload_tri(10), "tet": lambda: mg.workload_tet(5, seed=1),
         "hex": lambda: mg.workload_hex(4, seed=2)}[kind]()
    gm = Mesh.from_fixture(m)
    u = _state(m, torch.float64).requires_grad_(True)
    w = _dir(m, 4)
    (g,) = torch.autograd.grad(fa.energy(u, gm), u, create_graph=True)
    (hw,) = torch.autograd.grad(torch.dot(g, w), u)
    assert torch.equal(hw, gm.hvp(u.detach(), w, mask_in=False, mask_out=False))
    h = 1e-6
    with torch.no_grad():
        rp = gm.residual(u.detach() + h * w, mask_out=False)
        rm = gm.residual(u.detach() - h * w, mask_out=False)
    fd = (rp - rm) / (2 * h)
    assert (torch.linalg.norm(fd - hw) / torch.linalg.norm(hw)).item() <= 1e-7


def test_gradcheck_and_gradgradcheck():
    m = mg.workload_tri(3)
    gm = Mesh.from_fixture(m, precision="fp64")
    u = _state(m, torch.float64, amp=0.05).requires_grad_(True)
    assert torch.autograd.gradcheck(lambda x: fa.energy(x, gm), (u,), eps=1e-6, atol=1e-8, rtol=1e-6)
    assert torch.autograd.gradgradcheck(lambda x: fa.energy(x, gm), (u,), eps=1e-6, atol=1e-7, rtol=1e-5)
    assert torch.autograd.gradcheck(lambda x: fa.residual(x, gm), (u,), eps=1e-6, atol=1e-7, rtol=1e-5)


def test_mixed_precision_gradient_matches_oracle():
    m = mg.workload_tet(6, seed=5)
    gm = Mesh.from_fixture(m)
    u32 = _state(m, torch.float32).requires_grad_(True)
    (g,) = torch.autograd.grad(fa.energy(u32, gm), u32)
    assert g.dtype == torch.float32
    om = oracle.OracleMesh.from_mesh(m)
    ref = om.residual(u32.detach().double().cpu().numpy(), mask_out=False)
    err = np.linalg.norm(g.double().cpu().numpy() - ref) / np.linalg.norm(ref)
    assert err <= 1e-5


def test_third_derivative_is_refused():
    m = mg.workload_tri(3)
    gm = Mesh.from_fixture(m, precision="fp64")
    u = _state(m, torch.float64).requires_grad_(True)
    v = _dir(m, 2).requires_grad_(True)
    y = fa.Hvp.apply(u, v, gm)
    with pytest.raises(NotImplementedError):
        torch.autograd.grad(y.sum(), u)
    # with u a constant, d/dv (K v . w) = K w (K symmetric)
    y = fa.Hvp.apply(u.detach(), v, gm)
    (gv,) = torch.autograd.grad(torch.dot(y, v.detach()), v)
    assert torch.equal(gv, gm.hvp(u.detach(), v.detach(), mask_in=False, mask_out=False))


# ---------------------------------------------------------------------------
# adjoint compliance gradient
# ---------------------------------------------------------------------------
SHEAR = (0.1, 0.0, 0.0)
STEPS = (0.5, 1.0)


def _hex_case(n=6, seed=0):
    return mg.bc_base_and_top_3d(mg.lognormal_moduli(mg.hex_mesh(n), seed), SHEAR)


def _gpu_solve(m, mu, **opts):
    gm = Mesh(m.elem_type, m.coords, m.conn, mu, 10.0 * mu, dirichlet=m.dirichlet)
    u = torch.zeros(m.n_nodes * 3, dtype=torch.float64, device="cuda")
    ubar = torch.as_tensor(m.ubar.ravel(), dtype=torch.float64, device="cuda")
    s_prev = 0.0
    for s in STEPS:
        st = gm.newton_step(u, ubar, s_prev, s, **opts)
        assert st["status"] == 0
        s_prev = s
    return gm, u


def _compliance(gm, u):
    """c = u_c . r(u) in FP64 from the library's unmasked residual (the test's
    own evaluation, independent of fem_compliance_gradient)."""
    uc = torch.where(gm.dirichlet_mask(u.device), u, torch.zeros_like(u))
    return float(torch.dot(uc, gm.residual(u, mask_out=False)))


def _oracle_adjoint(m):
    om = oracle.OracleMesh.from_mesh(m)
    u = np.zeros(m.n_nodes * 3)
    s_prev = 0.0
    for s in STEPS:
        assert om.load_step(m.ubar, s_prev, s, u).status == 0
        s_prev = s
    mask = m.dirichlet.ravel().astype(bool)
    uc = np.where(mask, u, 0.0)
    rhs = om.hvp(u, uc, mask_in=False, mask_out=True)
    op = LinearOperator((u.size, u.size), matvec=lambda x: om.hvp(u, x, mask_in=True, mask_out=True),
                        dtype=np.float64)
    lam, info = cg(op, rhs, rtol=1e-12, atol=0.0, maxiter=20000)
    assert info == 0
    full = oracle.OracleMesh(m.elem_type, m.coords, m.conn, m.mu, m.lam, np.zeros_like(m.dirichlet))
    g_mu, g_lam = full.param_vjp(u, uc - np.where(mask, 0.0, lam))
    r = full.residual(u, mask_out=False)
    return uc @ r, g_mu + 10.0 * g_lam


def test_adjoint_gradient_matches_oracle_adjoint():
    # the 16^3 copy of the 128^3 hex benchmark mesh (moduli seed 0)
    m = _hex_case(16, seed=0)
    gm, u = _gpu_solve(m, m.mu)
    c, grad, iters = compliance_gradient(gm, u)
    c_ref, grad_ref = _oracle_adjoint(m)
    assert c == pytest.approx(c_ref, rel=1e-7)
    g = grad.cpu().numpy()
    assert np.linalg.norm(g - grad_ref) / np.linalg.norm(grad_ref) <= 1e-6
    assert iters > 0


def test_adjoint_gradient_matches_central_differences():
    m = _hex_case(5, seed=1)
    gm, u = _gpu_solve(m, m.mu, newton_rtol=1e-11)
    _, grad, _ = compliance_gradient(gm, u)
    grad = grad.cpu().numpy()
    rng = np.random.default_rng(11)
    for e in rng.choice(m.n_el, size=32, replace=False):
        h = 1e-3 * m.mu[e]
        cs = []
        for sgn in (1.0, -1.0):
            mu = m.mu.copy()
            mu[e] += sgn * h
            gp, up = _gpu_solve(m, mu, newton_rtol=1e-11)
            cs.append(_compliance(gp, up))
        fd = (cs[0] - cs[1]) / (2 * h)
        assert fd == pytest.approx(grad[e], rel=2e-5, abs=1e-9 * np.abs(grad).max())


def test_mixed_precision_adjoint_matches_fp64():
    m = _hex_case(6, seed=2)
    gm, u = _gpu_solve(m, m.mu, cg_dtype=torch.float32)
    _, g64, _ = compliance_gradient(gm, u)
    _, g32, _ = compliance_gradient(gm, u, rtol=1e-7, cg_dtype=torch.float32, vjp_dtype=torch.float32)
    assert (torch.linalg.norm(g32 - g64) / torch.linalg.norm(g64)).item() <= 1e-5
