"""Pins of the FP64 CPU oracle to facts it does not compute itself.

Each test checks the oracle against something fixed by the mathematics or by
textbook mechanics rather than against a retyped copy of its own formulas:
rest state, frame indifference, the small-strain (Lame) limit, the
linear-elastic stiffness in Voigt notation, patch tests and the virial
identity, finite differences, Hessian symmetry, brute-force dense K, the
uniaxial-bar closed forms and the reaction/energy consistency of a minimiser.
A plausible slip in the oracle (a dropped term, a flipped sign, a transposed
operand, a wrong quadrature weight) fails at least one of them.
"""
import numpy as np
import pytest
from scipy.optimize import brentq

from paper_2602_12365_b300 import meshgen as mg

MU, LAM = 1.0, 10.0
RNG = np.random.default_rng(1234)


def _rot3(rng):
    q, r = np.linalg.qr(rng.standard_normal((3, 3)))
    q = q * np.sign(np.diag(r))
    if np.linalg.det(q) < 0:
        q[:, 0] *= -1
    return q


def _near_identity(d, rng, s=0.2):
    return np.eye(d) + s * rng.standard_normal((d, d))


def _jitter(mesh, amp, seed):
    g = mg.grid_index(mesh)
    interior = np.all((g > 0) & (g < mesh.n), axis=1)
    rng = np.random.default_rng(seed)
    X = mesh.coords.copy()
    X[interior] += amp / mesh.n * (2 * rng.random(X[interior].shape) - 1)
    mesh.coords = X
    return mesh


def _omesh(ora, m, mask=None):
    return ora.OracleMesh(m.elem_type, m.coords, m.conn, m.mu_e(), m.lam_e(),
                          mask if mask is not None else m.dirichlet)


MESHES = {
    "tri": lambda: _jitter(mg.tri_mesh(3), 0.2, 1),
    "tet": lambda: mg.tet_mesh(2, jitter_seed=3),
    "hex": lambda: _jitter(mg.hex_mesh(2), 0.15, 2),
}


# ---------------------------------------------------------------------------
# material law
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("d", [2, 3])
def test_rest_state_density(ora, d):
    I = np.eye(d)
    assert ora.nh_psi(I) == 0.0
    assert np.all(ora.nh_P(I) == 0.0)


def test_frame_indifference(ora):
    rng = np.random.default_rng(7)
    for _ in range(10):
        F = _near_identity(3, rng)
        R = _rot3(rng)
        assert ora.nh_psi(R @ F) == pytest.approx(ora.nh_psi(F), rel=1e-12, abs=1e-14)
        # P is a two-point tensor: P(RF) = R P(F)
        np.testing.assert_allclose(ora.nh_P(R @ F), R @ ora.nh_P(F), atol=1e-12)
    c, s = np.cos(0.7), np.sin(0.7)
    R2 = np.array([[c, -s], [s, c]])
    F2 = _near_identity(2, rng)
    assert ora.nh_psi(R2 @ F2) == pytest.approx(ora.nh_psi(F2), rel=1e-12)


@pytest.mark.parametrize("d", [2, 3])
def test_small_strain_lame_limit(ora, d):
    """psi(I + eps A) = eps^2 [mu sym(A):sym(A) + lam/2 tr(A)^2] + O(eps^3)."""
    rng = np.random.default_rng(11 + d)
    for _ in range(5):
        A = rng.standard_normal((d, d))
        S = 0.5 * (A + A.T)
        lin = MU * np.sum(S * S) + 0.5 * LAM * np.trace(A) ** 2
        for eps in (1e-3, 1e-4):
            val = ora.nh_psi(np.eye(d) + eps * A, MU, LAM) / eps ** 2
            assert abs(val - lin) <= 30 * eps * (abs(lin) + 1)


def test_plane_strain_is_3d_with_unit_stretch(ora):
    rng = np.random.default_rng(5)
    for _ in range(5):
        F2 = _near_identity(2, rng)
        F3 = np.eye(3)
        F3[:2, :2] = F2
        assert ora.nh_psi(F2) == pytest.approx(ora.nh_psi(F3), rel=1e-13)
        np.testing.assert_allclose(ora.nh_P(F2), ora.nh_P(F3)[:2, :2], atol=1e-13)


@pytest.mark.parametrize("d", [2, 3])
def test_stress_is_fd_derivative_of_density(ora, d):
    rng = np.random.default_rng(21 + d)
    F = _near_identity(d, rng)
    P = ora.nh_P(F)
    h = 1e-6
    for i in range(d):
        for j in range(d):
            E = np.zeros((d, d))
            E[i, j] = h
            fd = (ora.nh_psi(F + E) - ora.nh_psi(F - E)) / (2 * h)
            assert fd == pytest.approx(P[i, j], abs=1e-8)


@pytest.mark.parametrize("d", [2, 3])
def test_tangent_is_fd_derivative_of_stress(ora, d):
    rng = np.random.default_rng(31 + d)
    F = _near_identity(d, rng)
    dF = rng.standard_normal((d, d))
    h = 1e-6
    fd = (ora.nh_P(F + h * dF) - ora.nh_P(F - h * dF)) / (2 * h)
    np.testing.assert_allclose(ora.nh_dP(F, dF), fd, atol=1e-7)


def test_inverted_density_is_infinite(ora):
    F = np.diag([1.0, 1.0, -0.5])
    assert ora.nh_psi(F) == np.inf


# ---------------------------------------------------------------------------
# assembled energy / residual / HVP
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("kind", ["tri", "tet", "hex"])
def test_rest_mesh(ora, kind):
    m = MESHES[kind]()
    om = _omesh(ora, m, mask=np.zeros((m.n_nodes, m.dim), np.uint8))
    u = np.zeros(m.n_nodes * m.dim)
    assert om.energy(u) == 0.0
    assert np.all(om.residual(u) == 0.0)


def _volume(m):
    return 1.0  # unit square / cube, boundary nodes never move


@pytest.mark.parametrize("kind", ["tri", "tet", "hex"])
def test_patch_test_affine_field(ora, kind):
    """u = A X + b: Psi = psi(I + A) |Omega|, zero interior residual, and the
    virial identity sum_a r_a (x) X_a = P |Omega|."""
    m = MESHES[kind]()
    d = m.dim
    rng = np.random.default_rng(41)
    A = 0.15 * rng.standard_normal((d, d))
    b = rng.standard_normal(d)
    u = m.coords @ A.T + b
    om = _omesh(ora, m, mask=np.zeros((m.n_nodes, d), np.uint8))
    F = np.eye(d) + A
    assert om.energy(u) == pytest.approx(ora.nh_psi(F) * _volume(m), rel=1e-12)
    r = om.residual(u).reshape(-1, d)
    g = mg.grid_index(m)
    interior = np.all((g > 0) & (g < m.n), axis=1)
    scale = np.abs(r).max()
    assert np.abs(r[interior]).max() <= 1e-12 * max(scale, 1.0)
    virial = r.T @ m.coords
    np.testing.assert_allclose(virial, ora.nh_P(F) * _volume(m), atol=1e-12)
    # sum of all nodal forces is zero (translation invariance of Psi)
    np.testing.assert_allclose(r.sum(axis=0), 0.0, atol=1e-12)


def _state(m, seed, s=0.05):
    rng = np.random.default_rng(seed)
    return s * rng.standard_normal(m.n_nodes * m.dim)


@pytest.mark.parametrize("kind", ["tri", "tet", "hex"])
def test_residual_is_fd_gradient(ora, kind):
    m = MESHES[kind]()
    om = _omesh(ora, m, mask=np.zeros((m.n_nodes, m.dim), np.uint8))
    u = _state(m, 3)
    r = om.residual(u)
    rng = np.random.default_rng(4)
    for _ in range(3):
        v = rng.standard_normal(u.size)
        h = 1e-5
        fd = (om.energy(u + h * v) - om.energy(u - h * v)) / (2 * h)
        assert fd == pytest.approx(r @ v, rel=1e-7, abs=1e-10)


@pytest.mark.parametrize("kind", ["tri", "tet", "hex"])
def test_hvp_is_fd_of_residual_and_symmetric(ora, kind):
    m = MESHES[kind]()
    om = _omesh(ora, m, mask=np.zeros((m.n_nodes, m.dim), np.uint8))
    u = _state(m, 5)
    rng = np.random.default_rng(6)
    v = rng.standard_normal(u.size)
    w = rng.standard_normal(u.size)
    h = 1e-6
    fd = (om.residual(u + h * v) - om.residual(u - h * v)) / (2 * h)
    Kv = om.hvp(u, v, mask_in=False, mask_out=False)
    np.testing.assert_allclose(Kv, fd, atol=1e-7 * np.abs(Kv).max())
    Kw = om.hvp(u, w, mask_in=False, mask_out=False)
    assert abs(w @ Kv - v @ Kw) <= 1e-12 * np.linalg.norm(v) * np.linalg.norm(Kw)


def _dense_K(om, u, masked=False):
    n = u.size
    K = np.zeros((n, n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        K[:, j] = om.hvp(u, e, mask_in=masked, mask_out=masked)
    return K


@pytest.mark.parametrize("kind", ["tri", "tet", "hex"])
def test_brute_force_dense_K(ora, kind):
    """Dense K on a 1-4 element mesh vs the FD Hessian of the energy."""
    builders = {"tri": lambda: mg.tri_mesh(1), "tet": lambda: mg.tet_mesh(1),
                "hex": lambda: mg.hex_mesh(1)}
    m = builders[kind]()
    if kind == "tet":  # keep 4 elements
        m.conn = m.conn[:4]
    om = _omesh(ora, m, mask=np.zeros((m.n_nodes, m.dim), np.uint8))
    u = _state(m, 8, 0.05)
    K = _dense_K(om, u)
    n = u.size
    h = 1e-4
    H = np.zeros((n, n))
    E = np.eye(n) * h
    for i in range(n):
        for j in range(i, n):
            H[i, j] = (om.energy(u + E[i] + E[j]) - om.energy(u + E[i] - E[j])
                       - om.energy(u - E[i] + E[j]) + om.energy(u - E[i] - E[j])) / (4 * h * h)
            H[j, i] = H[i, j]
    np.testing.assert_allclose(K, H, atol=2e-6 * np.abs(K).max())
    np.testing.assert_allclose(K, K.T, atol=1e-13 * np.abs(K).max())


def _voigt_stiffness(m, mu, lam):
    """Linear-elastic P1 stiffness sum_e vol B^T D B (Voigt notation, shape
    function gradients from the nodal interpolation matrix)."""
    d = m.dim
    n = m.n_nodes * d
    K = np.zeros((n, n))
    if d == 3:
        D = lam * np.outer([1, 1, 1, 0, 0, 0], [1, 1, 1, 0, 0, 0]) + mu * np.diag([2, 2, 2, 1, 1, 1])
    else:
        D = np.array([[lam + 2 * mu, lam, 0], [lam, lam + 2 * mu, 0], [0, 0, mu]])
    for e, c in enumerate(m.conn):
        Xe = m.coords[c]
        Mx = np.hstack([np.ones((d + 1, 1)), Xe])      # N_a(x_b) = delta_ab
        coef = np.linalg.inv(Mx)                        # columns: N_a coefficients
        grads = coef[1:, :].T                           # [a][k]
        vol = abs(np.linalg.det(Mx)) / (2.0 if d == 2 else 6.0)
        B = np.zeros((3 if d == 2 else 6, (d + 1) * d))
        for a in range(d + 1):
            gx, gy = grads[a, 0], grads[a, 1]
            if d == 2:
                B[:, 2 * a:2 * a + 2] = [[gx, 0], [0, gy], [gy, gx]]
            else:
                gz = grads[a, 2]
                B[:, 3 * a:3 * a + 3] = [[gx, 0, 0], [0, gy, 0], [0, 0, gz],
                                         [0, gz, gy], [gz, 0, gx], [gy, gx, 0]]
        Ke = vol * B.T @ D @ B
        dofs = (c[:, None] * d + np.arange(d)[None, :]).ravel()
        K[np.ix_(dofs, dofs)] += Ke
    return K


@pytest.mark.parametrize("kind", ["tri", "tet"])
def test_tangent_at_rest_is_linear_elastic_stiffness(ora, kind):
    m = MESHES[kind]()
    if kind == "tet":
        m = mg.tet_mesh(1, jitter_seed=None)
    om = _omesh(ora, m, mask=np.zeros((m.n_nodes, m.dim), np.uint8))
    K = _dense_K(om, np.zeros(m.n_nodes * m.dim))
    Kv = _voigt_stiffness(m, MU, LAM)
    np.testing.assert_allclose(K, Kv, atol=1e-12 * np.abs(Kv).max())


@pytest.mark.parametrize("kind", ["tri", "tet", "hex"])
def test_block_diag_matches_dense_K(ora, kind):
    m = MESHES[kind]()
    d = m.dim
    mask = np.zeros((m.n_nodes, d), np.uint8)
    mask[0, :] = 1
    mask[1, 0] = 1
    om = _omesh(ora, m, mask=mask)
    u = _state(m, 9)
    D = om.block_diag(u)
    K = _dense_K(_omesh(ora, m, mask=np.zeros_like(mask)), u)
    for i in range(m.n_nodes):
        blk = K[i * d:(i + 1) * d, i * d:(i + 1) * d].copy()
        for k in range(d):
            if mask[i, k]:
                blk[k, :] = 0
                blk[:, k] = 0
                blk[k, k] = 1
        np.testing.assert_allclose(D[i], blk, atol=1e-13 * np.abs(K).max())


def test_masks(ora):
    m = MESHES["tet"]()
    d = m.dim
    mask = np.zeros((m.n_nodes, d), np.uint8)
    mask[:5] = 1
    om = _omesh(ora, m, mask=mask)
    u = _state(m, 10)
    v = np.random.default_rng(3).standard_normal(u.size)
    full = _omesh(ora, m, mask=np.zeros_like(mask))
    mv = np.where(mask.ravel() == 1, 0.0, v)
    np.testing.assert_allclose(om.hvp(u, v), np.where(mask.ravel() == 1, 0.0, full.hvp(u, mv)),
                               atol=1e-14)
    np.testing.assert_allclose(om.residual(u), np.where(mask.ravel() == 1, 0, full.residual(u)))


def test_param_vjp_is_fd_in_moduli(ora):
    m = MESHES["hex"]()
    mg.lognormal_moduli(m, 3)
    om = _omesh(ora, m, mask=np.zeros((m.n_nodes, m.dim), np.uint8))
    u = _state(m, 12)
    a = np.random.default_rng(13).standard_normal(u.size)
    gm, gl = om.param_vjp(u, a)
    for e in range(m.n_el):
        h = 1e-6
        for which, g in (("mu", gm), ("lam", gl)):
            vals = []
            for sgn in (1, -1):
                mu, lam = m.mu.copy(), m.lam.copy()
                if which == "mu":
                    mu[e] += sgn * h
                else:
                    lam[e] += sgn * h
                o2 = ora.OracleMesh(m.elem_type, m.coords, m.conn, mu, lam,
                                    np.zeros((m.n_nodes, m.dim), np.uint8))
                vals.append(a @ o2.residual(u))
            assert (vals[0] - vals[1]) / (2 * h) == pytest.approx(g[e], rel=1e-6, abs=1e-9)


def test_hex_quadrature_volume(ora):
    """2x2x2 Gauss integrates det J of a trilinear map exactly; for a
    parallelepiped the element volume is |det(edge vectors)|."""
    rng = np.random.default_rng(17)
    Am = np.eye(3) + 0.3 * rng.standard_normal((3, 3))
    ref = np.array(mg.HEX_LOCAL, dtype=float)
    Xe = ref @ Am.T + rng.standard_normal(3)
    tot = sum(ora.geometry(2, Xe, q)[0] for q in range(8))
    assert tot == pytest.approx(abs(np.linalg.det(Am)), rel=1e-13)


# ---------------------------------------------------------------------------
# Newton-CG: uniaxial bar closed forms
# ---------------------------------------------------------------------------
def _bar(kind, delta):
    m = mg.tri_mesh(4) if kind == "tri" else mg.tet_mesh(2)
    return mg.bc_uniaxial_bar(m, delta)


def _reaction(om, u, m):
    r = om.residual(u, mask_out=False).reshape(-1, m.dim)
    ax = 0 if m.dim == 2 else 2
    hi = mg.grid_index(m)[:, ax] == m.n
    return r[hi, ax].sum()


@pytest.mark.parametrize("kind,modulus", [("tri", 4 * MU * (LAM + MU) / (LAM + 2 * MU)),
                                          ("tet", MU * (3 * LAM + 2 * MU) / (LAM + MU))])
def test_uniaxial_bar_small_strain_modulus(ora, kind, modulus):
    delta = 1e-6
    m = _bar(kind, delta)
    om = _omesh(ora, m)
    u = np.zeros(m.n_nodes * m.dim)
    st = om.load_step(m.ubar, 0.0, 1.0, u)
    assert st.status == 0
    assert _reaction(om, u, m) / delta == pytest.approx(modulus, rel=1e-5)


def _lateral_stretch(dim, delta):
    if dim == 2:   # F = diag(1 + delta, b), plane strain
        f = lambda b: MU * (b - 1 / b) + LAM * np.log((1 + delta) * b) / b
    else:          # F = diag(b, b, 1 + delta)
        f = lambda b: MU * (b - 1 / b) + LAM * np.log(b * b * (1 + delta)) / b
    return brentq(f, 0.3, 2.0, xtol=1e-15, rtol=1e-15)


@pytest.mark.parametrize("kind", ["tri", "tet"])
def test_uniaxial_bar_nonlinear_homogeneous_solution(ora, kind):
    delta = 0.3
    m = _bar(kind, delta)
    om = _omesh(ora, m)
    u = np.zeros(m.n_nodes * m.dim)
    s_prev = 0.0
    for s in (0.5, 1.0):
        st = om.load_step(m.ubar, s_prev, s, u)
        assert st.status == 0, st.status
        assert st.r_norm <= 1e-8 * st.r0_norm
        s_prev = s
    b = _lateral_stretch(m.dim, delta)
    X = m.coords
    if m.dim == 2:
        exact = np.stack([delta * X[:, 0], (b - 1) * X[:, 1]], axis=1)
    else:
        exact = np.stack([(b - 1) * X[:, 0], (b - 1) * X[:, 1], delta * X[:, 2]], axis=1)
    err = np.linalg.norm(u - exact.ravel()) / np.linalg.norm(exact)
    assert err <= 1e-8


def test_reaction_is_derivative_of_minimised_energy(ora):
    """At equilibrium the reaction equals d Psi*/d delta (a variational
    identity that holds for any hyperelastic law)."""
    def solve(delta):
        m = _bar("tri", delta)
        om = _omesh(ora, m)
        u = np.zeros(m.n_nodes * m.dim)
        st = om.load_step(m.ubar, 0.0, 1.0, u)
        assert st.status == 0
        return om.energy(u), _reaction(om, u, m)
    d0, h = 0.2, 1e-4
    _, R = solve(d0)
    Ep, _ = solve(d0 + h)
    Em, _ = solve(d0 - h)
    assert (Ep - Em) / (2 * h) == pytest.approx(R, rel=1e-6)


def test_newton_load_path_converges(ora):
    m = mg.workload_tri(6)
    om = _omesh(ora, m)
    u = np.zeros(m.n_nodes * 2)
    s_prev = 0.0
    E_prev = 0.0
    for k in range(1, 4):
        s = k / 3
        st = om.load_step(m.ubar, s_prev, s, u)
        assert st.status == 0
        assert st.r_norm <= 1e-8 * st.r0_norm
        E = om.energy(u)
        assert E > E_prev  # stretching stores more energy
        E_prev = E
        s_prev = s
        pres = m.dirichlet.ravel() == 1
        np.testing.assert_array_equal(u[pres], s * m.ubar.ravel()[pres])


def test_adjoint_compliance_gradient_matches_fd(ora):
    """dc/dmu_e by the adjoint recipe vs central FD of the converged
    compliance c = u_c^T r_c(u*) with lambda_e = 10 mu_e."""
    m = mg.bc_base_and_top_3d(mg.lognormal_moduli(mg.hex_mesh(2), 4), (0.05, 0.0, 0.0))
    d = m.dim
    mask = m.dirichlet.ravel().astype(bool)

    def converged(mu):
        om = ora.OracleMesh(m.elem_type, m.coords, m.conn, mu, 10 * mu, m.dirichlet)
        u = np.zeros(m.n_nodes * d)
        st = om.load_step(m.ubar, 0.0, 1.0, u)
        assert st.status == 0
        return om, u

    def compliance(mu):
        om, u = converged(mu)
        r = om.residual(u, mask_out=False)
        return u[mask] @ r[mask]

    om, u = converged(m.mu)
    full = ora.OracleMesh(m.elem_type, m.coords, m.conn, m.mu, m.lam,
                          np.zeros((m.n_nodes, d), np.uint8))
    K = _dense_K(full, u)
    free = ~mask
    uc = np.where(mask, u, 0.0)
    lam_f = np.linalg.solve(K[np.ix_(free, free)], (K @ uc)[free])
    a = uc.copy()
    a[free] = -lam_f
    gm, gl = full.param_vjp(u, a)
    grad = gm + 10 * gl
    for e in range(m.n_el):
        h = 1e-5 * m.mu[e]
        mp, mm = m.mu.copy(), m.mu.copy()
        mp[e] += h
        mm[e] -= h
        fd = (compliance(mp) - compliance(mm)) / (2 * h)
        assert fd == pytest.approx(grad[e], rel=1e-5)


def test_mlp_backward_is_fd_of_forward(ora):
    rng = np.random.default_rng(3)
    d_in, h1, h2, d_out, n = 5, 7, 6, 4, 3
    Ws = [0.5 * rng.standard_normal((h1, d_in)), 0.1 * rng.standard_normal(h1),
          0.5 * rng.standard_normal((h2, h1)), 0.1 * rng.standard_normal(h2),
          0.5 * rng.standard_normal((d_out, h2)), 0.1 * rng.standard_normal(d_out)]
    x = rng.standard_normal((n, d_in))
    gy = rng.standard_normal((n, d_out))
    grads, gx = ora.mlp_backward(x, *Ws, gy)
    L = lambda W, xx: np.sum(gy * ora.mlp_forward(xx, *W))
    h = 1e-6
    for k, W in enumerate(Ws):
        flat = W.reshape(-1)
        for idx in range(0, flat.size, max(1, flat.size // 5)):
            Wp = [w.copy() for w in Ws]
            Wm = [w.copy() for w in Ws]
            Wp[k].reshape(-1)[idx] += h
            Wm[k].reshape(-1)[idx] -= h
            fd = (L(Wp, x) - L(Wm, x)) / (2 * h)
            assert fd == pytest.approx(grads[k].reshape(-1)[idx], rel=1e-6, abs=1e-8)
    xp = x.copy()
    xp[1, 2] += h
    xm = x.copy()
    xm[1, 2] -= h
    assert (L(Ws, xp) - L(Ws, xm)) / (2 * h) == pytest.approx(gx[1, 2], rel=1e-6)


def test_mlp_special_cases(ora):
    """Zero hidden weights give y = W3 silu(silu(b1)...) structure; with all
    weights zero the output is the last bias; SiLU(0) = 0."""
    d_in, h1, h2, d_out = 3, 4, 4, 2
    z = lambda *s: np.zeros(s)
    b3 = np.array([0.25, -1.5])
    y = ora.mlp_forward(np.ones((2, d_in)), z(h1, d_in), z(h1), z(h2, h1), z(h2), z(d_out, h2), b3)
    np.testing.assert_array_equal(y, np.tile(b3, (2, 1)))
    # one path: W1 = e, W2 = e, W3 = e with b = 0: y = silu(silu(x0))
    W1 = z(1, 1) + 1
    x = np.array([[2.0]])
    s = lambda t: t / (1 + np.exp(-t))
    y = ora.mlp_forward(x, W1, z(1), W1, z(1), W1, z(1))
    assert y[0, 0] == pytest.approx(s(s(2.0)), rel=1e-15)


# ---------------------------------------------------------------------------
# learned block preconditioner: node graph, features, SPD blocks
# ---------------------------------------------------------------------------
def test_node_graph_brute_force_and_kuhn_counts(ora):
    m = mg.tet_mesh(3)
    ptr, idx = ora.node_graph(m.n_nodes, m.conn)
    nb = [set() for _ in range(m.n_nodes)]
    for e in m.conn:
        for a in e:
            nb[a].update(int(b) for b in e if b != a)
    for i in range(m.n_nodes):
        assert list(idx[ptr[i]:ptr[i + 1]]) == sorted(nb[i])
    # an interior vertex of the Kuhn (Freudenthal) triangulation has 14
    # neighbours and 24 incident tetrahedra
    g = mg.grid_index(m)
    interior = np.all((g > 0) & (g < m.n), axis=1)
    assert np.all(np.diff(ptr)[interior] == 14)
    val = np.bincount(m.conn.ravel(), minlength=m.n_nodes)
    assert np.all(val[interior] == 24)


def _spd_blocks(rng, n):
    B = rng.standard_normal((n, 3, 3))
    return B @ B.transpose(0, 2, 1) + 0.5 * np.eye(3)


def test_lp_blocks_identity_output_is_block_jacobi(ora):
    rng = np.random.default_rng(5)
    D = _spd_blocks(rng, 7)
    o = np.zeros((7, 6))
    o[:, [0, 2, 5]] = np.log(np.expm1(1.0 - 1e-4))  # softplus(o) + 1e-4 = 1
    M, ok = ora.lp_blocks(D, None, o)
    assert ok
    np.testing.assert_allclose(M, np.linalg.inv(D), rtol=1e-12, atol=1e-14)
    # a prescribed component gets an identity row and column
    mask = np.zeros((7, 3), np.uint8)
    mask[2, 1] = 1
    Mm, _ = ora.lp_blocks(D, mask, o)
    assert Mm[2, 1, 1] == 1.0 and Mm[2, 1, 0] == 0.0 and Mm[2, 0, 1] == 0.0
    np.testing.assert_array_equal(Mm[3], M[3])


def test_lp_blocks_are_spd_and_backward_is_fd(ora):
    rng = np.random.default_rng(6)
    D = _spd_blocks(rng, 5)
    o = rng.standard_normal((5, 6))
    M, ok = ora.lp_blocks(D, None, o)
    assert ok
    np.testing.assert_allclose(M, M.transpose(0, 2, 1), atol=1e-13)
    assert np.all(np.linalg.eigvalsh(M) > 0)
    mask = np.zeros((5, 3), np.uint8)
    mask[1, 2] = 1
    gM = rng.standard_normal((5, 3, 3))
    go = ora.lp_blocks_backward(D, mask, o, gM)
    L = lambda oo: np.sum(gM * ora.lp_blocks(D, mask, oo)[0])
    h = 1e-6
    for i in range(5):
        for k in range(6):
            op, om_ = o.copy(), o.copy()
            op[i, k] += h
            om_[i, k] -= h
            assert (L(op) - L(om_)) / (2 * h) == pytest.approx(go[i, k], rel=1e-6, abs=1e-9)


def test_lp_features_invariants(ora):
    m = mg.bc_base_and_top_3d(mg.tet_mesh(3))
    mu = np.full(m.n_el, 2.0)
    lam = 10 * mu
    D = np.tile(3.0 * np.eye(3), (m.n_nodes, 1, 1))  # every block the same
    F = ora.lp_features(m.elem_type, m.conn, mu, lam, m.dirichlet, D)
    assert F.shape == (m.n_nodes, 36)
    slog = lambda x: np.sign(x) * np.log1p(np.abs(x))
    np.testing.assert_allclose(F[:, 0:9], np.tile(slog(np.eye(3).ravel()), (m.n_nodes, 1)))
    np.testing.assert_allclose(F[:, 9:18], F[:, 0:9])       # neighbour mean = own block
    np.testing.assert_allclose(F[:, 18:27], 0.0, atol=0)     # no spread
    np.testing.assert_allclose(F[:, 27], np.log(2.0))
    np.testing.assert_allclose(F[:, 28], np.log(10.0))
    val = np.bincount(m.conn.ravel(), minlength=m.n_nodes)
    np.testing.assert_allclose(F[:, 29], val / 24.0)
    np.testing.assert_array_equal(F[:, 30:33], m.dirichlet)
    np.testing.assert_allclose(F[:, 33:36], 0.0, atol=1e-15)  # log(diag / s) = log 1
    # a block twice as stiff at one node: its neighbours see the spread
    D2 = D.copy()
    D2[0] *= 2.0
    F2 = ora.lp_features(m.elem_type, m.conn, mu, lam, m.dirichlet, D2)
    np.testing.assert_allclose(F2[0, 0:9], F[0, 0:9])         # normalised by its own trace
    ptr, idx = ora.node_graph(m.n_nodes, m.conn)
    j = idx[ptr[0]]
    nbj = ptr[j + 1] - ptr[j]
    assert F2[j, 9] == pytest.approx(slog(1.0 + 1.0 / nbj))   # mean of D_00 / s_j
