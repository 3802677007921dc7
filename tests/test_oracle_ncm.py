"""Pins of the oracle's neural constitutive model (psi = [NN(I1, J) -
NN(3, 1)] + psi_NH, Sec. "Neural Constitutive Modeling").

The network's derivatives are pinned to central differences of its value;
the law to the shift (zero energy at rest), frame indifference, central
differences of psi and P, and to the Neo-Hookean law when the output layer
is zero; the mesh-level energy, residual, HVP and block diagonal to finite
differences and to the dense K; the load step to equilibrium.
"""
import numpy as np
import pytest

import oracle
from paper_2602_12365_b300 import meshgen as mg

H = 8


def _rot(rng):
    q, r = np.linalg.qr(rng.standard_normal((3, 3)))
    q = q * np.sign(np.diag(r))
    if np.linalg.det(q) < 0:
        q[:, 0] *= -1
    return q


@pytest.fixture
def net():
    p = mg.ncm_params(H, seed=3, amp=0.5)
    with oracle.ncm(H, p):
        yield p


def test_network_derivatives_by_central_differences(net):
    for I1, J in ((3.0, 1.0), (3.3, 0.9), (2.9, 1.15)):
        y, g, h = oracle.ncm_eval(I1, J)
        e = 1e-5
        fd = np.array([(oracle.ncm_eval(I1 + e, J)[0] - oracle.ncm_eval(I1 - e, J)[0]) / (2 * e),
                       (oracle.ncm_eval(I1, J + e)[0] - oracle.ncm_eval(I1, J - e)[0]) / (2 * e)])
        np.testing.assert_allclose(g, fd, rtol=1e-7, atol=1e-9)
        hfd = np.stack([(oracle.ncm_eval(I1 + e, J)[1] - oracle.ncm_eval(I1 - e, J)[1]) / (2 * e),
                        (oracle.ncm_eval(I1, J + e)[1] - oracle.ncm_eval(I1, J - e)[1]) / (2 * e)])
        np.testing.assert_allclose(h, hfd, rtol=1e-6, atol=1e-8)
        np.testing.assert_allclose(h, h.T, rtol=1e-14, atol=0)


def test_shift_gives_zero_energy_at_rest(net):
    assert oracle.law_psi(np.eye(3)) == 0.0
    assert oracle.law_psi(np.eye(2)) == 0.0
    # but not zero stress: the paper shifts the energy only
    P = oracle.law_P(np.eye(3))
    _, g, _ = oracle.ncm_eval(3.0, 1.0)
    np.testing.assert_allclose(P, (2 * g[0] + g[1]) * np.eye(3), atol=1e-15)


def test_frame_indifference(net):
    rng = np.random.default_rng(0)
    for _ in range(3):
        F = np.eye(3) + 0.2 * rng.standard_normal((3, 3))
        Q = _rot(rng)
        assert oracle.law_psi(Q @ F) == pytest.approx(oracle.law_psi(F), rel=1e-12, abs=1e-14)
        np.testing.assert_allclose(oracle.law_P(Q @ F), Q @ oracle.law_P(F), atol=1e-12)


@pytest.mark.parametrize("d", [2, 3])
def test_P_and_dP_by_central_differences(net, d):
    rng = np.random.default_rng(d)
    F = np.eye(d) + 0.15 * rng.standard_normal((d, d))
    dF = rng.standard_normal((d, d))
    P = oracle.law_P(F, 1.3, 7.0)
    e = 1e-6
    Pfd = np.zeros((d, d))
    for i in range(d):
        for j in range(d):
            E = np.zeros((d, d))
            E[i, j] = e
            Pfd[i, j] = (oracle.law_psi(F + E, 1.3, 7.0) - oracle.law_psi(F - E, 1.3, 7.0)) / (2 * e)
    np.testing.assert_allclose(P, Pfd, rtol=1e-6, atol=1e-8)
    dP = oracle.law_dP(F, dF, 1.3, 7.0)
    dPfd = (oracle.law_P(F + e * dF, 1.3, 7.0) - oracle.law_P(F - e * dF, 1.3, 7.0)) / (2 * e)
    np.testing.assert_allclose(dP, dPfd, rtol=1e-6, atol=1e-7)


def test_zero_output_layer_is_neo_hookean():
    m = mg.workload_tet(2, seed=1, random_moduli=1)
    om = oracle.OracleMesh.from_mesh(m)
    u = mg.smooth_state(m, 0.5, amp=0.05).ravel()
    v = mg.random_direction(m, 2).ravel()
    ref = (om.energy(u), om.residual(u), om.hvp(u, v), om.block_diag(u))
    p = mg.ncm_params(H, seed=4)
    p[4 * H + H * H:5 * H + H * H] = 0.0  # w3 = 0: NN is the constant b3
    with oracle.ncm(H, p):
        got = (om.energy(u), om.residual(u), om.hvp(u, v), om.block_diag(u))
    for a, b in zip(got, ref):
        np.testing.assert_array_equal(np.asarray(a), np.asarray(b))


def test_mesh_derivatives_and_dense_K(net):
    m = mg.workload_tet(2, seed=2, random_moduli=2)
    om = oracle.OracleMesh.from_mesh(m)
    u = mg.smooth_state(m, 0.5, amp=0.05).ravel()
    rng = np.random.default_rng(5)
    v = rng.standard_normal(u.size)
    r = om.residual(u, mask_out=False)
    e = 1e-6
    dE = (om.energy(u + e * v) - om.energy(u - e * v)) / (2 * e)
    assert dE == pytest.approx(r @ v, rel=1e-6)
    y = om.hvp(u, v, mask_in=False, mask_out=False)
    yfd = (om.residual(u + e * v, mask_out=False) - om.residual(u - e * v, mask_out=False)) / (2 * e)
    np.testing.assert_allclose(y, yfd, rtol=1e-5, atol=1e-7 * np.abs(y).max())
    nd = u.size
    K = np.stack([om.hvp(u, np.eye(nd)[j], mask_in=False, mask_out=False) for j in range(nd)], axis=1)
    np.testing.assert_allclose(K, K.T, atol=1e-12 * np.abs(K).max())
    D = om.block_diag(u).reshape(-1, 3, 3)
    fixed = m.dirichlet.reshape(-1, 3).astype(bool)
    for n in range(m.n_nodes):
        if fixed[n].any():
            continue
        np.testing.assert_allclose(D[n], K[3 * n:3 * n + 3, 3 * n:3 * n + 3], rtol=1e-12, atol=1e-14)


def test_load_step_reaches_equilibrium():
    m = mg.workload_tet(3, seed=1, random_moduli=1)
    om = oracle.OracleMesh.from_mesh(m)
    p = mg.ncm_params(H, seed=5, amp=0.2)
    with oracle.ncm(H, p):
        u = np.zeros(m.n_nodes * 3)
        ubar = m.ubar.ravel()
        u = np.where(m.dirichlet.reshape(-1).astype(bool), 0.0, u)
        st = om.load_step(ubar, 0.0, 0.05, u)
        assert st.status == 0
        r = om.residual(u, mask_out=True)
        assert np.linalg.norm(r) <= 1e-8 * st.r0_norm
