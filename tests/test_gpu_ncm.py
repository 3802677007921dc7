"""Neural constitutive model on the GPU against the oracle.

Bars as for the Neo-Hookean kernels: FP64 within 1e-12 and FP32 within 1e-5
of the oracle (relative 2-norm; energies relative to their roundoff scale S,
which includes |NN| and |NN(3, 1)|), with the oracle evaluated at the inputs
an FP32 call sees.  The network is evaluated in the call's precision.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2602_12365_b300 import meshgen as mg
from paper_2602_12365_b300._lib import FemError
from paper_2602_12365_b300.fem import Mesh

pytestmark = pytest.mark.gpu

TOL = {torch.float64: 1e-12, torch.float32: 1e-5}


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _same(x, dtype):
    x = np.asarray(x, dtype=np.float64)
    return x.astype(np.float32).astype(np.float64) if dtype == torch.float32 else x


def _mesh(kind):
    return mg.workload_tri(5) if kind == "tri" else mg.workload_tet(3, seed=2, random_moduli=2)


@pytest.mark.parametrize("kind", ["tri", "tet"])
@pytest.mark.parametrize("H", [8, 16, 32])
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_operators_match_oracle(kind, H, dtype):
    m = _mesh(kind)
    gm = Mesh.from_fixture(m)
    p = mg.ncm_params(H, seed=H, amp=0.3)
    gm.set_ncm(H, p)
    om = oracle.OracleMesh.from_mesh(m)
    u = mg.smooth_state(m, 0.5, amp=0.05).ravel()
    v = mg.random_direction(m, 2).ravel()
    ut = torch.as_tensor(u, dtype=dtype, device="cuda")
    vt = torch.as_tensor(v, dtype=dtype, device="cuda")
    us, vs = _same(u, dtype), _same(v, dtype)
    e = gm.energy(ut).cpu().numpy()
    r = gm.residual(ut).cpu().numpy()
    y = gm.hvp(ut, vt).cpu().numpy()
    D = gm.block_diag(ut).cpu().numpy()
    with oracle.ncm(H, p):
        psi, _, S, st = om.energy(us, per_element=True)
        assert st == 0
        assert abs(e[0] - psi) <= TOL[dtype] * S and abs(e[1] - S) <= TOL[dtype] * S
        assert _rel(r, om.residual(us)) <= TOL[dtype]
        assert _rel(y, om.hvp(us, vs)) <= TOL[dtype]
        assert _rel(D, om.block_diag(us).ravel()) <= TOL[dtype]
    assert gm.sync_status() == 0


def test_zero_output_layer_and_removal_give_neo_hookean():
    m = mg.workload_tet(4, seed=1, random_moduli=1)
    gm = Mesh.from_fixture(m, precision="fp64")
    u = torch.as_tensor(mg.smooth_state(m, 0.5, amp=0.05).ravel(), device="cuda")
    v = torch.as_tensor(mg.random_direction(m, 3).ravel(), device="cuda")
    ref = (gm.energy(u).clone(), gm.residual(u).clone(), gm.hvp(u, v).clone())
    H = 16
    p = mg.ncm_params(H, seed=9)
    p[4 * H + H * H:5 * H + H * H] = 0.0  # w3 = 0: the network is the constant b3
    gm.set_ncm(H, p)
    for got, want in ((gm.residual(u), ref[1]), (gm.hvp(u, v), ref[2])):  # to rounding
        assert (torch.linalg.norm(got - want) / torch.linalg.norm(want)).item() <= 1e-14
    assert gm.energy(u)[0].item() == pytest.approx(ref[0][0].item(), rel=1e-14)
    gm.set_ncm(16, mg.ncm_params(16, seed=2, amp=0.5))
    assert not torch.equal(gm.residual(u), ref[1])
    gm.set_ncm(0)
    assert torch.equal(gm.residual(u), ref[1]) and torch.equal(gm.hvp(u, v), ref[2])


def test_newton_load_step_matches_oracle():
    """The solver needs no change for the network (the paper's point): the
    FP64 load step lands on the oracle's, the mixed one on the FP64 one."""
    m = mg.workload_tet(4, seed=3, random_moduli=3)
    H = 16
    p = mg.ncm_params(H, seed=5, amp=0.2)
    om = oracle.OracleMesh.from_mesh(m)
    ubar = m.ubar.ravel()
    uo = np.zeros(m.n_nodes * 3)
    with oracle.ncm(H, p):
        st = om.load_step(ubar, 0.0, 0.05, uo)
    assert st.status == 0
    gm = Mesh.from_fixture(m)
    gm.set_ncm(H, p)
    ub = torch.as_tensor(ubar, dtype=torch.float64, device="cuda")
    res = {}
    for dt in (torch.float64, torch.float32):
        u = torch.zeros(m.n_nodes * 3, dtype=torch.float64, device="cuda")
        s = gm.newton_step(u, ub, 0.0, 0.05, cg_dtype=dt)
        assert s["status"] == 0 and s["r_norm"] <= 1e-8 * s["r0_norm"]
        res[dt] = u.cpu().numpy()
    assert _rel(res[torch.float64], uo) <= 1e-7
    assert _rel(res[torch.float32], res[torch.float64]) <= 1e-6


def test_sparse_K_with_network():
    m = mg.workload_tet(2, seed=6, random_moduli=6)
    H = 8
    p = mg.ncm_params(H, seed=1, amp=0.4)
    gm = Mesh.from_fixture(m, precision="fp64")
    gm.set_ncm(H, p)
    u = mg.smooth_state(m, 0.5, amp=0.05).ravel()
    vals = gm.sparse_assemble(torch.as_tensor(u, device="cuda"), mask_in=False, mask_out=False).cpu().numpy()
    om = oracle.OracleMesh.from_mesh(m)
    with oracle.ncm(H, p):
        _, _, ref = om.sparse_K(u, mask_in=False, mask_out=False)
    assert _rel(vals, ref) <= 1e-12


def test_arguments_are_checked():
    mh = mg.workload_hex(2)
    gh = Mesh.from_fixture(mh)
    with pytest.raises(FemError, match="P1"):
        gh.set_ncm(8, mg.ncm_params(8))
    m = mg.workload_tet(2)
    gm = Mesh.from_fixture(m)
    with pytest.raises(FemError):
        gm.set_ncm(12, np.zeros(12 * 12 + 61))
    p = mg.ncm_params(8)
    p[3] = np.nan
    with pytest.raises(FemError):
        gm.set_ncm(8, p)
    gm.set_ncm(8, mg.ncm_params(8))
    u = torch.zeros(m.n_nodes * 3, dtype=torch.float32, device="cuda")
    with pytest.raises(FemError, match="Neo-Hookean"):
        gm.hvp_atomic(u, u.clone())
