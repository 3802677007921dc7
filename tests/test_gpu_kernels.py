"""GPU parity of the element kernels against the FP64 CPU oracle.

Bars: FP64 calls match to 1e-12 and FP32 calls to 1e-5, both as the relative
2-norm error ||x_gpu - x_oracle|| / ||x_oracle|| on non-equilibrium states,
and node by node: |x_gpu,i - x_oracle,i| <= tol * s_i, s_i the sum over the
elements touching node i of the size of their contributions there
(tests/parity.py), so that no single node can hide inside the 2-norm.
Both sides take the same inputs: an FP32 call receives u and v rounded to
FP32, so the oracle is evaluated at those rounded values (the input rounding
is a property of FP32 storage, not of the kernel's arithmetic).  Small meshes span
several tiles with a ragged last tile; the full-size workloads (64^3 Kuhn
tets, 128^3 hexes) run in the benchmark's launch configuration and are
checked on sampled nodes, each recomputed by the oracle from its incident
elements alone.
"""
import numpy as np
import pytest
import torch

import oracle
import parity
from paper_2602_12365_b300 import meshgen as mg

pytestmark = pytest.mark.gpu

TOL = {torch.float64: 1e-12, torch.float32: 1e-5}


def _jitter(m, amp, seed):
    g = mg.grid_index(m)
    interior = np.all((g > 0) & (g < m.n), axis=1)
    rng = np.random.default_rng(seed)
    m.coords = m.coords.copy()
    m.coords[interior] += amp / m.n * (2 * rng.random(m.coords[interior].shape) - 1)
    return m


CASES = {
    "tri": (lambda: _jitter(mg.workload_tri(40), 0.2, 1), 256),
    "tet": (lambda: mg.workload_tet(9, seed=2), 256),
    "tet_rand": (lambda: mg.workload_tet(7, seed=3, random_moduli=5), 200),
    "hex": (lambda: _jitter(mg.workload_hex(9, seed=4), 0.1, 2), 100),
}


def _rel(a, b):
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.fixture(scope="module", params=list(CASES))
def case(request):
    from paper_2602_12365_b300.fem import Mesh
    build, tile = CASES[request.param]
    m = build()
    gm = Mesh.from_fixture(m, precision="mixed", tile_elems=tile)
    om = oracle.OracleMesh.from_mesh(m)
    u = mg.smooth_state(m, 0.5).ravel()
    v = mg.random_direction(m, seed=1).ravel()
    return request.param, m, gm, om, u, v


def _t(x, dtype):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=dtype, device="cuda")


def _same(x, dtype):
    """The inputs an FP32 call actually sees, as FP64 for the oracle."""
    x = np.asarray(x, dtype=np.float64)
    return x.astype(np.float32).astype(np.float64) if dtype == torch.float32 else x


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_energy(case, dtype):
    name, m, gm, om, u, v = case
    out = gm.energy(_t(u, dtype)).cpu().numpy()
    psi, _, S, st = om.energy(_same(u, dtype), per_element=True)
    assert st == 0 and out[2] == 0
    assert abs(out[0] - psi) <= TOL[dtype] * abs(psi)
    assert abs(out[1] - S) <= TOL[dtype] * abs(S)
    assert gm.sync_status() == 0


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("mask_out", [True, False])
def test_residual(case, dtype, mask_out):
    name, m, gm, om, u, v = case
    r = gm.residual(_t(u, dtype), mask_out=mask_out).cpu().numpy()
    ro = om.residual(_same(u, dtype), mask_out=mask_out)
    assert _rel(r, ro) <= TOL[dtype]
    c, conn = parity.element_contributions(om, _same(u, dtype))
    sc = parity.node_scale(m.n_nodes, conn, c)
    assert parity.per_node_excess(r.reshape(-1, m.dim), ro.reshape(-1, m.dim), sc, TOL[dtype]) <= 1.0
    if mask_out:
        assert np.all(r[m.dirichlet.ravel() == 1] == 0)
    assert gm.sync_status() == 0


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("mask_in,mask_out", [(True, True), (False, True), (False, False)])
def test_hvp(case, dtype, mask_in, mask_out):
    name, m, gm, om, u, v = case
    vkv = torch.zeros(1, dtype=torch.float64, device="cuda")
    y = gm.hvp(_t(u, dtype), _t(v, dtype), mask_in=mask_in, mask_out=mask_out, vkv=vkv)
    u, v = _same(u, dtype), _same(v, dtype)
    yo = om.hvp(u, v, mask_in=mask_in, mask_out=mask_out)
    assert _rel(y.cpu().numpy(), yo) <= TOL[dtype]
    vm = np.where(m.dirichlet.ravel() == 1, 0.0, v) if mask_in else v
    c, conn = parity.element_contributions(om, u, vm)
    sc = parity.node_scale(m.n_nodes, conn, c)
    assert parity.per_node_excess(y.cpu().numpy().reshape(-1, m.dim), yo.reshape(-1, m.dim), sc, TOL[dtype]) <= 1.0
    ref = vm @ om.hvp(u, vm, mask_in=False, mask_out=False)
    assert abs(vkv.item() - ref) <= TOL[dtype] * abs(ref) * 10
    # without the fused vKv (the FP32 P1 call then runs the pair kernel)
    y2 = gm.hvp(_t(u, dtype), _t(v, dtype), mask_in=mask_in, mask_out=mask_out).cpu().numpy()
    assert _rel(y2, yo) <= TOL[dtype]
    assert parity.per_node_excess(y2.reshape(-1, m.dim), yo.reshape(-1, m.dim), sc, TOL[dtype]) <= 1.0
    assert gm.sync_status() == 0


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_block_diag(case, dtype):
    name, m, gm, om, u, v = case
    D = gm.block_diag(_t(u, dtype)).cpu().numpy().reshape(m.n_nodes, m.dim, m.dim)
    Do = om.block_diag(_same(u, dtype))
    assert _rel(D, Do) <= TOL[dtype]
    np.testing.assert_array_equal(D, np.swapaxes(D, 1, 2))


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_param_vjp(case, dtype):
    name, m, gm, om, u, v = case
    gmu, glam = gm.param_vjp(_t(u, dtype), _t(v, dtype))
    omu, olam = om.param_vjp(_same(u, dtype), _same(v, dtype))
    assert _rel(gmu.cpu().numpy(), omu) <= TOL[dtype]
    assert _rel(glam.cpu().numpy(), olam) <= TOL[dtype]


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_bitwise_reproducible(case, dtype):
    name, m, gm, om, u, v = case
    ut, vt = _t(u, dtype), _t(v, dtype)
    r1, r2 = gm.residual(ut), gm.residual(ut)
    y1, y2 = gm.hvp(ut, vt), gm.hvp(ut, vt)
    e1, e2 = gm.energy(ut), gm.energy(ut)
    assert torch.equal(r1, r2) and torch.equal(y1, y2) and torch.equal(e1, e2)


@pytest.mark.parametrize("kind", ["tet", "tri"])
def test_large_deformation_f32(kind):
    """|J - 1| spans both sides of 3/8, where the FP32 logarithm switches from
    its series to the library function."""
    from paper_2602_12365_b300.fem import Mesh
    m = mg.workload_tet(8, seed=1) if kind == "tet" else _jitter(mg.workload_tri(24), 0.2, 3)
    gm = Mesh.from_fixture(m, tile_elems=128)
    om = oracle.OracleMesh.from_mesh(m)
    u = mg.smooth_state(m, 0.5, amp=0.07).ravel()
    v = mg.random_direction(m, 2).ravel()
    Xe = m.coords[m.conn]
    ue = u.reshape(-1, m.dim)[m.conn]
    if m.dim == 3:
        J = np.linalg.det(np.linalg.solve(np.stack([Xe[:, k] - Xe[:, 3] for k in range(3)], 2).transpose(0, 2, 1),
                                          np.stack([Xe[:, k] + ue[:, k] - Xe[:, 3] - ue[:, 3] for k in range(3)], 2).transpose(0, 2, 1)))
    else:
        J = np.linalg.det(np.linalg.solve(np.stack([Xe[:, k] - Xe[:, 2] for k in range(2)], 2).transpose(0, 2, 1),
                                          np.stack([Xe[:, k] + ue[:, k] - Xe[:, 2] - ue[:, 2] for k in range(2)], 2).transpose(0, 2, 1)))
    assert J.min() > 0 and np.abs(J - 1).max() > 0.375 and np.abs(J - 1).min() < 0.375
    dt = torch.float32
    ur, vr = _same(u, dt), _same(v, dt)
    e = gm.energy(_t(u, dt)).cpu().numpy()
    assert abs(e[0] - om.energy(ur)) <= 1e-5 * abs(om.energy(ur))
    assert _rel(gm.residual(_t(u, dt)).cpu().numpy(), om.residual(ur)) <= 1e-5
    assert _rel(gm.hvp(_t(u, dt), _t(v, dt)).cpu().numpy(), om.hvp(ur, vr)) <= 1e-5
    assert gm.sync_status() == 0


# ---------------------------------------------------------------------------
# edge cases
# ---------------------------------------------------------------------------
def test_single_tile_and_orphan_node():
    from paper_2602_12365_b300.fem import Mesh
    m = mg.tet_mesh(1)
    coords = np.vstack([m.coords, [[2.0, 2.0, 2.0]]])  # node 8 belongs to no element
    mask = np.zeros((9, 3), np.uint8)
    mask[0] = 1
    gm = Mesh(m.elem_type, coords, m.conn, dirichlet=mask, precision="fp64")
    om = oracle.OracleMesh(m.elem_type, coords, m.conn, np.ones(6), np.full(6, 10.0), mask)
    rng = np.random.default_rng(0)
    u = 0.05 * rng.standard_normal(27)
    v = rng.standard_normal(27)
    ut = _t(u, torch.float64)
    r = gm.residual(ut).cpu().numpy()
    y = gm.hvp(ut, _t(v, torch.float64)).cpu().numpy()
    assert _rel(r, om.residual(u)) <= 1e-12
    assert _rel(y, om.hvp(u, v)) <= 1e-12
    assert np.all(r[24:] == 0) and np.all(y[24:] == 0)
    D = gm.block_diag(ut).cpu().numpy().reshape(9, 3, 3)
    np.testing.assert_array_equal(D[8], np.eye(3))


def test_rest_state_is_exact():
    from paper_2602_12365_b300.fem import Mesh
    m = mg.workload_tet(5, seed=1)
    gm = Mesh.from_fixture(m, tile_elems=100)
    for dt in (torch.float64, torch.float32):
        z = torch.zeros(m.n_nodes * 3, dtype=dt, device="cuda")
        assert gm.energy(z)[0].item() == 0.0
        assert torch.count_nonzero(gm.residual(z)).item() == 0


def test_inverted_element_flags_and_infinite_energy():
    from paper_2602_12365_b300.fem import Mesh
    m = mg.workload_tet(4, seed=1)
    gm = Mesh.from_fixture(m, tile_elems=64)
    u = np.zeros((m.n_nodes, 3))
    centre = np.argmin(np.linalg.norm(m.coords - 0.5, axis=1))
    u[centre] = [0.6, 0.6, 0.6]   # pushes the node through its neighbours
    for dt in (torch.float64, torch.float32):
        e = gm.energy(_t(u.ravel(), dt)).cpu().numpy()
        assert np.isinf(e[0]) and e[2] > 0
        assert gm.sync_status() & 1
        gm.residual(_t(u.ravel(), dt))
        assert gm.sync_status() & 1
    assert gm.sync_status() == 0  # cleared


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("kind", ["tri", "tet"])
def test_nonfinite_input_flagged(kind, dtype):
    from paper_2602_12365_b300.fem import Mesh
    m = mg.workload_tri(6) if kind == "tri" else mg.workload_tet(3, seed=1)
    gm = Mesh.from_fixture(m)
    u = np.zeros(m.n_nodes * m.dim)
    u[7] = np.nan
    gm.residual(_t(u, dtype))
    assert gm.sync_status() & 2
    gm.hvp(_t(np.zeros_like(u), dtype), _t(u, dtype), mask_in=False)
    assert gm.sync_status() & 2


def test_bad_mesh_rejected():
    from paper_2602_12365_b300.fem import Mesh
    from paper_2602_12365_b300._lib import FemError
    m = mg.tet_mesh(2)
    conn = m.conn.copy()
    conn[3, [1, 2]] = conn[3, [2, 1]]  # flip one tetrahedron
    with pytest.raises(FemError, match="BADMESH"):
        Mesh(m.elem_type, m.coords, conn)


def test_f32_on_fp64_mesh_is_refused():
    from paper_2602_12365_b300.fem import Mesh
    from paper_2602_12365_b300._lib import FemError
    m = mg.workload_tri(4)
    gm = Mesh.from_fixture(m, precision="fp64")
    with pytest.raises(FemError, match="ARG"):
        gm.residual(torch.zeros(m.n_nodes * 2, dtype=torch.float32, device="cuda"))


# ---------------------------------------------------------------------------
# full-size workloads, sampled
# ---------------------------------------------------------------------------
def _incident_submesh(m, nodes):
    hit = np.isin(m.conn, nodes).any(axis=1)
    els = np.flatnonzero(hit)
    sub_nodes, inv = np.unique(m.conn[els], return_inverse=True)
    conn = inv.reshape(-1, m.conn.shape[1]).astype(np.int32)
    om = oracle.OracleMesh(m.elem_type, m.coords[sub_nodes], conn, m.mu_e()[els], m.lam_e()[els],
                           np.zeros((len(sub_nodes), m.dim), np.uint8))
    return om, sub_nodes


def _sampled_check(m, gm, dtype, n_sample=400, seed=0):
    d = m.dim
    u = mg.smooth_state(m, 0.5)
    v = mg.random_direction(m, 1)
    ut, vt = _t(u.ravel(), dtype), _t(v.ravel(), dtype)
    r = gm.residual(ut).cpu().numpy().reshape(-1, d)
    y = gm.hvp(ut, vt).cpu().numpy().reshape(-1, d)
    e = gm.energy(ut).cpu().numpy()
    assert gm.sync_status() == 0 and e[2] == 0
    u = _same(u, dtype)
    v = _same(v, dtype)
    rng = np.random.default_rng(seed)
    nodes = np.unique(np.concatenate([rng.choice(m.n_nodes, n_sample, replace=False),
                                      [0, m.n_nodes - 1]]))
    om, sub = _incident_submesh(m, nodes)
    pos = np.searchsorted(sub, nodes)
    mask = m.dirichlet[nodes].astype(bool)
    ro = om.residual(u[sub].ravel(), mask_out=False).reshape(-1, d)[pos]
    ro[mask] = 0
    vm = np.where(m.dirichlet.astype(bool), 0.0, v)
    yo = om.hvp(u[sub].ravel(), vm[sub].ravel(), mask_in=False, mask_out=False).reshape(-1, d)[pos]
    yo[mask] = 0
    assert _rel(r[nodes], ro) <= TOL[dtype]
    assert _rel(y[nodes], yo) <= TOL[dtype]
    # node by node against the size of the incident elements' contributions
    els = np.flatnonzero(np.isin(m.conn, nodes).any(axis=1))
    cr, conn = parity.element_contributions(om_full_view(m), u.ravel(), None, els)
    cy, _ = parity.element_contributions(om_full_view(m), u.ravel(), vm.ravel(), els)
    sr = parity.node_scale(m.n_nodes, conn, cr)
    sy = parity.node_scale(m.n_nodes, conn, cy)
    assert parity.per_node_excess(r[nodes], ro, sr, TOL[dtype], nodes) <= 1.0
    assert parity.per_node_excess(y[nodes], yo, sy, TOL[dtype], nodes) <= 1.0
    return e


def om_full_view(m):
    """The whole mesh as the oracle sees it (element data only are read)."""
    return oracle.OracleMesh(m.elem_type, m.coords, m.conn, m.mu_e(), m.lam_e(), None)


def test_full_size_tet_64(tmp_path):
    from paper_2602_12365_b300.fem import Mesh
    m = mg.workload_tet(64, seed=0)
    gm = Mesh.from_fixture(m)
    info = gm.info()
    assert info["n_elems"] == 1_572_864 and info["n_nodes"] == 274_625
    _sampled_check(m, gm, torch.float32)
    _sampled_check(m, gm, torch.float64, n_sample=100)


def test_full_size_hex_128():
    from paper_2602_12365_b300.fem import Mesh
    m = mg.workload_hex(128, seed=0)
    gm = Mesh.from_fixture(m)
    assert gm.info()["n_elems"] == 2_097_152
    _sampled_check(m, gm, torch.float32, n_sample=200)
    _sampled_check(m, gm, torch.float64, n_sample=100, seed=1)


@pytest.mark.parametrize("name", ["tet", "tet_rand", "hex", "tri"])
def test_mixed_error_at_the_fp64_state(name):
    """The FP32 path fed the FP64 state (u, v rounded to FP32 on the way in)
    against the FP64 oracle at the unrounded state.  Its error is the
    kernel's (bounded by 1e-5 at the rounded inputs, tested above) plus what
    the input rounding itself moves the exact result, which the oracle
    measures: ||x_ora(u32) - x_ora(u)||.  The test holds the total to that
    sum; bench.py reports the same figures on the benchmark workload."""
    from paper_2602_12365_b300.fem import Mesh
    build, tile = CASES[name]
    m = build()
    gm = Mesh.from_fixture(m, precision="mixed", tile_elems=tile)
    om = oracle.OracleMesh.from_mesh(m)
    u = mg.smooth_state(m, 0.5).ravel()
    v = mg.random_direction(m, seed=1).ravel()
    u32, v32 = _same(u, torch.float32), _same(v, torch.float32)
    r = gm.residual(_t(u, torch.float32)).cpu().numpy()
    y = gm.hvp(_t(u, torch.float32), _t(v, torch.float32)).cpu().numpy()
    ro, ro32 = om.residual(u), om.residual(u32)
    yo, yo32 = om.hvp(u, v), om.hvp(u32, v32)
    in_r = np.linalg.norm(ro32 - ro) / np.linalg.norm(ro)
    in_y = np.linalg.norm(yo32 - yo) / np.linalg.norm(yo)
    assert _rel(r, ro) <= 1e-5 + in_r
    assert _rel(y, yo) <= 1e-5 + in_y
    assert gm.sync_status() == 0


def test_unknown_flag_bits_are_rejected():
    """Only FEM_MASK_IN / FEM_MASK_OUT reach the kernels from the public calls."""
    import ctypes as C
    from paper_2602_12365_b300 import _lib as L
    from paper_2602_12365_b300._lib import FemError
    from paper_2602_12365_b300.fem import Mesh
    m = mg.workload_tet(2)
    gm = Mesh.from_fixture(m)
    u = torch.zeros(m.n_nodes * 3, dtype=torch.float32, device="cuda")
    v, y = torch.ones_like(u), torch.empty_like(u)
    for bit in (1 << 2, 1 << 16, 1 << 17, 1 << 18):
        with pytest.raises(FemError, match="flags"):
            L.check(L.lib().fem_hvp(gm._h, L.FEM_F32, C.c_void_p(u.data_ptr()), C.c_void_p(v.data_ptr()),
                                    C.c_void_p(y.data_ptr()), C.c_uint32(3 | bit), None, None))
        with pytest.raises(FemError, match="flags"):
            L.check(L.lib().fem_residual(gm._h, L.FEM_F32, C.c_void_p(u.data_ptr()), C.c_void_p(y.data_ptr()),
                                         C.c_uint32(1 | bit), None))
    gm.hvp(u, v, out=y)  # the handle still works
    assert gm.sync_status() == 0
