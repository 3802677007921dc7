"""Sparse K by colouring on the GPU (Algorithm 2) against the oracle.

Bars: FP64 values within 1e-12 of the oracle's K (relative, in the
Frobenius norm over the pattern; the values come from FP64 HVPs, so they
differ from the oracle's only by summation order); FP32 values within 1e-5
(FP32 element kernels).  The CSR product K v is checked against the GPU HVP
in the same precision (the HVP itself is pinned to the oracle elsewhere), at
small sizes and on the 64^3 benchmark mesh (K v = HVP(v) holds at any size).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2602_12365_b300 import meshgen as mg
from paper_2602_12365_b300._lib import FemError
from paper_2602_12365_b300.fem import Mesh, sparse_pattern_host

pytestmark = pytest.mark.gpu


def _state(m, seed=1):
    u = mg.smooth_state(m, 0.5, amp=0.05).ravel()
    return u + 0.002 * np.random.default_rng(seed).standard_normal(u.size)


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


CASES = [("tri", 4, {}), ("tet", 3, {"seed": 2, "random_moduli": 2}), ("hex", 2, {"seed": 1})]


@pytest.mark.parametrize("kind,n,kw", CASES)
@pytest.mark.parametrize("masked", [False, True])
def test_assemble_fp64_matches_oracle(kind, n, kw, masked):
    m = {"tri": mg.workload_tri, "tet": mg.workload_tet, "hex": mg.workload_hex}[kind](n, **kw)
    gm = Mesh.from_fixture(m, precision="fp64")
    u = _state(m)
    vals = gm.sparse_assemble(torch.as_tensor(u, device="cuda"), mask_in=masked, mask_out=masked)
    om = oracle.OracleMesh.from_mesh(m)
    ptr, idx, ref = om.sparse_K(u, mask_in=masked, mask_out=masked)
    rp, ci, co = gm.sparse_pattern()
    assert np.array_equal(rp, ptr) and np.array_equal(ci, idx)
    assert _rel(vals.cpu().numpy(), ref) <= 1e-12


@pytest.mark.parametrize("kind,n,kw", CASES)
def test_assemble_fp32_matches_oracle(kind, n, kw):
    m = {"tri": mg.workload_tri, "tet": mg.workload_tet, "hex": mg.workload_hex}[kind](n, **kw)
    gm = Mesh.from_fixture(m, precision="mixed")
    u32 = torch.as_tensor(_state(m), dtype=torch.float32, device="cuda")
    vals = gm.sparse_assemble(u32)
    om = oracle.OracleMesh.from_mesh(m)
    _, _, ref = om.sparse_K(u32.double().cpu().numpy())
    assert _rel(vals.double().cpu().numpy(), ref) <= 1e-5


def test_handle_pattern_equals_host_pattern():
    m = mg.workload_tet(6, seed=4)
    gm = Mesh.from_fixture(m)
    rp, ci, co = gm.sparse_pattern()
    rp2, ci2, co2, nc2 = sparse_pattern_host(m.elem_type, m.coords, m.conn)
    nnz, nc = gm.sparse_info()
    assert np.array_equal(rp, rp2) and np.array_equal(ci, ci2) and np.array_equal(co, co2)
    assert nnz == ci.size and nc == nc2 == co.max() + 1


@pytest.mark.parametrize("precision,dt,tol", [("fp64", torch.float64, 1e-12), ("mixed", torch.float32, 1e-5)])
def test_spmv_equals_hvp(precision, dt, tol):
    m = mg.workload_tet(5, seed=3, random_moduli=3)
    gm = Mesh.from_fixture(m, precision=precision)
    u = torch.as_tensor(_state(m), dtype=dt, device="cuda")
    vals = gm.sparse_assemble(u)
    for s in range(3):
        v = torch.as_tensor(np.random.default_rng(s).standard_normal(m.n_nodes * 3), dtype=dt, device="cuda")
        y = gm.sparse_spmv(vals, v)
        h = gm.hvp(u, v)
        assert (torch.linalg.norm(y - h) / torch.linalg.norm(h)).item() <= tol


def test_benchmark_mesh_properties():
    """The 64^3 tet mesh (C2): 80-90 colours (App. A), K v = HVP(v) in FP32,
    and K symmetric on sampled entries."""
    m = mg.workload_tet(64)
    gm = Mesh.from_fixture(m)
    nnz, nc = gm.sparse_info()
    n = 64
    E = 3 * n * (n + 1) ** 2 + 3 * n * n * (n + 1) + n ** 3
    assert nnz == 9 * ((n + 1) ** 3 + 2 * E) and 80 <= nc <= 90
    u = torch.as_tensor(mg.smooth_state(m, 0.5).ravel(), dtype=torch.float32, device="cuda")
    vals = gm.sparse_assemble(u)
    v = torch.as_tensor(mg.random_direction(m, 1).ravel(), dtype=torch.float32, device="cuda")
    y, h = gm.sparse_spmv(vals, v), gm.hvp(u, v)
    assert (torch.linalg.norm(y - h) / torch.linalg.norm(h)).item() <= 1e-5
    rp, ci, _ = gm.sparse_pattern()
    K = vals.cpu().numpy()
    rng = np.random.default_rng(0)
    rows = rng.integers(0, m.n_nodes * 3, 2000)
    scale = np.abs(K).max()
    for i in rows:
        for k in range(rp[i], rp[i + 1], 7):
            j = ci[k]
            kj = rp[j] + np.searchsorted(ci[rp[j]:rp[j + 1]], i)
            assert abs(K[k] - K[kj]) <= 1e-5 * scale


def test_arguments_are_checked():
    m = mg.workload_tet(2)
    gm = Mesh.from_fixture(m)
    u = torch.zeros(m.n_nodes * 3, dtype=torch.float32, device="cuda")
    vals = gm.sparse_assemble(u)
    with pytest.raises(FemError):
        gm.sparse_spmv(vals, u, out=u)  # x and y alias
    g64 = Mesh.from_fixture(m, precision="fp64")
    with pytest.raises(FemError):
        g64.sparse_assemble(u)  # FP32 on an FP64 mesh


@pytest.mark.parametrize("kind", ["tri", "tet", "hex"])
@pytest.mark.parametrize("dt", [torch.float64, torch.float32])
def test_spmv_matches_host_csr(kind, dt):
    """The CSR product against an FP64 CSR product on the host, entry by
    entry: |y_i - (K x)_i| <= tol sum_j |K_ij x_j|; also with the values at a
    4- or 8-byte offset from a 16-byte boundary."""
    import scipy.sparse as sps
    m = {"tri": mg.workload_tri(9), "tet": mg.workload_tet(3, seed=1), "hex": mg.workload_hex(3)}[kind]
    gm = Mesh.from_fixture(m, precision="fp64" if dt == torch.float64 else "mixed")
    rp, ci, _ = gm.sparse_pattern()
    rng = np.random.default_rng(5)
    vt = torch.as_tensor(rng.standard_normal(ci.size), dtype=dt, device="cuda")
    xt = torch.as_tensor(rng.standard_normal(m.n_nodes * m.dim), dtype=dt, device="cuda")
    K = sps.csr_matrix((vt.double().cpu().numpy(), ci, rp))
    x = xt.double().cpu().numpy()
    ref, scale = K @ x, abs(K) @ np.abs(x)
    buf = torch.zeros(ci.size + 1, dtype=dt, device="cuda")
    buf[1:] = vt
    mis = buf[1:]
    assert vt.data_ptr() % 16 == 0 and mis.data_ptr() % 16 != 0
    tol = 1e-12 if dt == torch.float64 else 1e-5
    for vals in (vt, mis):
        y = gm.sparse_spmv(vals, xt).double().cpu().numpy()
        assert np.all(np.abs(y - ref) <= tol * scale)
    assert gm.sync_status() == 0


def _jittered_hex(n, seed):
    m = mg.workload_hex(n, seed=seed)
    g = mg.grid_index(m)
    interior = np.all((g > 0) & (g < m.n), axis=1)
    rng = np.random.default_rng(seed)
    m.coords = m.coords.copy()
    m.coords[interior] += 0.15 / m.n * (2 * rng.random(m.coords[interior].shape) - 1)
    return m


@pytest.mark.parametrize("kind,n,tile", [("hex", 1, 0), ("hex", 4, 16), ("hex_jittered", 4, 16), ("tet", 1, 0),
                                         ("tet", 3, 40)])
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("mixed", 1e-5)])
def test_assemble_edge_plans_match_oracle(kind, n, tile, precision, tol):
    """Algorithm 2 through the stored linearisation on plans with a single
    element (one lane of one round) and with many small tiles (partial
    rounds, most nodes shared between tiles); Q1 on parallelepipeds and on a
    jittered grid (J varying between the Gauss points)."""
    m = {"hex": lambda: mg.workload_hex(n, seed=4), "hex_jittered": lambda: _jittered_hex(n, 4),
         "tet": lambda: mg.workload_tet(n, seed=4, random_moduli=4)}[kind]()
    gm = Mesh.from_fixture(m, precision=precision, tile_elems=tile)
    dt = torch.float64 if precision == "fp64" else torch.float32
    u = torch.as_tensor(_state(m), dtype=dt, device="cuda")
    vals = gm.sparse_assemble(u, mask_in=False, mask_out=False)
    om = oracle.OracleMesh.from_mesh(m)
    _, _, ref = om.sparse_K(u.double().cpu().numpy(), mask_in=False, mask_out=False)
    assert _rel(vals.double().cpu().numpy(), ref) <= tol
    assert gm.sync_status() == 0
