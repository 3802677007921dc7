"""The atomic scatter-add ablation (fem_residual_atomic / fem_hvp_atomic)
against the oracle and the tiled, coloured kernels.

Bars as for the tiled kernels: FP64 within 1e-12 and FP32 within 1e-5 of the
oracle (relative, 2-norm).  Determinism: the tiled kernels repeat bit for
bit; the atomic ones are only checked to agree to rounding between runs (the
order of their additions is not fixed; how many bits differ is reported).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2602_12365_b300 import meshgen as mg
from paper_2602_12365_b300._lib import FemError
from paper_2602_12365_b300.fem import Mesh

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("kind,n", [("tri", 6), ("tet", 4)])
@pytest.mark.parametrize("precision,dt,tol", [("fp64", torch.float64, 1e-12), ("mixed", torch.float32, 1e-5)])
def test_atomic_matches_oracle(kind, n, precision, dt, tol):
    m = (mg.workload_tri(n) if kind == "tri" else mg.workload_tet(n, seed=2, random_moduli=2))
    gm = Mesh.from_fixture(m, precision=precision)
    om = oracle.OracleMesh.from_mesh(m)
    u = torch.as_tensor(mg.smooth_state(m, 0.5, amp=0.05).ravel(), dtype=dt, device="cuda")
    v = torch.as_tensor(mg.random_direction(m, 3).ravel(), dtype=dt, device="cuda")
    u64, v64 = u.double().cpu().numpy(), v.double().cpu().numpy()
    r = gm.residual_atomic(u).double().cpu().numpy()
    assert _rel(r, om.residual(u64, mask_out=True)) <= tol
    y = gm.hvp_atomic(u, v).double().cpu().numpy()
    assert _rel(y, om.hvp(u64, v64)) <= tol
    y0 = gm.hvp_atomic(u, v, mask_in=False, mask_out=False).double().cpu().numpy()
    assert _rel(y0, om.hvp(u64, v64, mask_in=False, mask_out=False)) <= tol


def test_determinism_tiled_vs_atomic():
    m = mg.workload_tet(32)
    gm = Mesh.from_fixture(m)
    u = torch.as_tensor(mg.smooth_state(m, 0.5).ravel(), dtype=torch.float32, device="cuda")
    v = torch.as_tensor(mg.random_direction(m, 1).ravel(), dtype=torch.float32, device="cuda")
    tiled = [gm.hvp(u, v) for _ in range(4)]
    assert all(torch.equal(tiled[0], t) for t in tiled[1:])  # bit for bit
    atomic = [gm.hvp_atomic(u, v) for _ in range(4)]
    scale = torch.linalg.norm(tiled[0]).item()
    for a in atomic:
        assert torch.linalg.norm(a - tiled[0]).item() <= 1e-5 * scale
    differing = max(int((a != atomic[0]).sum()) for a in atomic[1:])
    print(f"atomic HVP: up to {differing} of {u.numel()} entries differ between runs")


def test_ablation_rejects_hex_and_bad_dtype():
    m = mg.workload_hex(2)
    gm = Mesh.from_fixture(m)
    u = torch.zeros(m.n_nodes * 3, dtype=torch.float32, device="cuda")
    with pytest.raises(FemError, match="P1"):
        gm.hvp_atomic(u, u.clone())
    mt = mg.workload_tet(2)
    g64 = Mesh.from_fixture(mt, precision="fp64")
    with pytest.raises(FemError):
        g64.residual_atomic(torch.zeros(mt.n_nodes * 3, dtype=torch.float32, device="cuda"))


@pytest.mark.parametrize("precision,dt,tol", [("fp64", torch.float64, 1e-12), ("mixed", torch.float32, 1e-5)])
@pytest.mark.parametrize("masked", [False, True])
def test_atomic_assembly_matches_algorithm_2(precision, dt, tol, masked):
    m = mg.workload_tet(5, seed=3, random_moduli=3)
    gm = Mesh.from_fixture(m, precision=precision)
    u = torch.as_tensor(mg.smooth_state(m, 0.5, amp=0.05).ravel(), dtype=dt, device="cuda")
    ref = gm.sparse_assemble(u, mask_in=masked, mask_out=masked)
    got = gm.sparse_assemble_atomic(u, mask_in=masked, mask_out=masked)
    assert (torch.linalg.norm(got - ref) / torch.linalg.norm(ref)).item() <= tol
    assert gm.sync_status() == 0
