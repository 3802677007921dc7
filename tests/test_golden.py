"""Stored fixtures of tests/golden: the colour counts App. A prints, and
oracle outputs on tiny seeded meshes (written by tests/golden/make_golden.py,
which calls only the oracle).

CPU: the oracle reproduces its stored outputs (a guard against a silent
change of the oracle's arithmetic), and the library's and the oracle's
greedy distance-2 colourings give App. A's colour counts on 3D meshes.
GPU: the FP64 path matches the stored oracle outputs within 1e-12.
"""
import glob
import json
import os

import numpy as np
import pytest

import oracle
from paper_2602_12365_b300 import meshgen as mg
from paper_2602_12365_b300.fem import sparse_pattern_host

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
CASES = sorted(os.path.basename(p)[:-5] for p in glob.glob(os.path.join(GOLDEN, "*_*x*.json")))


def _load(name):
    with open(os.path.join(GOLDEN, name + ".json")) as f:
        return json.load(f)


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


def test_fixtures_present():
    assert CASES == ["hex8_lognormal_2x2x2", "tet4_jittered_2x2x2", "tri3_plane_strain_3x3"]


@pytest.mark.parametrize("name", CASES)
def test_oracle_reproduces_fixture(name):
    d = _load(name)
    om = oracle.OracleMesh(d["elem_type"], np.array(d["coords"]), np.array(d["conn"]), np.array(d["mu"]),
                           np.array(d["lam"]), np.array(d["dirichlet"], np.uint8))
    u, v = np.array(d["u"]), np.array(d["v"])
    psi, _, S, st = om.energy(u, per_element=True)
    assert st == 0
    assert abs(psi - d["energy"]) <= 1e-14 * S and abs(S - d["energy_scale"]) <= 1e-14 * S
    assert _rel(om.residual(u), d["residual"]) <= 1e-14
    assert _rel(om.hvp(u, v), d["hvp"]) <= 1e-14
    assert _rel(om.block_diag(u).ravel(), d["block_diag"]) <= 1e-14
    # the fixture is not trivial: a non-zero state, masked rows present
    assert np.abs(u).max() > 0 and np.array(d["dirichlet"]).any() and np.abs(d["residual"]).max() > 0


@pytest.mark.parametrize("kind", ["tet", "hex"])
def test_app_a_colour_counts_3d(kind):
    rng_ = _load("app_a_colour_counts")["3d_tet4_hex8_colours"]
    m = mg.workload_tet(16, seed=3) if kind == "tet" else mg.workload_hex(8)
    _, _, _, nc_lib = sparse_pattern_host(m.elem_type, m.coords, m.conn)
    ptr, idx = oracle.dof_pattern(m.n_nodes, m.dim, m.conn)
    _, nc_ora = oracle.distance2_colors(ptr, idx)
    assert nc_lib == nc_ora and rng_[0] <= nc_lib <= rng_[1]


def test_app_a_colour_bound_2d():
    lo, hi = _load("app_a_colour_counts")["2d_tri3_quad4_max_colours"]
    m = mg.workload_tri(32)
    _, _, _, nc = sparse_pattern_host(m.elem_type, m.coords, m.conn)
    assert nc <= hi


@pytest.mark.gpu
@pytest.mark.parametrize("name", CASES)
def test_cuda_fp64_matches_fixture(name):
    import torch
    from paper_2602_12365_b300.fem import Mesh
    d = _load(name)
    dim = len(d["coords"][0])
    gm = Mesh(d["elem_type"], np.array(d["coords"]), np.array(d["conn"], np.int32), np.array(d["mu"]),
              np.array(d["lam"]), dirichlet=np.array(d["dirichlet"], np.uint8), precision="fp64")
    u = torch.tensor(d["u"], dtype=torch.float64, device="cuda")
    v = torch.tensor(d["v"], dtype=torch.float64, device="cuda")
    e = gm.energy(u).cpu().numpy()
    S = d["energy_scale"]
    assert abs(e[0] - d["energy"]) <= 1e-12 * S and abs(e[1] - S) <= 1e-12 * S
    assert _rel(gm.residual(u).cpu().numpy(), d["residual"]) <= 1e-12
    assert _rel(gm.hvp(u, v).cpu().numpy(), d["hvp"]) <= 1e-12
    assert _rel(gm.block_diag(u).cpu().numpy(), d["block_diag"]) <= 1e-12
    assert gm.n_dofs == len(d["u"]) == gm.n_nodes * dim
    assert gm.sync_status() == 0
