"""fem_energy_static against fem_energy.

fem_energy_static runs the energy kernel with its reduction scratch (arrival
counter and per-tile partials) in a fixed module-scope device array instead of
the handle's workspace.  Same kernel, same fixed summation order, so its
output must equal fem_energy's bit for bit, on two calls in a row (the second
call sees the counter the first one left) and after any other call made
earlier in the process.  The file name keeps it last in collection so that it
also runs after the rest of the suite; it passes on its own as well.
"""
import numpy as np
import pytest
import torch

from paper_2602_12365_b300 import meshgen as mg
from paper_2602_12365_b300._lib import FemError
from paper_2602_12365_b300.fem import Mesh

pytestmark = pytest.mark.gpu

STATIC_MAX_TILES = 16384  # FEM_STATIC_MAX_TILES in include/fem_b300.h


def _states(m, dtype):
    s1 = torch.as_tensor(mg.smooth_state(m, 0.5).ravel(), dtype=dtype, device="cuda")
    s2 = torch.as_tensor(mg.smooth_state(m, 1.5, amp=0.05).ravel(), dtype=dtype, device="cuda")
    return s1, s2


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("kind", ["tet", "hex", "tri"])
def test_static_equals_energy_on_consecutive_calls(kind, dtype):
    m = {"tet": lambda: mg.workload_tet(10, seed=5),
         "hex": lambda: mg.workload_hex(8, seed=6),
         "tri": lambda: mg.workload_tri(48)}[kind]()
    gm = Mesh.from_fixture(m, tile_elems=96)
    assert gm.info()["n_tiles"] > 1
    for u in _states(m, dtype):
        ref = gm.energy(u).clone()
        a = gm.energy_static(u).clone()
        b = gm.energy_static(u).clone()
        torch.cuda.synchronize()
        assert torch.isfinite(ref[0])
        assert torch.equal(a, ref), (a, ref)
        assert torch.equal(b, ref), (b, ref)
    assert gm.sync_status() == 0


def test_static_near_the_tile_limit():
    m = mg.workload_tri(180)
    gm = Mesh.from_fixture(m, tile_elems=4)
    n_tiles = gm.info()["n_tiles"]
    assert STATIC_MAX_TILES - 512 < n_tiles <= STATIC_MAX_TILES
    u, _ = _states(m, torch.float64)
    ref = gm.energy(u).clone()
    got = [gm.energy_static(u).clone() for _ in range(2)]
    torch.cuda.synchronize()
    for g in got:
        assert torch.equal(g, ref)
    assert gm.sync_status() == 0


def test_static_inverted_state_matches():
    m = mg.workload_tet(6, seed=7)
    gm = Mesh.from_fixture(m)
    x = m.coords
    u = np.zeros_like(x)
    u[:, 2] = -2.0 * x[:, 2]  # z -> -z: every J < 0
    ut = torch.as_tensor(u.ravel(), device="cuda")
    ref = gm.energy(ut).clone()
    got = gm.energy_static(ut).clone()
    torch.cuda.synchronize()
    assert torch.isinf(ref[0]) and ref[2].item() > 0
    assert torch.equal(got, ref)
    gm.sync_status()  # clears the inverted flag both calls raised


def test_static_rejects_a_mesh_over_the_limit():
    m = mg.workload_tri(184)
    gm = Mesh.from_fixture(m, tile_elems=4)
    assert gm.info()["n_tiles"] > STATIC_MAX_TILES
    u, _ = _states(m, torch.float64)
    out = torch.full((4,), 7.0, dtype=torch.float64, device="cuda")
    with pytest.raises(FemError, match=str(STATIC_MAX_TILES)):
        gm.energy_static(u, out=out)
    torch.cuda.synchronize()
    assert torch.equal(out, torch.full_like(out, 7.0))  # nothing enqueued
    # the regular entry point still serves this mesh
    assert torch.isfinite(gm.energy(u)[0])


def test_static_rejects_a_bad_dtype_before_touching_the_shared_array():
    # An FP32 call on a mesh built without FP32 records is refused before it
    # touches the shared array: a static call of another handle queued just
    # before it on the same stream keeps its arrival counter and its result.
    m = mg.workload_tet(6, seed=8)
    g64 = Mesh.from_fixture(m, precision="fp64", tile_elems=64)
    gmx = Mesh.from_fixture(m, tile_elems=64)
    u64, _ = _states(m, torch.float64)
    ref = gmx.energy(u64).clone()
    torch.cuda.synchronize()
    first = gmx.energy_static(u64)  # queued, not yet synchronised
    with pytest.raises(FemError, match="FEM_F32"):
        g64.energy_static(u64.float())
    second = gmx.energy_static(u64)
    torch.cuda.synchronize()
    assert torch.equal(first, ref) and torch.equal(second, ref)
    assert g64.sync_status() == 0 and gmx.sync_status() == 0
