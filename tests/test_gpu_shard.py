"""The sharded residual and HVP with the library's kernels, ranks emulated
one after another on one GPU (the halo sum done in-process by
`shard.halo_sum_local`, which performs the additions `shard.halo_sum` does on
each rank): equal to the whole-mesh calls to rounding (FP64 1e-12, FP32
1e-5 relative) and bitwise the same on every rank at shared nodes."""
import numpy as np
import pytest
import torch

from paper_2602_12365_b300 import meshgen as mg
from paper_2602_12365_b300 import shard as sh
from paper_2602_12365_b300.fem import Mesh

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision,dt,tol", [("fp64", torch.float64, 1e-12), ("mixed", torch.float32, 1e-5)])
@pytest.mark.parametrize("world", [2, 4])
def test_sharded_calls_equal_whole_mesh(precision, dt, tol, world):
    m = mg.workload_tet(12, seed=2, random_moduli=2)
    u = mg.smooth_state(m, 0.5, amp=0.05).ravel()
    v = mg.random_direction(m, 3).ravel()
    g = Mesh.from_fixture(m, precision=precision)
    ut, vt = torch.as_tensor(u, dtype=dt, device="cuda"), torch.as_tensor(v, dtype=dt, device="cuda")
    r_full, y_full = g.residual(ut), g.hvp(ut, vt)
    shards = sh.partition(m, world)
    rp, yp = [], []
    for s in shards:
        gs = Mesh.from_fixture(sh.submesh(m, s), precision=precision)
        idx = torch.as_tensor((s.nodes[:, None] * 3 + np.arange(3)).ravel(), device="cuda")
        rp.append(gs.residual(ut[idx]))
        yp.append(gs.hvp(ut[idx], vt[idx]))
    ra, ya = sh.halo_sum_local(rp, shards), sh.halo_sum_local(yp, shards)
    seen = {}
    for s, r, y in zip(shards, ra, ya):
        idx = torch.as_tensor((s.nodes[:, None] * 3 + np.arange(3)).ravel(), device="cuda")
        for got, want in ((r, r_full[idx]), (y, y_full[idx])):
            assert (torch.linalg.norm(got - want) / torch.linalg.norm(want)).item() <= tol
        rc, yc = r.view(-1, 3).cpu().numpy(), y.view(-1, 3).cpu().numpy()
        for k, n in enumerate(s.nodes):
            vals = (rc[k].tobytes(), yc[k].tobytes())
            assert seen.setdefault(int(n), vals) == vals
