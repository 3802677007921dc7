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


def _solve_worker(rank, world, port, out):
    import os
    import sys
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    torch.cuda.set_device(0)
    m = mg.workload_tet(6, seed=3, random_moduli=3)
    s = sh.partition(m, world)[rank]
    sub = sh.submesh(m, s)
    mask = torch.as_tensor(sub.dirichlet.ravel().astype(bool))
    ubar = torch.as_tensor(sub.ubar.ravel())
    u = torch.zeros(s.n_local * 3, dtype=torch.float64)
    ops = sh.LibraryRankOps(sub)
    sts = [sh.sharded_load_step(ops, s, mask, ubar, 0.0, 0.05, u),
           sh.sharded_load_step(ops, s, mask, ubar, 0.05, 0.1, u)]
    out[rank] = (s.nodes, u.numpy().copy(), sts)
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_load_steps_with_the_library(world):
    """Two Newton-CG load steps of the sharded solver (shard.sharded_load_step)
    on gloo ranks, each rank's element work the library's FP64 kernels on its
    submesh (the ranks are processes sharing this GPU; the exchange is
    host-driven, so no kernel waits for another rank): the displacements
    equal fem_newton_step on the whole mesh to 1e-10, bitwise the same on
    every rank holding a node."""
    import socket

    import torch.multiprocessing as mp
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    out = mp.Manager().dict()
    mp.spawn(_solve_worker, args=(world, port, out), nprocs=world, join=True)
    m = mg.workload_tet(6, seed=3, random_moduli=3)
    g = Mesh.from_fixture(m, precision="fp64")
    ubar = torch.as_tensor(m.ubar.ravel(), dtype=torch.float64, device="cuda")
    uw = torch.zeros(m.n_nodes * 3, dtype=torch.float64, device="cuda")
    for a, b in ((0.0, 0.05), (0.05, 0.1)):
        assert g.newton_step(uw, ubar, a, b)["status"] == 0
    uw = uw.cpu().numpy()
    seen = {}
    for rank in range(world):
        nodes, u, sts = out[rank]
        assert all(st["status"] == 0 for st in sts)
        idx = (nodes[:, None] * 3 + np.arange(3)).ravel()
        assert np.linalg.norm(u - uw[idx]) <= 1e-10 * np.linalg.norm(uw[idx])
        for k, n in enumerate(nodes):
            vals = u[3 * k:3 * k + 3].tobytes()
            assert seen.setdefault(int(n), vals) == vals
    assert len(seen) == m.n_nodes
