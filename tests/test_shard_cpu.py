"""Element sharding and the halo sum (the multi-GPU layout) on CPU ranks.

Each gloo rank evaluates its slab's residual and HVP with the oracle on its
submesh (standing in for the GPU kernels), then `shard.halo_sum` exchanges
the interface partials with its neighbours.  The assembled vectors must
equal the whole-mesh oracle on every local node, be bitwise the same on all
ranks at shared nodes, and the owned-node dot product must equal the
whole-mesh one.
"""
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2602_12365_b300 import meshgen as mg
from paper_2602_12365_b300 import shard as sh

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _case(kind):
    if kind == "tet":
        m = mg.workload_tet(4, seed=1, random_moduli=1)
    else:
        m = mg.workload_tri(8)
    u = mg.smooth_state(m, 0.5, amp=0.05).ravel()
    v = mg.random_direction(m, 2).ravel()
    return m, u, v


@pytest.mark.parametrize("kind,world", [("tet", 2), ("tet", 3), ("tri", 4)])
def test_partition_covers_the_mesh(kind, world):
    m, _, _ = _case(kind)
    shards = sh.partition(m, world)
    allel = np.sort(np.concatenate([s.elems for s in shards]))
    assert np.array_equal(allel, np.arange(m.n_el))  # every element once
    owned = np.zeros(m.n_nodes, int)
    for s in shards:
        assert np.array_equal(s.nodes, np.unique(m.conn[s.elems]))
        owned[s.nodes[s.owned]] += 1
        for q, idx in s.iface.items():  # symmetric interfaces, same global order
            assert np.array_equal(s.nodes[idx], shards[q].nodes[shards[q].iface[s.rank]])
    assert np.all(owned == 1)  # every node owned once
    sizes = [s.elems.size for s in shards]
    assert max(sizes) - min(sizes) <= 1


def _worker(rank, world, port, kind, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    import oracle
    dist.init_process_group("gloo", rank=rank, world_size=world)
    m, u, v = _case(kind)
    s = sh.partition(m, world)[rank]
    sub = sh.submesh(m, s)
    om = oracle.OracleMesh.from_mesh(sub)
    idx = (s.nodes[:, None] * m.dim + np.arange(m.dim)).ravel()
    r = torch.as_tensor(om.residual(u[idx]))
    y = torch.as_tensor(om.hvp(u[idx], v[idx]))
    ra, ya = sh.halo_sum(r, s), sh.halo_sum(y, s)
    out[rank] = (s.nodes, ra.numpy(), ya.numpy(), sh.dot(ra, ra, s), sh.dot(ra, ya, s))
    dist.destroy_process_group()


@pytest.mark.parametrize("kind,world", [("tet", 2), ("tet", 3), ("tri", 2)])
def test_halo_sum_on_gloo_ranks(kind, world):
    import oracle
    out = mp.Manager().dict()
    mp.spawn(_worker, args=(world, _free_port(), kind, out), nprocs=world, join=True)
    m, u, v = _case(kind)
    om = oracle.OracleMesh.from_mesh(m)
    r, y = om.residual(u), om.hvp(u, v)
    d = m.dim
    seen = {}
    for rank in range(world):
        nodes, ra, ya, rr, ry = out[rank]
        idx = (nodes[:, None] * d + np.arange(d)).ravel()
        np.testing.assert_allclose(ra, r[idx], rtol=0, atol=1e-13 * np.abs(r).max())
        np.testing.assert_allclose(ya, y[idx], rtol=0, atol=1e-13 * np.abs(y).max())
        assert rr == pytest.approx(r @ r, rel=1e-13) and ry == pytest.approx(r @ y, rel=1e-13)
        for k, n in enumerate(nodes):  # the same bits on every rank holding a node
            key = int(n)
            vals = (ra[k * d:(k + 1) * d].tobytes(), ya[k * d:(k + 1) * d].tobytes())
            assert seen.setdefault(key, vals) == vals


def test_partition_rejects_more_ranks_than_elements():
    m = mg.workload_tet(1)
    with pytest.raises(ValueError):
        sh.partition(m, m.n_el + 1)
    assert len(sh.partition(m, m.n_el)) == m.n_el


class _OracleRankOps(sh.RankOps):
    """A rank's element work by the oracle on its submesh (no masks: the
    sharded solver masks after the halo sum)."""

    def __init__(self, sub):
        import oracle
        self.om = oracle.OracleMesh(sub.elem_type, sub.coords, sub.conn, sub.mu_e(), sub.lam_e(), None)
        self.d = sub.dim

    def residual(self, u):
        return torch.as_tensor(self.om.residual(u.numpy(), mask_out=False))

    def hvp(self, u, v):
        return torch.as_tensor(self.om.hvp(u.numpy(), v.numpy(), mask_in=False, mask_out=False))

    def energy(self, u):
        psi, S, st = self.om.energy_status(u.numpy())
        return (0.0 if st == 3 else psi), S, (1.0 if st == 3 else 0.0)

    def block_diag(self, u):
        return torch.as_tensor(self.om.block_diag(u.numpy()))


import torch  # noqa: E402  (the worker processes import it themselves)


def _solve_worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    m = mg.workload_tet(4, seed=1, random_moduli=1)
    s = sh.partition(m, world)[rank]
    sub = sh.submesh(m, s)
    mask = torch.as_tensor(sub.dirichlet.ravel().astype(bool))
    ubar = torch.as_tensor(sub.ubar.ravel())
    u = torch.zeros(s.n_local * m.dim, dtype=torch.float64)
    st = sh.sharded_load_step(_OracleRankOps(sub), s, mask, ubar, 0.0, 0.05, u)
    st2 = sh.sharded_load_step(_OracleRankOps(sub), s, mask, ubar, 0.05, 0.1, u)
    out[rank] = (s.nodes, u.numpy().copy(), st, st2)
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_load_steps_match_the_single_rank_solve(world):
    """Two Newton-CG load steps on gloo ranks, the oracle as each rank's
    element work, residuals / HVPs / nodal blocks through halo_sum and every
    dot product and norm through dot: the displacements equal the single-rank
    oracle load steps to 1e-10 and are bitwise the same on every rank that
    holds a node; every rank takes the same iteration counts."""
    import oracle
    out = mp.Manager().dict()
    mp.spawn(_solve_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    m = mg.workload_tet(4, seed=1, random_moduli=1)
    om = oracle.OracleMesh.from_mesh(m)
    uo = np.zeros(m.n_nodes * 3)
    assert om.load_step(m.ubar.ravel(), 0.0, 0.05, uo).status == 0
    assert om.load_step(m.ubar.ravel(), 0.05, 0.1, uo).status == 0
    d = m.dim
    seen, stats = {}, set()
    for rank in range(world):
        nodes, u, st, st2 = out[rank]
        assert st["status"] == 0 and st2["status"] == 0
        stats.add((st["newton_iters"], st["cg_iters"], st2["newton_iters"], st2["cg_iters"]))
        idx = (nodes[:, None] * d + np.arange(d)).ravel()
        assert np.linalg.norm(u - uo[idx]) <= 1e-10 * np.linalg.norm(uo[idx])
        for k, n in enumerate(nodes):
            key = int(n)
            vals = u[k * d:(k + 1) * d].tobytes()
            assert seen.setdefault(key, vals) == vals
    assert len(stats) == 1  # the same decisions on every rank
    assert len(seen) == m.n_nodes
