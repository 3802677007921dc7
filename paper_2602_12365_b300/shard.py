"""Element sharding with halo sums: the layout of the path on several GPUs.

The energy is a sum of element terms (Eq. 2), so the mesh shards by element.
Each rank owns a slab of elements (ordered by centroid along one axis, equal
counts) and the nodes they touch, numbered locally in ascending global order;
nodes touched by several ranks are interface nodes.  A residual or HVP is
each rank's local call (`fem_residual` / `fem_hvp` on its submesh) followed
by one halo sum: every interface node's value becomes the sum of the
touching ranks' partials, added in rank order, so that all ranks hold the
same bits.  A dot product sums every node once (on the lowest rank that
touches it) and all-reduces the scalar.

The exchange is host-driven point-to-point traffic between neighbouring
ranks (`torch.distributed` isend/irecv: NCCL on GPUs, gloo on CPU); no kernel
waits for another rank.  This module holds the partition and the exchange;
the element work stays in the library.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import torch

from . import meshgen as mg


@dataclass
class Shard:
    rank: int
    world: int
    dim: int
    elems: np.ndarray                 # global element ids, ascending
    nodes: np.ndarray                 # global node id of each local node, ascending
    owned: np.ndarray                 # per local node: this rank is the lowest rank touching it
    iface: dict = field(default_factory=dict)  # neighbour rank -> local node ids shared with it

    @property
    def n_local(self) -> int:
        return self.nodes.size


def partition(mesh: mg.Mesh, world: int, axis: int | None = None) -> list[Shard]:
    """Slabs of equal element counts along `axis` (default: the last)."""
    if world < 1 or world > mesh.n_el:
        raise ValueError("world must be between 1 and the number of elements")
    axis = mesh.dim - 1 if axis is None else axis
    cen = mesh.coords[mesh.conn].mean(axis=1)[:, axis]
    order = np.lexsort((np.arange(mesh.n_el), cen))  # ties by element id
    owner = np.empty(mesh.n_el, np.int64)
    for r, part in enumerate(np.array_split(order, world)):
        owner[part] = r
    # ranks touching each node
    touch = [set() for _ in range(mesh.n_nodes)]
    for e, r in enumerate(owner):
        for n in mesh.conn[e]:
            touch[n].add(int(r))
    low = np.array([min(t) if t else -1 for t in touch])
    shards = []
    for r in range(world):
        elems = np.flatnonzero(owner == r)
        nodes = np.unique(mesh.conn[elems])
        shards.append(Shard(r, world, mesh.dim, elems, nodes, low[nodes] == r))
    for s in shards:
        local = {int(g): i for i, g in enumerate(s.nodes)}
        for q in range(world):
            if q == s.rank:
                continue
            shared = [g for g in s.nodes if q in touch[g]]
            if shared:
                s.iface[q] = np.array([local[int(g)] for g in shared], np.int64)
    return shards


def submesh(mesh: mg.Mesh, s: Shard) -> mg.Mesh:
    """The rank's elements as a mesh of their own (local node numbering)."""
    g2l = np.full(mesh.n_nodes, -1, np.int64)
    g2l[s.nodes] = np.arange(s.n_local)
    sub = mg.Mesh(mesh.elem_type, mesh.coords[s.nodes].copy(), g2l[mesh.conn[s.elems]].astype(np.int32), mesh.n,
                  None if mesh.mu is None else mesh.mu[s.elems].copy(),
                  None if mesh.lam is None else mesh.lam[s.elems].copy(), mesh.mu0, mesh.lam0,
                  None if mesh.dirichlet is None else mesh.dirichlet[s.nodes].copy(),
                  None if mesh.ubar is None else mesh.ubar[s.nodes].copy(), f"{mesh.name}/rank{s.rank}")
    return sub


def _sum_in_rank_order(x: torch.Tensor, s: Shard, received: dict) -> torch.Tensor:
    """acc[node] = sum of the partials of the ranks touching it, in rank
    order (every rank performs the same additions for a shared node)."""
    d = s.dim
    xv = x.view(-1, d)
    acc = torch.zeros_like(xv)
    for q in sorted(set(received) | {s.rank}):
        if q == s.rank:
            acc += xv
        else:
            idx = torch.as_tensor(s.iface[q], device=x.device)
            acc.index_add_(0, idx, received[q].view(-1, d))
    return acc.view(-1)


def halo_sum(x: torch.Tensor, s: Shard, group=None) -> torch.Tensor:
    """The assembled vector on the rank's local nodes from its partial x
    (local numbering, [n_local * dim]); exchanges with every neighbour."""
    import torch.distributed as dist
    d = s.dim
    xv = x.view(-1, d)
    sends, recvs, reqs = {}, {}, []
    for q in sorted(s.iface):
        idx = torch.as_tensor(s.iface[q], device=x.device)
        sends[q] = xv.index_select(0, idx).contiguous()
        recvs[q] = torch.empty_like(sends[q])
    for q in sorted(s.iface):  # lower ranks send first: the pairs never wait on each other
        if q < s.rank:
            reqs.append(dist.irecv(recvs[q], src=q, group=group))
            reqs.append(dist.isend(sends[q], dst=q, group=group))
        else:
            reqs.append(dist.isend(sends[q], dst=q, group=group))
            reqs.append(dist.irecv(recvs[q], src=q, group=group))
    for rq in reqs:
        rq.wait()
    return _sum_in_rank_order(x, s, recvs)


def halo_sum_local(parts: list, shards: list) -> list:
    """The same sums with every rank's partial in one process (no
    communication): what `halo_sum` returns on each rank."""
    out = []
    for s in shards:
        received = {}
        for q, idx in s.iface.items():
            other = shards[q]
            # node ids shared with q, in q's numbering: same global ids, same order
            g = s.nodes[idx]
            qi = np.searchsorted(other.nodes, g)
            received[q] = parts[q].view(-1, s.dim)[torch.as_tensor(qi, device=parts[q].device)].reshape(-1)
        out.append(_sum_in_rank_order(parts[s.rank], s, received))
    return out


def dot(x: torch.Tensor, y: torch.Tensor, s: Shard, group=None) -> float:
    """Global x . y of assembled vectors: owned nodes only, FP64, all-reduced."""
    import torch.distributed as dist
    d = s.dim
    m = torch.as_tensor(s.owned, device=x.device)
    v = (x.view(-1, d)[m].double() * y.view(-1, d)[m].double()).sum().reshape(1)
    dist.all_reduce(v, group=group)
    return float(v.item())
