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


def _sum_in_rank_order(x: torch.Tensor, s: Shard, received: dict, width: int | None = None) -> torch.Tensor:
    """acc[node] = sum of the partials of the ranks touching it, in rank
    order (every rank performs the same additions for a shared node); a node
    holds `width` values (default: dim)."""
    d = width or s.dim
    xv = x.view(-1, d)
    acc = torch.zeros_like(xv)
    for q in sorted(set(received) | {s.rank}):
        if q == s.rank:
            acc += xv
        else:
            idx = torch.as_tensor(s.iface[q], device=x.device)
            acc.index_add_(0, idx, received[q].view(-1, d))
    return acc.view(-1)


def halo_sum(x: torch.Tensor, s: Shard, group=None, width: int | None = None) -> torch.Tensor:
    """The assembled vector on the rank's local nodes from its partial x
    (local numbering, [n_local * width], width = dim for nodal vectors, dim^2
    for nodal blocks); exchanges with every neighbour."""
    import torch.distributed as dist
    d = width or s.dim
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
    return _sum_in_rank_order(x, s, recvs, d)


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


# ---------------------------------------------------------------------------
# The sharded Newton-CG load step
# ---------------------------------------------------------------------------
class RankOps:
    """One rank's element work on its submesh, unmasked and unsummed: the
    library's calls on a GPU, or the oracle in the CPU tests.  Subclasses
    provide residual(u) -> r partial, hvp(u, v) -> y partial,
    energy(u) -> (psi, S, n_inverted) partial, block_diag(u) -> [n, d, d]
    partial blocks; vectors are FP64 tensors in local numbering."""


def _allsum(vals, group=None):
    import torch.distributed as dist
    t = torch.tensor(vals, dtype=torch.float64)
    dist.all_reduce(t, group=group)
    return t.tolist()


def _block_inverse(D: torch.Tensor, mask: torch.Tensor):
    """Block Jacobi from assembled nodal blocks: prescribed rows and columns
    replaced by the identity, inverse through the Cholesky factor (as the
    oracle and the library).  Returns (Minv, ok)."""
    d = D.shape[-1]
    A = D.clone()
    m = mask.view(-1, d)
    eye = torch.eye(d, dtype=A.dtype)
    for c in range(d):
        pc = m[:, c]
        A[pc, c, :] = 0.0
        A[pc, :, c] = 0.0
        A[pc, c, c] = 1.0
    Lc, info = torch.linalg.cholesky_ex(A)
    if int(info.max()) != 0:
        return None, False
    Li = torch.linalg.solve_triangular(Lc, eye.expand_as(A), upper=False)
    return Li.transpose(1, 2) @ Li, True


def sharded_load_step(ops: RankOps, s: Shard, mask: torch.Tensor, ubar: torch.Tensor, s0: float, s1: float,
                      u: torch.Tensor, opts: dict | None = None, group=None) -> dict:
    """One load increment s0 -> s1 of the Newton-CG method (the algorithm the
    oracle and fem_newton_step run: predictor, Eisenstat-Walker PCG with block
    Jacobi, Armijo line search with the roundoff guard, bisection) on an
    element-sharded mesh.  Every residual, HVP and nodal block is the rank's
    element work followed by `halo_sum`; every dot product and norm is `dot`
    (owned nodes, FP64, all-reduced); energies are all-reduced.  All ranks
    therefore take identical decisions and hold identical values at shared
    nodes.  u (FP64, local numbering) is updated in place; mask is the
    rank's per-DOF Dirichlet mask (bool), ubar its prescribed values."""
    o = {"newton_rtol": 1e-8, "newton_max": 50, "eta_max": 0.1, "cg_max": 0, "predictor_rtol": 1e-2,
         "armijo_c": 1e-4, "ls_max": 20, "ls_eps": 2.220446049250313e-16, "max_bisect": 5}
    o.update(opts or {})
    d = s.dim
    nd_global = int(_allsum([float(s.owned.sum() * d)], group)[0])
    cg_max = o["cg_max"] if o["cg_max"] > 0 else 10 * nd_global
    st = {"newton_iters": 0, "cg_iters": 0, "bisections": 0, "ls_halvings": 0, "r0_norm": 0.0, "r_norm": 0.0}
    free = ~mask

    def dotg(x, y):
        return dot(x, y, s, group)

    def residual(uu):
        return torch.where(mask, torch.zeros_like(uu), halo_sum(ops.residual(uu), s, group))

    def hvp_masked(uu, v):
        vm = torch.where(mask, torch.zeros_like(v), v)
        return torch.where(mask, torch.zeros_like(v), halo_sum(ops.hvp(uu, vm), s, group))

    def energy(uu):
        psi, S, ninv = _allsum(list(ops.energy(uu)), group)
        return (float("inf") if ninv > 0 else psi), S

    def precond(uu):
        Db = halo_sum(ops.block_diag(uu).reshape(-1), s, group, d * d).view(-1, d, d)
        Minv, ok = _block_inverse(Db, mask)
        # a collective decision: every rank leaves (or not) together
        ok_all = _allsum([0.0 if ok else 1.0], group)[0] == 0.0
        return Minv, ok_all

    def apply(Minv, x):
        return (Minv @ x.view(-1, d, 1)).reshape(-1)

    def pcg(uu, Minv, b, tol_abs):
        x = torch.zeros_like(b)
        res = b.clone()
        z = apply(Minv, res)
        p = z.clone()
        rz = dotg(res, z)
        if dotg(res, res) ** 0.5 <= tol_abs:
            return x, 0
        k = 0
        while k < cg_max:
            q = hvp_masked(uu, p)
            pq = dotg(p, q)
            if not pq > 0.0:
                return (z if k == 0 else x), k + 1
            alpha = rz / pq
            x = x + alpha * p
            res = res - alpha * q
            if dotg(res, res) ** 0.5 <= tol_abs:
                return x, k + 1
            z = apply(Minv, res)
            rz_new = dotg(res, z)
            beta = rz_new / rz
            rz = rz_new
            p = z + beta * p
            k += 1
        return x, k

    def increment(a0, a1):
        du = torch.where(mask, (a1 - a0) * ubar, torch.zeros_like(ubar))
        # t = M K(u) (I - M) du_c: the HVP with the prescribed increment, free rows
        t = torch.where(mask, torch.zeros_like(du), halo_sum(ops.hvp(u, du), s, group))
        r0 = dotg(t, t) ** 0.5
        if r0 > 0.0:
            Minv, ok = precond(u)
            if not ok:
                return 5
            x, it = pcg(u, Minv, -t, o["predictor_rtol"] * r0)
            st["cg_iters"] += it
            u.copy_(u + torch.where(mask, du, x))
        u.copy_(torch.where(mask, a1 * ubar, u))
        psi, S = energy(u)
        if not np.isfinite(psi):
            return 3
        r = residual(u)
        rn = dotg(r, r) ** 0.5
        if not r0 > 0.0:
            r0 = rn
        st["r0_norm"] = r0
        for it in range(o["newton_max"] + 1):
            st["r_norm"] = rn
            if rn <= o["newton_rtol"] * r0:
                return 0
            if it == o["newton_max"]:
                return 6
            st["newton_iters"] += 1
            eta = min(o["eta_max"], (rn / r0) ** 0.5)
            Minv, ok = precond(u)
            if not ok:
                return 5
            x, k = pcg(u, Minv, -r, eta * rn)
            st["cg_iters"] += k
            g = dotg(r, x)
            alpha, accepted = 1.0, False
            for _ in range(o["ls_max"] + 1):
                ut = u + alpha * x
                pt, St = energy(ut)
                if np.isfinite(pt):
                    if pt <= psi + o["armijo_c"] * alpha * g:
                        accepted = True
                    elif abs(pt - psi) <= 16.0 * o["ls_eps"] * S:
                        rt = residual(ut)
                        if dotg(rt, rt) ** 0.5 < rn:
                            accepted = True
                if accepted:
                    psi, S = pt, St
                    break
                alpha *= 0.5
                st["ls_halvings"] += 1
            if not accepted:
                return 7
            u.copy_(ut)
            r = residual(u)
            rn = dotg(r, r) ** 0.5
        return 6

    def step_rec(a0, a1, depth):
        save = u.clone()
        rc = increment(a0, a1)
        if rc != 0 and depth < o["max_bisect"]:
            u.copy_(save)
            st["bisections"] += 1
            am = 0.5 * (a0 + a1)
            rc = step_rec(a0, am, depth + 1)
            if rc == 0:
                rc = step_rec(am, a1, depth + 1)
        return rc

    st["status"] = step_rec(s0, s1, 0)
    return st


class LibraryRankOps(RankOps):
    """A rank's element work by the library on its submesh (FP64 calls, no
    Dirichlet mask on the submesh: the sharded solver masks after the halo
    sum).  The solver's vectors may live on the host (a gloo group) or on the
    device (an NCCL group); each call moves its inputs to the device and its
    results back to the vectors' device."""

    def __init__(self, sub: mg.Mesh, device="cuda"):
        from .fem import Mesh
        self.mesh = Mesh(sub.elem_type, sub.coords, sub.conn, sub.mu_e(), sub.lam_e(), dirichlet=None,
                         precision="fp64")
        self.dev = torch.device(device)
        self.d = sub.dim

    def residual(self, u):
        return self.mesh.residual(u.to(self.dev), mask_out=False).to(u.device)

    def hvp(self, u, v):
        return self.mesh.hvp(u.to(self.dev), v.to(self.dev), mask_in=False, mask_out=False).to(u.device)

    def energy(self, u):
        e = self.mesh.energy(u.to(self.dev)).cpu()
        inv = float(e[2])
        return (0.0 if inv > 0 else float(e[0])), float(e[1]), inv

    def block_diag(self, u):
        return self.mesh.block_diag(u.to(self.dev)).view(-1, self.d, self.d).to(u.device)
