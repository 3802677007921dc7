"""Seeded synthetic inputs: structured meshes, material fields, boundary data.

This module produces *inputs only*.  It holds none of the method's arithmetic
(no shape functions, no energy, no derivatives), so both the CUDA path and the
CPU oracle may consume what it generates without sharing any method code.

Meshes follow the structured families of the benchmark workloads:

* ``tri_mesh(n)``   -- unit square, n x n cells, each split into two P1
  triangles along the (i, j) -> (i+1, j+1) diagonal, counter-clockwise.
* ``tet_mesh(n)``   -- unit cube, n^3 cells, each split into the six Kuhn
  (Freudenthal) tetrahedra that share the (0,0,0) -> (1,1,1) diagonal, one per
  permutation of the axes; vertex order is chosen from the permutation parity
  so every tetrahedron has positive orientation.
* ``hex_mesh(n)``   -- unit cube, n^3 trilinear hexahedra, VTK_HEXAHEDRON
  vertex order.

Node ids are ``i + (n+1) j (+ (n+1)^2 k)``; elements are numbered cell-major
with ``i`` fastest.

Random numbers come from a counter-based SplitMix64 hash (Steele, Lea and
Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014): the
value for ``(seed, stream, counter)`` is the SplitMix64 output finaliser applied
to ``key(seed, stream) + (counter + 1) * 0x9E3779B97F4A7C15``, mapped to
[0, 1) with its top 53 bits.  Normal variates use Box--Muller on two such
uniforms.
"""
from __future__ import annotations

import itertools
from dataclasses import dataclass, field

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

STREAM_JITTER = 1
STREAM_MU = 2
STREAM_VEC = 3
STREAM_STATE = 4


def _finalize(z: np.ndarray) -> np.ndarray:
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def _key(seed: int, stream: int) -> np.uint64:
    z = np.array([(int(seed) * 0x2545F4914F6CDD1D + int(stream) * 0xD1B54A32D192ED03)
                  & 0xFFFFFFFFFFFFFFFF], dtype=np.uint64)
    return _finalize(z)[0]


def uniform(seed: int, stream: int, n: int) -> np.ndarray:
    """n uniforms in [0, 1) for counters 0..n-1 of (seed, stream)."""
    c = np.arange(1, n + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = _key(seed, stream) + c * _GOLDEN
    x = _finalize(z)
    return (x >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def normal(seed: int, stream: int, n: int) -> np.ndarray:
    """n standard normal variates (Box--Muller on counters 2i, 2i+1)."""
    u = uniform(seed, stream, 2 * n).reshape(n, 2)
    u1 = 1.0 - u[:, 0]                      # (0, 1]
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u[:, 1])


# ----------------------------------------------------------------------------
# meshes
# ----------------------------------------------------------------------------
TRI3, TET4, HEX8 = 0, 1, 2
N_EN = {TRI3: 3, TET4: 4, HEX8: 8}
DIM = {TRI3: 2, TET4: 3, HEX8: 3}


@dataclass
class Mesh:
    elem_type: int
    coords: np.ndarray            # [n_nodes, dim] float64
    conn: np.ndarray              # [n_el, n_en] int32
    n: int                        # cells per side
    mu: np.ndarray | None = None  # [n_el] float64 or None (uniform)
    lam: np.ndarray | None = None
    mu0: float = 1.0
    lam0: float = 10.0
    dirichlet: np.ndarray | None = None  # [n_nodes, dim] uint8, 1 = prescribed
    ubar: np.ndarray | None = None       # [n_nodes, dim] prescribed values at load factor 1
    name: str = ""
    extra: dict = field(default_factory=dict)

    @property
    def dim(self) -> int:
        return self.coords.shape[1]

    @property
    def n_nodes(self) -> int:
        return self.coords.shape[0]

    @property
    def n_el(self) -> int:
        return self.conn.shape[0]

    def mu_e(self) -> np.ndarray:
        return self.mu if self.mu is not None else np.full(self.n_el, self.mu0)

    def lam_e(self) -> np.ndarray:
        return self.lam if self.lam is not None else np.full(self.n_el, self.lam0)


def _grid_ids_2d(n):
    i, j = np.meshgrid(np.arange(n), np.arange(n), indexing="xy")
    return i.ravel(), j.ravel()            # i fastest


def tri_mesh(n: int) -> Mesh:
    m = n + 1
    jj, ii = np.meshgrid(np.arange(m), np.arange(m), indexing="ij")
    coords = np.stack([ii.ravel() / n, jj.ravel() / n], axis=1).astype(np.float64)
    i, j = _grid_ids_2d(n)
    v00 = i + m * j
    v10 = v00 + 1
    v01 = v00 + m
    v11 = v01 + 1
    t0 = np.stack([v00, v10, v11], axis=1)
    t1 = np.stack([v00, v11, v01], axis=1)
    conn = np.stack([t0, t1], axis=1).reshape(-1, 3).astype(np.int32)
    return Mesh(TRI3, coords, conn, n, name=f"tri{n}")


def _grid_coords_3d(n):
    m = n + 1
    kk, jj, ii = np.meshgrid(np.arange(m), np.arange(m), np.arange(m), indexing="ij")
    return np.stack([ii.ravel() / n, jj.ravel() / n, kk.ravel() / n], axis=1).astype(np.float64)


def _cell_base_3d(n):
    m = n + 1
    kk, jj, ii = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    return (ii + m * jj + m * m * kk).ravel()


def _perm_parity(p):
    inv = 0
    for a in range(3):
        for b in range(a + 1, 3):
            inv += p[a] > p[b]
    return inv % 2


def tet_mesh(n: int, jitter_seed: int | None = None, jitter: float = 0.1) -> Mesh:
    m = n + 1
    coords = _grid_coords_3d(n)
    base = _cell_base_3d(n)
    step = [1, m, m * m]
    tets = []
    for p in itertools.permutations(range(3)):
        a = base + step[p[0]]
        b = a + step[p[1]]
        c = b + step[p[2]]
        if _perm_parity(p):
            tets.append(np.stack([base, a, c, b], axis=1))
        else:
            tets.append(np.stack([base, a, b, c], axis=1))
    conn = np.stack(tets, axis=1).reshape(-1, 4).astype(np.int32)
    if jitter_seed is not None:
        h = 1.0 / n
        ijk = np.rint(coords * n).astype(np.int64)
        interior = np.all((ijk > 0) & (ijk < n), axis=1)
        u = uniform(jitter_seed, STREAM_JITTER, coords.size).reshape(coords.shape)
        coords = coords + np.where(interior[:, None], (2.0 * u - 1.0) * jitter * h, 0.0)
    return Mesh(TET4, coords, conn, n, name=f"tet{n}")


# VTK_HEXAHEDRON local order as (di, dj, dk)
HEX_LOCAL = [(0, 0, 0), (1, 0, 0), (1, 1, 0), (0, 1, 0),
             (0, 0, 1), (1, 0, 1), (1, 1, 1), (0, 1, 1)]


def hex_mesh(n: int) -> Mesh:
    m = n + 1
    coords = _grid_coords_3d(n)
    base = _cell_base_3d(n)
    conn = np.stack([base + di + m * dj + m * m * dk for di, dj, dk in HEX_LOCAL],
                    axis=1).astype(np.int32)
    return Mesh(HEX8, coords, conn, n, name=f"hex{n}")


def lognormal_moduli(mesh: Mesh, seed: int, sigma: float = 0.5, ratio: float = 10.0):
    """Per-element mu = exp(sigma z), z ~ N(0, 1); lambda = ratio * mu."""
    z = normal(seed, STREAM_MU, mesh.n_el)
    mesh.mu = np.exp(sigma * z)
    mesh.lam = ratio * mesh.mu
    return mesh


# ----------------------------------------------------------------------------
# boundary data
# ----------------------------------------------------------------------------
def grid_index(mesh: Mesh) -> np.ndarray:
    """Integer grid coordinates of every node (independent of jitter)."""
    n = mesh.n
    m = n + 1
    ids = np.arange(mesh.n_nodes)
    if mesh.dim == 2:
        return np.stack([ids % m, ids // m], axis=1)
    return np.stack([ids % m, (ids // m) % m, ids // (m * m)], axis=1)


def bc_clamp_and_pull_2d(mesh: Mesh, pull: float = 0.1):
    """Left edge clamped; right edge x-displacement ``pull``, y free."""
    g = grid_index(mesh)
    mask = np.zeros((mesh.n_nodes, 2), np.uint8)
    ubar = np.zeros((mesh.n_nodes, 2))
    left = g[:, 0] == 0
    right = g[:, 0] == mesh.n
    mask[left, :] = 1
    mask[right, 0] = 1
    ubar[right, 0] = pull
    mesh.dirichlet, mesh.ubar = mask, ubar
    return mesh


def bc_base_and_top_3d(mesh: Mesh, top=(0.0, 0.0, -0.2)):
    """z = 0 face clamped; z = 1 face displaced by ``top`` (all components)."""
    g = grid_index(mesh)
    mask = np.zeros((mesh.n_nodes, 3), np.uint8)
    ubar = np.zeros((mesh.n_nodes, 3))
    bot = g[:, 2] == 0
    topf = g[:, 2] == mesh.n
    mask[bot | topf, :] = 1
    ubar[topf, :] = np.asarray(top, dtype=np.float64)
    mesh.dirichlet, mesh.ubar = mask, ubar
    return mesh


def bc_uniaxial_bar(mesh: Mesh, delta: float):
    """Rollers for a homogeneous uniaxial stretch by ``delta``.

    2D: stretch along x (u_x = 0 on x = 0, u_x = delta on x = 1, u_y = 0 at
    the origin).  3D: stretch along z (u_z = 0 on z = 0, u_z = delta on z = 1,
    u_x = u_y = 0 at the origin, u_y = 0 at (1, 0, 0)).
    """
    g = grid_index(mesh)
    n = mesh.n
    d = mesh.dim
    mask = np.zeros((mesh.n_nodes, d), np.uint8)
    ubar = np.zeros((mesh.n_nodes, d))
    ax = 0 if d == 2 else 2
    lo = g[:, ax] == 0
    hi = g[:, ax] == n
    mask[lo, ax] = 1
    mask[hi, ax] = 1
    ubar[hi, ax] = delta
    origin = np.all(g == 0, axis=1)
    if d == 2:
        mask[origin, 1] = 1
    else:
        mask[origin, 0] = 1
        mask[origin, 1] = 1
        xcorner = (g[:, 0] == n) & (g[:, 1] == 0) & (g[:, 2] == 0)
        mask[xcorner, 1] = 1
    mesh.dirichlet, mesh.ubar = mask, ubar
    return mesh


# ----------------------------------------------------------------------------
# the benchmark workloads (sizes scale with ``n``)
# ----------------------------------------------------------------------------
def workload_tri(n: int = 32) -> Mesh:
    """2D plane-strain P1 square, mu = 1, lambda = 10, clamp-and-pull (0.1)."""
    return bc_clamp_and_pull_2d(tri_mesh(n), 0.1)


def workload_tet(n: int = 64, seed: int = 0, random_moduli: int | None = None) -> Mesh:
    """3D Kuhn tets on a jittered cube; base clamped, top compressed 20 %.

    ``random_moduli`` (a seed) draws per-element lognormal(0, 0.5) moduli, the
    random-modulus mesh family used to train the learned preconditioner.
    """
    m = tet_mesh(n, jitter_seed=seed)
    if random_moduli is not None:
        lognormal_moduli(m, random_moduli)
    return bc_base_and_top_3d(m, (0.0, 0.0, -0.2))


def workload_hex(n: int = 128, seed: int = 0) -> Mesh:
    """3D Q1 hexes, lognormal(0, 0.5) mu with lambda = 10 mu; top sheared 0.1."""
    m = lognormal_moduli(hex_mesh(n), seed)
    return bc_base_and_top_3d(m, (0.1, 0.0, 0.0))


def ncm_params(H: int = 16, seed: int = 0, amp: float = 0.2) -> np.ndarray:
    """Synthetic (untrained) weights of the neural constitutive model's MLP
    2 -> H -> H -> 1: W1 [H][2], b1, W2 [H][H], b2, w3, b3 flattened, all
    from the seeded normal stream; `amp` scales the output layer."""
    z = normal(seed, 11, H * H + 5 * H + 1)
    W1 = z[:2 * H]
    b1 = 0.5 * z[2 * H:3 * H]
    W2 = z[3 * H:3 * H + H * H] / np.sqrt(H)
    b2 = 0.5 * z[3 * H + H * H:4 * H + H * H]
    w3 = amp * z[4 * H + H * H:5 * H + H * H] / np.sqrt(H)
    b3 = z[5 * H + H * H:]
    return np.concatenate([W1, b1, W2, b2, w3, b3]).astype(np.float64)


def smooth_state(mesh: Mesh, s: float, amp: float = 0.02) -> np.ndarray:
    """BC-consistent displacement at load factor s: the affine interpolant of
    the prescribed data plus ``amp * prod_k sin(2 pi x_k)`` in every component
    (which vanishes on the boundary of the unit box)."""
    X = mesh.coords
    g = grid_index(mesh)
    d = mesh.dim
    # affine part: blend of the prescribed values along the loading axis
    ax = 0 if d == 2 else d - 1
    t = g[:, ax] / mesh.n
    top = mesh.ubar[g[:, ax] == mesh.n]
    top_val = top.mean(axis=0) if len(top) else np.zeros(d)
    if d == 2:
        # 2D clamp-and-pull: u_x grows linearly in x; u_y zero
        u = np.zeros_like(X)
        u[:, 0] = s * top_val[0] * t
    else:
        u = s * t[:, None] * top_val[None, :]
    bump = amp * np.prod(np.sin(2.0 * np.pi * X), axis=1)
    u = u + bump[:, None]
    # prescribed entries exactly s * ubar
    pres = mesh.dirichlet.astype(bool)
    u[pres] = s * mesh.ubar[pres]
    return u


def random_direction(mesh: Mesh, seed: int = 1) -> np.ndarray:
    """v ~ N(0, 1) on free DOFs, zero on prescribed ones."""
    v = normal(seed, STREAM_VEC, mesh.n_nodes * mesh.dim).reshape(mesh.n_nodes, mesh.dim)
    v[mesh.dirichlet.astype(bool)] = 0.0
    return v
