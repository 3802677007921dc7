"""Pins of the oracle's sparse-K functions (Sec. 2.2, Algorithm 2; App. A, B).

The DOF pattern is pinned to closed forms of the mesh topology (one
element, two triangles, the edge count of the Kuhn subdivision of a cube
grid) and to the support of K itself (dense columns K e_j from the oracle's
HVP at a generic state).  The colouring is pinned to its defining properties
(no two columns of one colour share a row, and every colour below a column's
own is held by an earlier conflicting column) and to a dense brute-force
greedy on tiny meshes; the colour counts to the bounds of App. A.  The K
values are pinned to symmetry, to translation invariance, to the vanishing of
infinitesimal rotations at the rest state and to the HVP.
"""
import numpy as np
import pytest

import oracle
from paper_2602_12365_b300 import meshgen as mg


def _csr_dense(ptr, idx, vals, n):
    K = np.zeros((n, n))
    for i in range(n):
        K[i, idx[ptr[i]:ptr[i + 1]]] = vals[ptr[i]:ptr[i + 1]]
    return K


def _csr_matvec(ptr, idx, vals, x):
    rows = np.repeat(np.arange(ptr.size - 1), np.diff(ptr))
    return np.bincount(rows, weights=vals * x[idx], minlength=ptr.size - 1)


def test_pattern_of_one_tet_is_dense():
    conn = np.array([[0, 1, 2, 3]], np.int32)
    ptr, idx = oracle.dof_pattern(4, 3, conn)
    assert idx.size == 144
    for i in range(12):
        assert list(idx[ptr[i]:ptr[i + 1]]) == list(range(12))


def test_pattern_of_two_triangles():
    # square 0-1-2-3 cut along 0-2: nodes 1 and 3 share no element
    conn = np.array([[0, 1, 2], [0, 2, 3]], np.int32)
    ptr, idx = oracle.dof_pattern(4, 2, conn)
    assert idx.size == 4 * (4 + 3 + 4 + 3)
    row1 = set(idx[ptr[2]:ptr[3]])  # first DOF of node 1
    assert row1 == {0, 1, 2, 3, 4, 5}
    row3 = set(idx[ptr[6]:ptr[7]])  # first DOF of node 3
    assert row3 == {0, 1, 4, 5, 6, 7}


@pytest.mark.parametrize("n", [1, 2, 3, 5])
def test_pattern_of_kuhn_grid_closed_form(n):
    # Kuhn subdivision of n^3 cells: axis edges 3n(n+1)^2, one diagonal per
    # square face 3n^2(n+1), one body diagonal per cell n^3; every node pair
    # on an edge, and every node with itself, gives a 3x3 block
    m = mg.tet_mesh(n)
    ptr, idx = oracle.dof_pattern(m.n_nodes, 3, m.conn)
    E = 3 * n * (n + 1) ** 2 + 3 * n * n * (n + 1) + n ** 3
    assert idx.size == 9 * ((n + 1) ** 3 + 2 * E)
    if n >= 2:  # an interior node has 14 neighbours in the Kuhn subdivision
        assert np.diff(ptr).max() == 9 * 15 // 3
    assert np.all(np.diff(idx[ptr[0]:ptr[1]]) > 0)  # ascending columns


def test_pattern_is_the_support_of_K():
    m = mg.workload_tet(2, seed=3, random_moduli=3)
    om = oracle.OracleMesh.from_mesh(m)
    u = mg.smooth_state(m, 0.5, amp=0.05).ravel()
    rng = np.random.default_rng(7)
    u = u + 0.01 * rng.standard_normal(u.size)  # a generic state
    nd = u.size
    K = np.zeros((nd, nd))
    for j in range(nd):
        e = np.zeros(nd)
        e[j] = 1.0
        K[:, j] = om.hvp(u, e, mask_in=False, mask_out=False)
    ptr, idx = oracle.dof_pattern(m.n_nodes, 3, m.conn)
    S = np.zeros((nd, nd), bool)
    for i in range(nd):
        S[i, idx[ptr[i]:ptr[i + 1]]] = True
    assert np.all(S == (K != 0.0))


def _greedy_dense(ptr, idx):
    n = ptr.size - 1
    A = np.zeros((n, n), bool)
    for i in range(n):
        A[i, idx[ptr[i]:ptr[i + 1]]] = True
    conflict = (A.T.astype(int) @ A.astype(int)) > 0  # columns sharing a row
    col = -np.ones(n, int)
    for j in range(n):
        taken = set(col[:j][conflict[j, :j]])
        c = 0
        while c in taken:
            c += 1
        col[j] = c
    return col


@pytest.mark.parametrize("kind,n", [("tet", 1), ("tet", 2), ("tri", 3), ("hex", 2)])
def test_colouring_equals_dense_greedy(kind, n):
    m = {"tet": mg.tet_mesh, "tri": mg.tri_mesh, "hex": mg.hex_mesh}[kind](n)
    ptr, idx = oracle.dof_pattern(m.n_nodes, m.dim, m.conn)
    col, nc = oracle.distance2_colors(ptr, idx)
    ref = _greedy_dense(ptr, idx)
    assert np.array_equal(col, ref) and nc == ref.max() + 1


@pytest.mark.parametrize("kind,n", [("tet", 6), ("tri", 12), ("hex", 5)])
def test_colouring_properties(kind, n):
    m = {"tet": mg.tet_mesh, "tri": mg.tri_mesh, "hex": mg.hex_mesh}[kind](n)
    ptr, idx = oracle.dof_pattern(m.n_nodes, m.dim, m.conn)
    col, nc = oracle.distance2_colors(ptr, idx)
    assert nc == col.max() + 1
    rows = np.repeat(np.arange(ptr.size - 1), np.diff(ptr))
    # valid: within every row the columns' colours are distinct
    key = rows.astype(np.int64) * nc + col[idx]
    assert np.unique(key).size == key.size
    # greedy: below its own colour, every colour is held by an earlier
    # column that shares a row with it
    for j in np.random.default_rng(0).choice(ptr.size - 1, 200, replace=False):
        nb = np.unique(np.concatenate([idx[ptr[i]:ptr[i + 1]] for i in idx[ptr[j]:ptr[j + 1]]]))
        earlier = set(col[nb[nb < j]])
        assert all(c in earlier for c in range(col[j]))


def test_colour_counts_against_appendix_a():
    # App. A: about 80-90 colours for 3D P1 tets, independent of the size
    for n in (8, 16):
        m = mg.tet_mesh(n)
        ptr, idx = oracle.dof_pattern(m.n_nodes, 3, m.conn)
        _, nc = oracle.distance2_colors(ptr, idx)
        assert 80 <= nc <= 90
        assert nc >= np.diff(ptr).max()  # a row's columns all differ
    # Q1 hexes on a grid: the 3x3x3 node stencil times 3 components
    m = mg.hex_mesh(6)
    ptr, idx = oracle.dof_pattern(m.n_nodes, 3, m.conn)
    _, nc = oracle.distance2_colors(ptr, idx)
    assert nc == 81
    # structured right triangles (valence 6): 14 columns a row; the greedy
    # needs 18 (App. A quotes 30-40 for its unstructured triangle meshes)
    m = mg.tri_mesh(16)
    ptr, idx = oracle.dof_pattern(m.n_nodes, 2, m.conn)
    _, nc = oracle.distance2_colors(ptr, idx)
    assert np.diff(ptr).max() == 14 and 14 <= nc <= 40


def test_sparse_K_values():
    m = mg.workload_tet(2, seed=5, random_moduli=5)
    om = oracle.OracleMesh.from_mesh(m)
    u = mg.smooth_state(m, 0.5, amp=0.05).ravel()
    nd = u.size
    ptr, idx, vals = om.sparse_K(u, mask_in=False, mask_out=False)
    K = _csr_dense(ptr, idx, vals, nd)
    scale = np.abs(K).max()
    np.testing.assert_allclose(K, K.T, atol=1e-12 * scale)
    # translation invariance of the energy: K t = 0 for a uniform translation
    for c in range(3):
        t = np.zeros((m.n_nodes, 3))
        t[:, c] = 1.0
        assert np.abs(K @ t.ravel()).max() <= 1e-12 * scale
    # K agrees with the HVP in every direction
    v = np.random.default_rng(2).standard_normal(nd)
    y = om.hvp(u, v, mask_in=False, mask_out=False)
    np.testing.assert_allclose(_csr_matvec(ptr, idx, vals, v), y, atol=1e-12 * np.abs(y).max())


def test_sparse_K_at_rest_annihilates_rotations():
    # at u = 0 the stress vanishes and an infinitesimal rotation v = W X
    # (W skew) strains nothing, so K(0) v = 0
    m = mg.workload_tet(2, seed=4)
    om = oracle.OracleMesh.from_mesh(m)
    nd = m.n_nodes * 3
    ptr, idx, vals = om.sparse_K(np.zeros(nd), mask_in=False, mask_out=False)
    K = _csr_dense(ptr, idx, vals, nd)
    W = np.array([[0.0, 0.3, -0.2], [-0.3, 0.0, 0.5], [0.2, -0.5, 0.0]])
    v = (m.coords @ W.T).ravel()
    assert np.abs(K @ v).max() <= 1e-12 * np.abs(K).max()
    assert np.abs(K @ (m.coords @ np.diag([1.0, 2.0, 3.0])).ravel()).max() > 1e-3  # a stretch does not vanish


def test_sparse_K_masked_rows_and_columns():
    m = mg.workload_tet(2, seed=6)
    om = oracle.OracleMesh.from_mesh(m)
    u = mg.smooth_state(m, 0.5).ravel()
    ptr, idx, vals = om.sparse_K(u)
    K = _csr_dense(ptr, idx, vals, u.size)
    fixed = m.dirichlet.reshape(-1).astype(bool)
    assert fixed.any() and (~fixed).any()
    assert np.all(K[fixed] == 0.0) and np.all(K[:, fixed] == 0.0)
    _, _, vu = om.sparse_K(u, mask_in=False, mask_out=False)
    Ku = _csr_dense(ptr, idx, vu, u.size)
    np.testing.assert_array_equal(K[np.ix_(~fixed, ~fixed)], Ku[np.ix_(~fixed, ~fixed)])
