"""The library's host-side sparse-K pattern and colouring (Algorithm 2's
inputs, App. A/B) against the oracle, bit for bit, without a GPU."""
import numpy as np
import pytest

import oracle
from paper_2602_12365_b300 import meshgen as mg
from paper_2602_12365_b300._lib import FemError
from paper_2602_12365_b300.fem import sparse_pattern_host


@pytest.mark.parametrize("kind,n", [("tri", 1), ("tri", 7), ("tet", 1), ("tet", 5), ("tet", 16),
                                    ("hex", 1), ("hex", 6)])
def test_pattern_and_colours_equal_oracle(kind, n):
    m = {"tri": mg.workload_tri, "tet": mg.workload_tet, "hex": mg.workload_hex}[kind](n)
    rp, ci, co, nc = sparse_pattern_host(m.elem_type, m.coords, m.conn)
    ptr, idx = oracle.dof_pattern(m.n_nodes, m.dim, m.conn)
    col, ncol = oracle.distance2_colors(ptr, idx)
    assert np.array_equal(rp, ptr) and np.array_equal(ci, idx)
    assert np.array_equal(co, col) and nc == ncol


def test_single_element_and_shuffled_numbering():
    # one tet: every DOF couples to every DOF, 12 colours
    conn = np.array([[0, 1, 2, 3]], np.int32)
    X = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], float)
    rp, ci, co, nc = sparse_pattern_host(1, X, conn)
    assert ci.size == 144 and nc == 12 and np.array_equal(co, np.arange(12))
    # a renumbered mesh: same as the oracle on the same numbering
    m = mg.workload_tet(4)
    perm = np.random.default_rng(3).permutation(m.n_nodes)
    conn2 = perm[m.conn].astype(np.int32)
    X2 = np.zeros_like(m.coords)
    X2[perm] = m.coords
    rp, ci, co, nc = sparse_pattern_host(1, X2, conn2)
    ptr, idx = oracle.dof_pattern(m.n_nodes, 3, conn2)
    col, ncol = oracle.distance2_colors(ptr, idx)
    assert np.array_equal(ci, idx) and np.array_equal(co, col) and nc == ncol


def test_bad_descriptions_raise():
    X = np.zeros((4, 3))
    with pytest.raises(FemError):
        sparse_pattern_host(1, X, np.array([[0, 1, 2, 4]], np.int32))  # node out of range
    with pytest.raises(FemError):
        sparse_pattern_host(5, X, np.array([[0, 1, 2, 3]], np.int32))  # no such element type
