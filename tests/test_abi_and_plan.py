"""CPU checks of the C ABI library: it loads, exports every entry point the
header declares, and its host partitioner produces a valid two-level
colouring (no GPU call is made)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_2602_12365_b300 import build as B
from paper_2602_12365_b300 import meshgen as mg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    from paper_2602_12365_b300 import _lib
    return _lib


def _declared():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        txt = open(os.path.join(ROOT, "include", h)).read()
        names |= set(re.findall(r"^\s*(?:fem_status|const char\s*\*)\s*(fem_\w+)\s*\(", txt, re.M))
    return names


def test_library_exports_every_declared_symbol(lib):
    names = _declared()
    assert len(names) >= 10
    so = C.CDLL(lib.LIB_PATH)
    missing = [n for n in names if not hasattr(so, n)]
    assert not missing, missing
    assert set(lib.EXPORTED) >= names


def test_bad_descriptor_is_rejected_without_gpu(lib):
    from paper_2602_12365_b300.fem import make_desc
    m = mg.tri_mesh(2)
    conn = m.conn.copy()
    conn[0, 0] = 10_000
    d, keep = make_desc(m.elem_type, m.coords, conn)
    info = lib.MeshInfo()
    st = lib.lib().fem_plan_partition(C.byref(d), None, None, None, None, C.byref(info))
    assert st == 1  # FEM_ERR_ARG
    assert b"out of range" in lib.lib().fem_last_error()
    st = lib.lib().fem_plan_partition(None, None, None, None, None, None)
    assert st == 1


@pytest.mark.parametrize("kind,n,tile", [("tri", 24, 128), ("tri", 48, 0), ("tet", 6, 200), ("tet", 9, 0),
                                         ("hex", 7, 64), ("hex", 5, 0)])
def test_two_level_colouring_is_valid(lib, kind, n, tile):
    from paper_2602_12365_b300.fem import plan_partition
    m = {"tri": lambda: mg.tri_mesh(n), "tet": lambda: mg.tet_mesh(n, jitter_seed=1),
         "hex": lambda: mg.hex_mesh(n)}[kind]()
    tile_of, rnd, lane, nodes, info = plan_partition(m.elem_type, m.coords, m.conn, tile)
    ne = m.n_el
    # the kernel's vertex order is a permutation of each element's vertices
    np.testing.assert_array_equal(np.sort(nodes, axis=1), np.sort(m.conn, axis=1))
    # every element exactly once: (round, lane) pairs are unique
    key = rnd * 32 + lane
    assert len(np.unique(key)) == ne
    assert np.all((lane >= 0) & (lane < 32))
    # no node repeats within a round (the element colouring)
    order = np.argsort(rnd, kind="stable")
    r_sorted = rnd[order]
    bounds = np.flatnonzero(np.diff(r_sorted)) + 1
    for grp in np.split(order, bounds):
        nodes = m.conn[grp].ravel()
        assert len(np.unique(nodes)) == nodes.size
        assert len(np.unique(tile_of[grp])) == 1   # a round lies inside one tile
    # tiles are at most the requested size and cover everything
    T = tile if tile > 0 else (512 if kind == "hex" else 1024)
    assert np.bincount(tile_of).max() <= T
    assert info["n_tiles"] == tile_of.max() + 1
    # shared-node bookkeeping: slots = sum over nodes of (#tiles touching) for shared nodes
    node_tiles = {}
    for e in range(ne):
        for nd in m.conn[e]:
            node_tiles.setdefault(int(nd), set()).add(int(tile_of[e]))
    counts = np.array([len(s) for s in node_tiles.values()])
    assert info["n_shared"] == int((counts > 1).sum())
    assert info["n_slots"] == int(counts[counts > 1].sum())
    assert 0 < info["round_fill"] <= 1.0


def test_plan_is_deterministic(lib):
    from paper_2602_12365_b300.fem import plan_partition
    m = mg.tet_mesh(6, jitter_seed=3)
    a = plan_partition(m.elem_type, m.coords, m.conn, 128)
    b = plan_partition(m.elem_type, m.coords, m.conn, 128)
    for x, y in zip(a[:4], b[:4]):
        np.testing.assert_array_equal(x, y)


def test_round_repair_is_deterministic(lib):
    """The tabu repair draws from a generator seeded by each tile's first
    element, and tiles are built on several host threads: two plans of the
    same mesh are identical, round for round and lane for lane."""
    from paper_2602_12365_b300.fem import plan_partition
    m = mg.tet_mesh(16, jitter_seed=2)
    a = plan_partition(m.elem_type, m.coords, m.conn, 0)
    b = plan_partition(m.elem_type, m.coords, m.conn, 0)
    assert a[4]["max_rounds"] == 32  # every tile repaired to the floor
    for x, y in zip(a[:4], b[:4]):
        np.testing.assert_array_equal(x, y)


@pytest.mark.parametrize("n,tile", [(16, 512), (16, 256), (8, 256)])
def test_structured_hex_rounds_are_full(lib, n, tile):
    """On a structured Q1 grid whose tiles are boxes of at least 256 cells
    (each cell parity then has a multiple of 32 cells), the class-first
    colouring finds the 8 parities: every round holds 32 elements.  (Smaller
    boxes cap a round at the parity class: 8 cells in a 4 x 4 x 4 box.)"""
    from paper_2602_12365_b300.fem import plan_partition
    m = mg.hex_mesh(n)
    *_, info = plan_partition(m.elem_type, m.coords, m.conn, tile)
    assert info["n_rounds"] == m.n_el // 32 and info["round_fill"] == 1.0


def test_tet_round_fill_benchmark_family(lib):
    """Kuhn tets (jittered), 1024-element tiles: the tabu repair of the
    colouring reaches the floor ceil(E / 32) in every tile, i.e. 32 rounds of
    32 elements, still node-disjoint (the greedy orders alone leave most of
    these tiles at 33 rounds)."""
    from paper_2602_12365_b300.fem import plan_partition
    m = mg.tet_mesh(16, jitter_seed=1)
    tile_of, rnd, lane, nodes, info = plan_partition(m.elem_type, m.coords, m.conn, 0)
    assert info["round_fill"] == 1.0 and info["max_rounds"] == 32
    per_tile = np.bincount(tile_of)
    rounds_of_tile = np.array([len(np.unique(rnd[tile_of == t])) for t in range(len(per_tile))])
    np.testing.assert_array_equal(rounds_of_tile, -(-per_tile // 32))
    order = np.argsort(rnd, kind="stable")
    bounds = np.flatnonzero(np.diff(rnd[order])) + 1
    for grp in np.split(order, bounds):
        assert len(grp) == 32 and len(np.unique(m.conn[grp])) == 4 * 32
