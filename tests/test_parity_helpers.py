"""The per-node parity helpers (tests/parity.py) on the CPU: the exploded-mesh
element contributions add up to the oracle's nodal residual and HVP, and the
per-node bound catches a single bad node that the whole-vector 2-norm bar lets
through."""
import numpy as np
import pytest

import oracle
import parity
from paper_2602_12365_b300 import meshgen as mg


@pytest.mark.parametrize("kind", ["tri", "tet", "hex"])
def test_contributions_sum_to_the_oracle(kind):
    m = {"tri": lambda: mg.workload_tri(6), "tet": lambda: mg.workload_tet(3, seed=2, random_moduli=3),
         "hex": lambda: mg.workload_hex(3, seed=1)}[kind]()
    om = oracle.OracleMesh.from_mesh(m)
    u = mg.smooth_state(m, 0.5).ravel()
    v = mg.random_direction(m, 1).ravel()
    for vv in (None, v):
        c, conn = parity.element_contributions(om, u, vv)
        tot = np.zeros((m.n_nodes, m.dim))
        np.add.at(tot, conn.reshape(-1), c.reshape(-1, m.dim))
        ref = om.residual(u, mask_out=False) if vv is None else om.hvp(u, v, mask_in=False, mask_out=False)
        ref = ref.reshape(-1, m.dim)
        s = parity.node_scale(m.n_nodes, conn, c)
        assert np.all(s > 0)
        assert parity.per_node_excess(tot, ref, s, 1e-12) <= 1.0


def test_per_node_bound_catches_one_bad_node():
    m = mg.workload_tet(10, seed=2)
    om = oracle.OracleMesh.from_mesh(m)
    u = mg.smooth_state(m, 0.5).ravel()
    c, conn = parity.element_contributions(om, u)
    s = parity.node_scale(m.n_nodes, conn, c)
    ref = om.residual(u, mask_out=False).reshape(-1, 3)
    bad = ref.copy()
    i = int(np.argmin(np.where(s > 0, s, np.inf)))  # the node with the smallest scale
    bad[i] += 20e-5 * s[i]  # 20x the FP32 per-node bar at that node
    rel = np.linalg.norm(bad - ref) / np.linalg.norm(ref)
    assert rel <= 1e-5  # the whole-vector bar misses it
    assert parity.per_node_excess(bad, ref, s, 1e-5) > 1.0
    # an orphan node (no element) must match exactly
    s2 = s.copy()
    s2[i] = 0.0
    assert parity.per_node_excess(bad, ref, s2, 1e-5) == np.inf
