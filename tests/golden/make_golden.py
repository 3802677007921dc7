"""Writes the oracle fixtures of this folder (run from the repository root:
``python tests/golden/make_golden.py``).  Only the oracle computes the
stored outputs; the inputs come from the seeded mesh and state generators.

Each fixture holds a tiny mesh (coordinates, connectivity, per-element
moduli, Dirichlet mask), a state u and a direction v, and the oracle's FP64
energy (Eq. 2), residual (Eq. 1, Dirichlet rows zero), Hessian-vector
product (Sec. 2.1, masked in and out) and nodal 3x3 / 2x2 diagonal blocks.
The tests recompute them with the oracle (a guard against silent changes of
the oracle) and compare the CUDA path against the stored values.
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_2602_12365_b300 import meshgen as mg  # noqa: E402

CASES = {
    # name: (mesh, state load factor, state amplitude, direction seed)
    "tri3_plane_strain_3x3": (lambda: mg.workload_tri(3), 0.5, 0.05, 2),
    "tet4_jittered_2x2x2": (lambda: mg.workload_tet(2, seed=7, random_moduli=7), 0.5, 0.05, 3),
    "hex8_lognormal_2x2x2": (lambda: mg.workload_hex(2, seed=5), 0.5, 0.05, 4),
}


def fixture(name):
    make, s, amp, vseed = CASES[name]
    m = make()
    om = oracle.OracleMesh.from_mesh(m)
    u = mg.smooth_state(m, s, amp=amp).ravel()
    v = mg.random_direction(m, vseed).ravel()
    psi, _, S, st = om.energy(u, per_element=True)
    assert st == 0
    return {
        "what": "oracle outputs (FP64) on a tiny seeded mesh; written by tests/golden/make_golden.py",
        "cites": "Eq. 2 (energy), Eq. 1 (residual), Sec. 2.1 (Hessian-vector product); Dirichlet masking of Sec. 3",
        "elem_type": int(m.elem_type),
        "coords": m.coords.tolist(),
        "conn": m.conn.tolist(),
        "mu": m.mu_e().tolist(),
        "lam": m.lam_e().tolist(),
        "dirichlet": (np.zeros((m.n_nodes, m.dim), np.uint8) if m.dirichlet is None else m.dirichlet).tolist(),
        "u": u.tolist(),
        "v": v.tolist(),
        "energy": psi,
        "energy_scale": S,
        "residual": om.residual(u).tolist(),
        "hvp": om.hvp(u, v).tolist(),
        "block_diag": om.block_diag(u).ravel().tolist(),
    }


def main():
    for name in CASES:
        with open(os.path.join(HERE, name + ".json"), "w") as f:
            json.dump(fixture(name), f, indent=0)
            f.write("\n")


if __name__ == "__main__":
    main()
