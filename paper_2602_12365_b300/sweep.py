"""One call of every entry point of the library on the benchmark meshes, for
a launch-by-launch profile (every kernel's device time and DRAM bytes under
ncu).  Nothing is timed here and nothing is checked beyond the device status.

    python -m paper_2602_12365_b300.sweep            # tet64 (FP32) then hex64 (FP32)

Order (tet64, 1,572,864 P1 tets, random moduli): energy, residual, HVP,
block diagonal, parameter VJP, a tangent solve (stored linearisation, PCG
kernels), the learned preconditioner's features, network and blocks, one
training step, Algorithm 2's assembly and the CSR product, the atomic
ablation (residual, HVP, K), the neural constitutive model (coefficients on
the tensor cores, residual, HVP); then hex64 (262,144 Q1 hexes): residual,
HVP, a tangent solve (per-point stored linearisation).
"""
from __future__ import annotations

import argparse
import os

import torch

from . import meshgen as mg
from .fem import Mesh

HERE = os.path.dirname(os.path.abspath(__file__))


def tet_sweep(n: int) -> None:
    from .learned import LearnedPreconditioner
    m = mg.workload_tet(n, seed=101, random_moduli=101)
    gm = Mesh.from_fixture(m, precision="mixed")
    u = torch.as_tensor(mg.smooth_state(m, 0.5).ravel(), dtype=torch.float32, device="cuda")
    v = torch.as_tensor(mg.random_direction(m, 1).ravel(), dtype=torch.float32, device="cuda")
    gm.energy(u)
    gm.residual(u)
    gm.hvp(u, v)
    gm.block_diag(u)
    gm.param_vjp(u, v)
    ud = torch.zeros(m.n_nodes * 3, dtype=torch.float64, device="cuda")
    gm.tangent_solve(ud, v.double(), rtol=1e-2, cg_dtype=torch.float32)
    lp = LearnedPreconditioner.load(os.path.join(HERE, "weights", "lp_tet64.npz"))
    LearnedPreconditioner.features(gm, u)
    lp.blocks(gm, u)
    lp.train_step(gm, u, gm.residual(u), 1e-4)
    vals = gm.sparse_assemble(u)
    gm.sparse_spmv(vals, v)
    gm.residual_atomic(u)
    gm.hvp_atomic(u, v)
    gm.sparse_assemble_atomic(u)
    gm.set_ncm(32, mg.ncm_params(32, seed=7))
    gm.residual(u)
    gm.hvp(u, v)
    torch.cuda.synchronize()
    assert gm.sync_status() == 0


def hex_sweep(n: int) -> None:
    m = mg.workload_hex(n)
    gm = Mesh.from_fixture(m, precision="mixed")
    u = torch.as_tensor(mg.smooth_state(m, 0.5).ravel(), dtype=torch.float32, device="cuda")
    v = torch.as_tensor(mg.random_direction(m, 1).ravel(), dtype=torch.float32, device="cuda")
    gm.residual(u)
    gm.hvp(u, v)
    ud = torch.zeros(m.n_nodes * 3, dtype=torch.float64, device="cuda")
    gm.tangent_solve(ud, v.double(), rtol=1e-2, cg_dtype=torch.float32)
    torch.cuda.synchronize()
    assert gm.sync_status() == 0


def main() -> None:
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--tet", type=int, default=64, help="tet cells per side (0: skip)")
    ap.add_argument("--hex", type=int, default=64, help="hex cells per side (0: skip)")
    a = ap.parse_args()
    if a.tet:
        tet_sweep(a.tet)
    if a.hex:
        hex_sweep(a.hex)
    print("sweep done")


if __name__ == "__main__":
    main()
