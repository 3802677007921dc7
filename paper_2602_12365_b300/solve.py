"""Run a Newton-CG load path on one of the synthetic workloads.

    python -m paper_2602_12365_b300.solve --workload tet --n 64 --moduli 101 \
        --steps 2 --of 20 --cg f32 [--learned weights.npz]

Prints one line per load step (seconds, Newton and CG iterations, residual
norms).  The workloads are those of meshgen: ``tri`` (plane strain, clamp and
pull), ``tet`` (Kuhn tets, base clamped, top compressed 20 %), ``hex`` (Q1,
lognormal moduli, top sheared).
"""
from __future__ import annotations

import argparse
import time

import torch

from . import meshgen as mg
from .fem import Mesh


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="tet", choices=["tri", "tet", "hex"])
    ap.add_argument("--n", type=int, default=64, help="cells per side")
    ap.add_argument("--seed", type=int, default=None, help="jitter / moduli seed (default: --moduli or 0)")
    ap.add_argument("--moduli", type=int, default=None, help="tet: lognormal per-element moduli from this seed")
    ap.add_argument("--steps", type=int, default=1, help="load steps to run")
    ap.add_argument("--of", type=int, default=20, help="load steps of the whole path")
    ap.add_argument("--cg", default="f32", choices=["f32", "f64"])
    ap.add_argument("--learned", default=None, help="weights (.npz) of the learned preconditioner")
    ap.add_argument("--adjoint", action="store_true",
                    help="then the compliance and its gradient in the per-element mu (lambda = 10 mu)")
    a = ap.parse_args()
    seed = a.seed if a.seed is not None else (a.moduli if a.moduli is not None else 0)
    if a.workload == "tri":
        m = mg.workload_tri(a.n)
    elif a.workload == "tet":
        m = mg.workload_tet(a.n, seed=seed, random_moduli=a.moduli)
    else:
        m = mg.workload_hex(a.n, seed=seed)
    gm = Mesh.from_fixture(m, precision="mixed")
    kw = {}
    if a.learned:
        from .learned import LearnedPreconditioner
        kw["learned"] = LearnedPreconditioner.load(a.learned)
    dt = torch.float32 if a.cg == "f32" else torch.float64
    u = torch.zeros(m.n_nodes * m.dim, dtype=torch.float64, device="cuda")
    ubar = torch.as_tensor(m.ubar.ravel(), dtype=torch.float64, device="cuda")
    s_prev = 0.0
    for k in range(1, a.steps + 1):
        s = k / a.of
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st = gm.newton_step(u, ubar, s_prev, s, cg_dtype=dt, **kw)
        torch.cuda.synchronize()
        print(f"step {k}/{a.of} s={s:.4f}: {time.perf_counter() - t0:.3f} s, newton {st['newton_iters']}, "
              f"cg {st['cg_iters']}, |r| {st['r_norm']:.3e} / r0 {st['r0_norm']:.3e}", flush=True)
        s_prev = s
    if a.adjoint:
        from .adjoint import compliance_gradient
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        c, g, iters = compliance_gradient(gm, u, rtol=1e-8, cg_dtype=dt, vjp_dtype=dt)
        torch.cuda.synchronize()
        print(f"adjoint: {time.perf_counter() - t0:.3f} s, c = {c:.6e}, |dc/dmu| = {torch.linalg.norm(g).item():.6e}, "
              f"cg {iters}", flush=True)


if __name__ == "__main__":
    main()
