"""Learned block preconditioner: handle, training data and training loop.

The network and its kernels are described in include/fem_b300.h (fem_lp_*):
a per-node MLP corrects block Jacobi, M_i = F A A^T F^T / s_i, and starts as
block Jacobi exactly.  Training samples are states u and residuals r that the
method itself produces on its load path: at every load step of a Newton-CG
solve, the converged state with the next step's prescribed values (the
residual a Newton solve starts from), and states part of the way to the next
converged state.  The loss is ||H M r - r||^2 / ||r||^2, H = M K(u) M.

Command line (trains on random-modulus tet meshes and writes the weights):
    python -m paper_2602_12365_b300.learned --n 64 --meshes 16 --out lp.npz
"""
from __future__ import annotations

import argparse
import ctypes as C
import time

import numpy as np
import torch

from . import _lib as L
from . import meshgen as mg
from .fem import Mesh, _ptr, _stream


class LearnedPreconditioner:
    """Owns a fem_lp handle (FP32 master weights, Adam state, BF16 copy)."""

    N_PARAMS = L.FEM_LP_PARAMS

    def __init__(self, seed: int = 0, loss: str = "residual"):
        h = C.c_void_p()
        L.check(L.lib().fem_lp_create(C.c_uint64(seed), C.byref(h)))
        self._h = h
        self.set_loss(loss)

    def set_loss(self, loss: str) -> None:
        """'residual': ||H M r - r||^2 / ||r||^2; 'energy': the same in the
        H^-1 norm (see fem_lp_set_loss)."""
        kind = {"residual": L.FEM_LP_LOSS_RESIDUAL, "energy": L.FEM_LP_LOSS_ENERGY}[loss]
        L.check(L.lib().fem_lp_set_loss(self._h, kind))
        self.loss = loss

    def set_clip(self, max_grad_norm: float) -> None:
        """Gradient-norm clipping of the Adam steps (0: none)."""
        L.check(L.lib().fem_lp_set_clip(self._h, C.c_float(max_grad_norm)))

    def close(self):
        if getattr(self, "_h", None):
            L.lib().fem_lp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    def params(self) -> np.ndarray:
        p = np.zeros(self.N_PARAMS, np.float32)
        L.check(L.lib().fem_lp_get_params(self._h, p.ctypes.data_as(C.c_void_p)))
        return p

    def set_params(self, p) -> None:
        p = np.ascontiguousarray(p, dtype=np.float32)
        assert p.size == self.N_PARAMS
        L.check(L.lib().fem_lp_set_params(self._h, p.ctypes.data_as(C.c_void_p)))

    def save(self, path: str) -> None:
        np.savez(path, params=self.params())

    @classmethod
    def load(cls, path: str) -> "LearnedPreconditioner":
        lp = cls(0)
        lp.set_params(np.load(path)["params"])
        return lp

    @staticmethod
    def unpack(p):
        """(W1, b1, W2, b2, W3, b3) views of a parameter vector."""
        o = 0
        out = []
        for shape in ((64, 36), (64,), (64, 64), (64,), (6, 64), (6,)):
            n = int(np.prod(shape))
            out.append(np.asarray(p[o:o + n]).reshape(shape))
            o += n
        return out

    def blocks(self, mesh: Mesh, u32: torch.Tensor, stream=None) -> torch.Tensor:
        """Preconditioner blocks [n_nodes, 3, 3] (FP32) at the FP32 state u."""
        M = torch.empty(mesh.n_nodes * 9, dtype=torch.float32, device=u32.device)
        L.check(L.lib().fem_lp_blocks(self._h, mesh._h, _ptr(u32), _ptr(M), _stream(stream)))
        return M.view(-1, 3, 3)

    @staticmethod
    def features(mesh: Mesh, u32: torch.Tensor, stream=None) -> torch.Tensor:
        """Features [n_nodes, 48] (BF16; columns 36..47 are zero)."""
        X = torch.empty(mesh.n_nodes * 48, dtype=torch.bfloat16, device=u32.device)
        L.check(L.lib().fem_lp_features(mesh._h, _ptr(u32), _ptr(X), _stream(stream)))
        return X.view(-1, 48)

    def gradient(self, mesh: Mesh, u32, r32, stream=None):
        g = np.zeros(self.N_PARAMS, np.float32)
        loss = C.c_double(0.0)
        L.check(L.lib().fem_lp_gradient(self._h, mesh._h, _ptr(u32), _ptr(r32),
                                        g.ctypes.data_as(C.c_void_p), C.byref(loss), _stream(stream)))
        return loss.value, g

    def train_step(self, mesh: Mesh, u32, r32, lr: float, want_loss: bool = True, stream=None):
        loss = C.c_double(0.0)
        L.check(L.lib().fem_lp_train_step(self._h, mesh._h, _ptr(u32), _ptr(r32), C.c_float(lr),
                                          C.byref(loss) if want_loss else None, _stream(stream)))
        return loss.value if want_loss else None


def load_path_samples(mesh: Mesh, m, n_steps: int, total_steps: int = 20, thetas=(0.0, 0.5)):
    """(u, r) FP32 pairs along the mixed-precision block-Jacobi load path of
    ``m``: for each step k and theta, the state u_k + theta (u_{k+1} - u_k)
    with prescribed values at s_k + theta (s_{k+1} - s_k) (theta = 0: the
    state a Newton solve starts from), and its masked residual."""
    dev = "cuda"
    u = torch.zeros(m.n_nodes * m.dim, dtype=torch.float64, device=dev)
    ubar = torch.as_tensor(m.ubar.ravel(), dtype=torch.float64, device=dev)
    mask = mesh.dirichlet_mask(dev)
    out = []
    s_prev = 0.0
    for k in range(1, n_steps + 1):
        s = k / total_steps
        u_prev = u.clone()
        st = mesh.newton_step(u, ubar, s_prev, s, cg_dtype=torch.float32)
        assert st["status"] == 0, st
        for th in thetas:
            if th == 0.0:  # the previous state under the new prescribed values
                ut = torch.where(mask, s * ubar, u_prev)
            else:          # part of the way to the new equilibrium
                ut = u_prev + th * (u - u_prev)
            r = mesh.residual(ut, mask_out=True)
            out.append((ut.float().contiguous(), r.float().contiguous()))
        s_prev = s
    return out


def protocol_samples(mesh: Mesh, m, thetas=(0.0, 0.2, 0.4, 0.6, 0.8), cg_thetas=(0.0, 0.4),
                     cg_iters=(10, 40, 160, 640), total_steps: int = 20):
    """(u, r) FP32 pairs the method generates along the 20-step mixed
    block-Jacobi load path of ``m``.  For each load step k: the states
    u_k + theta (u_{k+1} - u_k) (prescribed values at s_k + theta ds; theta =
    0 is the state a Newton solve starts from) with their masked Newton
    residuals, and, at the states of ``cg_thetas``, the residuals b - M K M x_j
    of the Newton system M K M d = -r after j block-Jacobi PCG iterations
    (``cg_iters``): the slow modes that block Jacobi leaves behind late in a
    solve.  20 x (5 + 2 x 4) = 260 samples per mesh with the defaults.
    Returns (samples, kinds), kinds[i] "newton" or "cg"."""
    dev = "cuda"
    u = torch.zeros(m.n_nodes * m.dim, dtype=torch.float64, device=dev)
    ubar = torch.as_tensor(m.ubar.ravel(), dtype=torch.float64, device=dev)
    mask = mesh.dirichlet_mask(dev)
    out, kinds = [], []
    s_prev = 0.0
    for k in range(1, total_steps + 1):
        s = k / total_steps
        u_prev = u.clone()
        st = mesh.newton_step(u, ubar, s_prev, s, cg_dtype=torch.float32)
        assert st["status"] == 0, st
        for th in thetas:
            ut = torch.where(mask, (s_prev + th * (s - s_prev)) * ubar, u_prev + th * (u - u_prev))
            if th == 0.0:
                ut = torch.where(mask, s * ubar, u_prev)  # the previous state under the new prescribed values
            r = mesh.residual(ut, mask_out=True)
            out.append((ut.float().contiguous(), r.float().contiguous()))
            kinds.append("newton")
            if th in cg_thetas:
                b = -r
                for j in cg_iters:
                    x, _, _ = mesh.tangent_solve(ut, b, rtol=1e-30, cg_dtype=torch.float32, cg_max=j, check=False)
                    rj = torch.where(mask, torch.zeros_like(b), b) - mesh.hvp(ut, x, mask_in=True, mask_out=True)
                    if torch.linalg.norm(rj) > 0:
                        out.append((ut.float().contiguous(), rj.float().contiguous()))
                        kinds.append("cg")
        s_prev = s
    return out, kinds


def evaluate(lp, seeds=(101, 102, 103, 104), n: int = 64, steps: int = 20):
    """Mixed-precision Newton-CG over the first ``steps`` load steps of the
    20-step path on each unseen seed, block Jacobi against the learned blocks:
    CG iterations and seconds (CUDA events) per arm, and the relative
    difference of the final displacements."""
    out = {"block_jacobi": {"cg": 0, "s": 0.0}, "learned": {"cg": 0, "s": 0.0}, "u_rel_diff_max": 0.0}
    for sd in seeds:
        m = mg.workload_tet(n, seed=sd, random_moduli=sd)
        mesh = Mesh.from_fixture(m)
        ubar = torch.as_tensor(m.ubar.ravel(), dtype=torch.float64, device="cuda")
        finals = {}
        for arm, kw in (("block_jacobi", {}), ("learned", {"learned": lp})):
            u = torch.zeros(m.n_nodes * 3, dtype=torch.float64, device="cuda")
            mesh.newton_step(u, ubar, 0.0, 0.0, cg_dtype=torch.float32, **kw)  # workspace
            s_prev = 0.0
            for k in range(1, steps + 1):
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record()
                st = mesh.newton_step(u, ubar, s_prev, k / 20, cg_dtype=torch.float32, check=False, **kw)
                b.record()
                b.synchronize()
                if st["status"] != 0:  # recorded, not raised: a failed arm is a result
                    out[arm]["failed"] = f"seed {sd}, load step {k}: status {st['status']}"
                    break
                out[arm]["cg"] += st["cg_iters"]
                out[arm]["s"] += a.elapsed_time(b) * 1e-3
                s_prev = k / 20
            finals[arm] = u
            if "failed" in out[arm]:
                break
        if any("failed" in out[a] for a in ("block_jacobi", "learned")):
            break
        d = torch.linalg.norm(finals["learned"] - finals["block_jacobi"]) / torch.linalg.norm(finals["block_jacobi"])
        out["u_rel_diff_max"] = max(out["u_rel_diff_max"], float(d))
    if any("failed" in out[a] for a in ("block_jacobi", "learned")):
        out["cg_ratio"] = out["time_ratio"] = float("inf")
        return out
    out["cg_ratio"] = out["learned"]["cg"] / out["block_jacobi"]["cg"]
    out["time_ratio"] = out["learned"]["s"] / out["block_jacobi"]["s"]
    return out


def train(lp: LearnedPreconditioner, datasets, epochs: int, lr: float = 1e-3, seed: int = 0,
          log_every: int = 0):
    """Adam over (mesh, [(u, r), ...]) datasets, samples in a seeded random
    order each epoch; returns the per-epoch mean loss."""
    rng = np.random.default_rng(seed)
    items = [(mi, si) for mi, (_, samples) in enumerate(datasets) for si in range(len(samples))]
    history = []
    for ep in range(epochs):
        order = rng.permutation(len(items))
        tot = 0.0
        for j, k in enumerate(order):
            mi, si = items[k]
            mesh, samples = datasets[mi]
            u, r = samples[si]
            tot += lp.train_step(mesh, u, r, lr)
            if log_every and (j + 1) % log_every == 0:
                print(f"epoch {ep} sample {j + 1}/{len(items)} mean loss {tot / (j + 1):.5f}", flush=True)
        history.append(tot / len(items))
    return history


def sample_loss(lp: LearnedPreconditioner, datasets) -> float:
    tot, n = 0.0, 0
    for mesh, samples in datasets:
        for u, r in samples:
            tot += lp.gradient(mesh, u, r)[0]
            n += 1
    return tot / max(n, 1)


def main():
    """The training protocol: 4096 (u, r) samples from the method's own load
    paths on 16 seeded random-modulus 64^3 meshes (seeds 1-16), Adam on the
    chosen loss, then the evaluation on the unseen seeds 101-104 against
    block Jacobi (20 load steps each).  --variants trains every (loss, data)
    combination on the same samples and prints one JSON line per variant."""
    import json
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=64)
    ap.add_argument("--meshes", type=int, default=16, help="training seeds 1..meshes")
    ap.add_argument("--samples", type=int, default=4096)
    ap.add_argument("--epochs", type=int, default=6)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--loss", default="residual", choices=["residual", "energy"])
    ap.add_argument("--data", default="newton+cg", choices=["newton", "newton+cg"])
    ap.add_argument("--variants", action="store_true", help="train and evaluate every loss x data variant")
    ap.add_argument("--only", default="", help="comma-separated loss:data variants (overrides --variants)")
    ap.add_argument("--eval-steps", type=int, default=20)
    ap.add_argument("--out", default="lp_weights.npz")
    a = ap.parse_args()
    t0 = time.time()
    rng = np.random.default_rng(a.seed)
    pools = []
    for sd in range(1, a.meshes + 1):
        m = mg.workload_tet(a.n, seed=sd, random_moduli=sd)
        mesh = Mesh.from_fixture(m)
        smp, kinds = protocol_samples(mesh, m)
        pools.append((mesh, smp, kinds))
        print(f"mesh seed {sd}: {len(smp)} samples, {time.time() - t0:.1f} s", flush=True)
    per = a.samples // a.meshes

    def take(kind):
        ds = []
        for mesh, smp, kinds in pools:
            idx = [i for i in range(len(smp)) if kind == "newton+cg" or kinds[i] == "newton"]
            pick = rng.choice(len(idx), size=min(per, len(idx)), replace=False)
            ds.append((mesh, [smp[idx[i]] for i in sorted(pick)]))
        return ds

    variants = ([(lo, da) for lo in ("residual", "energy") for da in ("newton", "newton+cg")]
                if a.variants else [(a.loss, a.data)])
    if a.only:
        variants = [tuple(v.split(":")) for v in a.only.split(",")]
    best = None
    for loss, data in variants:
        ds = take(data)
        lp = LearnedPreconditioner(a.seed, loss)
        before = sample_loss(lp, ds)
        hist = train(lp, ds, a.epochs, a.lr, a.seed)
        ev = evaluate(lp, steps=a.eval_steps)
        row = {"loss": loss, "data": data, "samples": sum(len(x) for _, x in ds), "epochs": a.epochs,
               "loss_before": before, "loss_after": hist[-1], **ev, "elapsed_s": time.time() - t0}
        print(json.dumps(row), flush=True)
        if best is None or ev["cg_ratio"] < best[0]:
            best = (ev["cg_ratio"], lp, loss, data)
            lp.save(a.out)  # the best so far
    print(f"best: loss {best[2]}, data {best[3]}, CG ratio {best[0]:.4f}", flush=True)


if __name__ == "__main__":
    main()
