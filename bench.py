#!/usr/bin/env python3
"""Benchmark: residual + HVP throughput of the energy-based FEM hot path.

Workload: 64^3 cube of Kuhn tetrahedra (1,572,864 P1 elements, 274,625 nodes,
interior nodes jittered by U(-0.1h, 0.1h) from seed 0), compressible
Neo-Hookean mu = 1, lambda = 10, base clamped and top prescribed; FP32
element kernels with FP64 reductions.  One step = one residual + one HVP at
the BC-consistent state u (load factor 0.5: affine part plus a 0.02 sine
bump) along v ~ N(0, 1) on free DOFs.  Metric: elements per second of the
pair, N_el / (t_residual + t_hvp), in GElem/s.

L2 (126 MB) is flushed before every timed step by writing a 256 MB buffer and
then reading another 256 MB one (so the flush's dirty lines are written back
before the timed kernels start); each step is timed with CUDA events on the
stream the kernels run on.
The line also carries: the same step warm (L2 not flushed, "warm"); the
Newton-CG measurement ("newton"): seconds per load step to relative residual
1e-8 on the 64^3 random-moduli tet family, every load step of the 20-step
path on seeds 101-104, FP64 against mixed precision (FP32 CG with FP64 dots,
FP64 residual and energy) with block-Jacobi PCG, and mixed precision with the
learned block preconditioner (weights trained on seeds 1-16, so these seeds
are unseen); the 128^3 Q1 hex workload ("hex128": residual and HVP against a
measured FP32 FMA rate, and its mixed Newton-CG load path); the FP32 path's
error against the FP64 path and the FP64 oracle at the benchmark's FP64 state
("precision_error"); and the oracle on one pinned host core
("cpu_baseline").  `--impl reference` times the FP64 CPU oracle instead (the
reference arm).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# Algorithmic bytes per element for the tet workload (FP32): element stream
# conn 16 + 3 grad N 36 + w detJ 4 = 56 B, plus nodal vectors at 0.1746 nodes
# per element: residual u 12 + r 12 + mask 1 = 25 B, HVP u 12 + v 12 + y 12 +
# mask 1 = 37 B (each read or written once).
B_RES_PER_EL = 60.4
B_HVP_PER_EL = 62.5
WORKLOAD = "tet64"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cells", dest="n", type=int, default=64, help="cells per side of the tet workload")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-ncm", action="store_true", help="skip the neural-constitutive-model measurement")
    ap.add_argument("--no-sparse", action="store_true",
                    help="skip the sparse-K (Algorithm 2) and atomic-scatter ablation measurements")
    ap.add_argument("--newton-steps", type=int, default=20,
                    help="load steps of the Newton-CG measurement per arm and seed (0 = skip)")
    ap.add_argument("--newton-seeds", default="101,102,103,104",
                    help="mesh seeds of the Newton-CG measurement (the learned preconditioner's unseen seeds)")
    ap.add_argument("--no-hex", action="store_true", help="skip the 128^3 Q1 hex measurement")
    ap.add_argument("--hex-steps", type=int, default=10, help="load steps of the hex128 mixed Newton measurement")
    return ap.parse_args()


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6400.0, "fallback"


# the sources that define what a residual or HVP call runs (tile and
# finalize kernels, plan, records, launch); the solver, learned-
# preconditioner, sparse and ablation sources do not change those kernels
KERNEL_SOURCES = ("fem_api.cu", "fem_internal.h", "fem_kernels.cuh", "fem_material.cuh", "fem_pair.cuh",
                  "fem_plan.cpp", "fem_plan.h", "fem_vec.cuh")


SPMV_SOURCES = ("fem_spmv.cu",)


def kernel_source_hash(files=KERNEL_SOURCES):
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2602_12365_b300", "csrc")
    for f in files:
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def traffic_for(kernel_tag, files=KERNEL_SOURCES):
    """DRAM bytes per call from a committed ncu summary, if it was taken on
    the current kernel sources (else None)."""
    p = os.path.join(ROOT, "profiles", f"{kernel_tag}.traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    if d.get("source_hash") != kernel_source_hash(files):
        return None
    return d.get("dram_bytes_per_call")


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            out, _ = self.proc.communicate(timeout=10)
            self.lines = out.splitlines()

    def summary(self):
        if not self.proc or not self.lines:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        rows = []
        for line in self.lines:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for _, _, parts in rows:
            for k, nm in enumerate(names):
                if parts[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(r[0] for r in rows),
                "sm_max_mhz": max(r[1] for r in rows), "reasons": sorted(reasons),
                "samples": len(rows)}


def dist_init(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if args.impl == "ours" else "gloo")
    return world, rank, local


def max_over_ranks(x, world, device=None):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def workload(n):
    from paper_2602_12365_b300 import meshgen as mg
    m = mg.workload_tet(n, seed=0)
    u = mg.smooth_state(m, 0.5).ravel()
    v = mg.random_direction(m, 1).ravel()
    return m, u, v


def config_dict(m, step, extra=None):
    d = {"workload": f"{WORKLOAD}: 3D P1 Kuhn tetrahedra on a {m.n}^3 unit cube, "
                     f"{m.n_el} elements, {m.n_nodes} nodes, interior jitter 0.1h (seed 0), "
                     "Neo-Hookean mu=1 lambda=10, base clamped, top prescribed; "
                     "u = BC-consistent state at load factor 0.5, v ~ N(0,1) on free DOFs",
         "n_el": m.n_el, "n_nodes": m.n_nodes, "step": step,
         "l2": "flushed before every timed step (256 MB write, then 256 MB read)",
         "parallelism": "replicas"}
    if extra:
        d.update(extra)
    return d


def run_reference(args):
    world, rank, _ = dist_init(args)
    if rank != 0:
        return
    import oracle
    m, u, v = workload(args.n)
    # each step: oracle residual + HVP over a fixed contiguous quarter of the
    # elements (a bounded sample of the same workload)
    ne = m.n_el // 4
    sub = oracle.OracleMesh(m.elem_type, m.coords, m.conn[:ne], m.mu_e()[:ne], m.lam_e()[:ne],
                            m.dirichlet)
    try:
        core = min(os.sched_getaffinity(0))
        os.sched_setaffinity(0, {core})
        pinned = f"core {core} (sched_setaffinity, as taskset -c {core})"
    except (AttributeError, OSError):
        pinned = "not pinned"
    for _ in range(args.warmup):
        sub.residual(u)
        sub.hvp(u, v)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        sub.residual(u)
        sub.hvp(u, v)
    dt = time.perf_counter() - t0
    val = ne * args.steps / dt / 1e9
    sample = f"oracle residual+HVP over the first {ne} of {m.n_el} elements, {args.steps} steps"
    line = {"impl": "reference", "metric": "residual+HVP GElem/s", "value": val, "unit": "GElem/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_dict(m, "1 residual + 1 HVP (FP64 CPU oracle, 1 thread)",
                                  {"sample": sample}),
            "cpu_baseline": {"value": val, "unit": "GElem/s", "cores": 1, "kind": "oracle",
                             "sample": sample, "cpu_model": cpu_info()[0], "nproc": cpu_info()[1],
                             "pinned": pinned},
            "e2e": {"value": val, "unit": "GElem/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


NEWTON_WORKLOAD = ("tet64 random moduli (C4 family): 64^3 Kuhn tets (jitter seed = mesh seed), per-element mu "
                   "lognormal(0, 0.5) (same seed), lambda = 10 mu; base clamped, top compressed 20 % in 20 load steps")


def newton_arms(n, n_steps, seeds, dev):
    """Seconds per Newton-CG load step (relative residual 1e-8) on the 64^3
    random-moduli tet family, per arm: FP64 block Jacobi, mixed precision
    (FP32 CG, FP64 dots, FP64 residual and energy) with block Jacobi, and
    mixed with the learned block preconditioner (weights trained on seeds
    1-16 of the same family; the seeds here are unseen).  Every arm runs the
    first n_steps load steps of the 20-step path on every seed; the headline
    is the median over all those steps."""
    import torch
    from paper_2602_12365_b300 import meshgen as mg
    from paper_2602_12365_b300.fem import Mesh
    stream = torch.cuda.current_stream()
    arms = [("fp64_block_jacobi", torch.float64, False), ("mixed_block_jacobi", torch.float32, False)]
    weights = os.path.join(ROOT, "paper_2602_12365_b300", "weights", "lp_tet64.npz")
    lp = None
    if os.path.exists(weights):
        from paper_2602_12365_b300.learned import LearnedPreconditioner
        lp = LearnedPreconditioner.load(weights)
        arms.append(("mixed_learned", torch.float32, True))
    per = {a: {"s_each": [], "newton_iters": [], "cg_iters": [], "u_rel_diff_vs_fp64": [], "seeds": []}
           for a, _, _ in arms}
    for seed in seeds:
        m = mg.workload_tet(n, seed=seed, random_moduli=seed)
        gm = Mesh.from_fixture(m, precision="mixed")
        ubar = torch.as_tensor(m.ubar.ravel(), dtype=torch.float64, device=dev)
        finals = {}
        for arm, dt, learned in arms:
            kw = {"learned": lp} if learned else {}
            u = torch.zeros(m.n_nodes * 3, dtype=torch.float64, device=dev)
            # one-time setup outside the timing: the solver workspace (a step at
            # rest returns at once) and, for the learned arm, the node graph
            gm.newton_step(u, ubar, 0.0, 0.0, cg_dtype=dt, **kw)
            if learned:
                lp.blocks(gm, u.float())
            s_prev = 0.0
            times, newton, cg = [], [], []
            for k in range(1, n_steps + 1):
                s = k / 20
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                torch.cuda.synchronize()
                a.record(stream)
                st = gm.newton_step(u, ubar, s_prev, s, cg_dtype=dt, **kw)
                b.record(stream)
                b.synchronize()
                times.append(a.elapsed_time(b) * 1e-3)
                newton.append(st["newton_iters"])
                cg.append(st["cg_iters"])
                s_prev = s
            finals[arm] = u
            per[arm]["s_each"].append(times)
            per[arm]["newton_iters"].append(newton)
            per[arm]["cg_iters"].append(cg)
            per[arm]["seeds"].append(seed)
        ref = finals["fp64_block_jacobi"]
        for arm, u in finals.items():
            per[arm]["u_rel_diff_vs_fp64"].append(float(torch.linalg.norm(u - ref) / torch.linalg.norm(ref)))
        del gm
    out = {}
    for arm, d in per.items():
        flat = [t for ts in d["s_each"] for t in ts]
        out[arm] = {"s_per_load_step": statistics.median(flat),
                    "s_per_load_step_by_seed": [statistics.median(ts) for ts in d["s_each"]],
                    "newton_iters_per_step_median": statistics.median(x for xs in d["newton_iters"] for x in xs),
                    "cg_iters_per_step_median": statistics.median(x for xs in d["cg_iters"] for x in xs),
                    "cg_iters_total_by_seed": [sum(xs) for xs in d["cg_iters"]],
                    "u_rel_diff_vs_fp64_max": max(d["u_rel_diff_vs_fp64"]), **d}
    res = {"workload": NEWTON_WORKLOAD, "metric": "Newton-CG s/load step at relative residual 1e-8 "
                                                  "(median over every load step of every seed)",
           "seeds": list(seeds), "load_steps": list(range(1, n_steps + 1)), "arms": out}
    t64 = out["fp64_block_jacobi"]["s_per_load_step"]
    for arm in out:
        if arm != "fp64_block_jacobi":
            res[f"speedup_{arm}_vs_fp64_block_jacobi"] = t64 / out[arm]["s_per_load_step"]
    if "mixed_learned" in out:
        res["learned_vs_mixed_block_jacobi"] = {
            "time_ratio": out["mixed_learned"]["s_per_load_step"] / out["mixed_block_jacobi"]["s_per_load_step"],
            "cg_iter_ratio": (sum(out["mixed_learned"]["cg_iters_total_by_seed"]) /
                              sum(out["mixed_block_jacobi"]["cg_iters_total_by_seed"]))}
        res["learned_weights"] = "paper_2602_12365_b300/weights/lp_tet64.npz (trained on seeds 1-16)"
    return res


# FP32 flops per Q1 element of the hex operators (this formulation: J rebuilt
# at each of the 8 Gauss points, FMA = 2), counted by ncu on a hex64 call
# (smsp__sass_thread_inst_executed_op_{ffma,fadd,fmul}_pred_on.sum, every
# round full)
HEX_FLOPS_RES = 4.69e3
HEX_FLOPS_HVP = 6.57e3


def fp32_peak(dev, clk=None):
    """Measured FP32 FMA rate (TFLOP/s): the library's FMA-chain kernel on
    8 blocks of 256 threads per SM, best of 5 (CUDA events)."""
    import torch
    from paper_2602_12365_b300 import fem
    nsm = torch.cuda.get_device_properties(dev).multi_processor_count
    blocks = nsm * 8
    out = torch.empty(blocks * 256, dtype=torch.float32, device=dev)
    fl = fem.fp32_fma_rate(blocks, 4096, out)
    best = None
    for _ in range(5):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        fem.fp32_fma_rate(blocks, 4096, out)
        b.record()
        b.synchronize()
        t = a.elapsed_time(b) * 1e-3
        best = t if best is None else min(best, t)
    return fl / best / 1e12


def hex_arm(dev, flush_l2, steps, hex_steps):
    """The 128^3 Q1 hex workload (C3): residual and HVP (FP32 element kernels,
    L2 flushed before each call), their FP32 rate against the FMA rate
    measured here and the nominal one, and the mixed-precision Newton-CG
    seconds per load step over the 10-step shear path."""
    import torch
    from paper_2602_12365_b300 import meshgen as mg
    from paper_2602_12365_b300.fem import Mesh
    m = mg.workload_hex(128, seed=0)
    gm = Mesh.from_fixture(m, precision="mixed")
    ut = torch.as_tensor(mg.smooth_state(m, 0.5).ravel(), dtype=torch.float32, device=dev)
    vt = torch.as_tensor(mg.random_direction(m, 1).ravel(), dtype=torch.float32, device=dev)
    r, y = torch.empty_like(ut), torch.empty_like(ut)
    for k in range(3):
        flush_l2(k)
        gm.residual(ut, out=r)
        gm.hvp(ut, vt, out=y)
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(steps)]
    for k in range(steps):
        flush_l2(k)
        ev[k][0].record()
        gm.residual(ut, out=r)
        ev[k][1].record()
        gm.hvp(ut, vt, out=y)
        ev[k][2].record()
    torch.cuda.synchronize()
    assert gm.sync_status() == 0
    t_r = statistics.median(e[0].elapsed_time(e[1]) for e in ev) * 1e-3
    t_h = statistics.median(e[1].elapsed_time(e[2]) for e in ev) * 1e-3
    peak_meas = fp32_peak(dev)
    props = torch.cuda.get_device_properties(dev)
    nominal = props.multi_processor_count * 128 * 2 * 2.032e9 / 1e12
    tf_r = HEX_FLOPS_RES * m.n_el / t_r / 1e12
    tf_h = HEX_FLOPS_HVP * m.n_el / t_h / 1e12
    # the mixed Newton-CG load path (configs: base clamped, top shear 0.1 in 10 steps)
    ubar = torch.as_tensor(m.ubar.ravel(), dtype=torch.float64, device=dev)
    u = torch.zeros(m.n_nodes * 3, dtype=torch.float64, device=dev)
    gm.newton_step(u, ubar, 0.0, 0.0, cg_dtype=torch.float32)  # workspace
    times, newton, cg = [], [], []
    s_prev = 0.0
    for k in range(1, hex_steps + 1):
        s = k / 10
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record()
        st = gm.newton_step(u, ubar, s_prev, s, cg_dtype=torch.float32)
        b.record()
        b.synchronize()
        times.append(a.elapsed_time(b) * 1e-3)
        newton.append(st["newton_iters"])
        cg.append(st["cg_iters"])
        s_prev = s
    return {"workload": "hex128: 128^3 Q1 hexahedra (2,097,152 elements, 2,146,689 nodes), 2x2x2 Gauss, "
                        "per-element mu lognormal(0, 0.5) (seed 0), lambda = 10 mu; base clamped, top sheared",
            "residual_us": t_r * 1e6, "hvp_us": t_h * 1e6,
            "residual_gelem_s": m.n_el / t_r / 1e9, "hvp_gelem_s": m.n_el / t_h / 1e9,
            "pair_gelem_s": m.n_el / (t_r + t_h) / 1e9,
            "roofline": {"bound": "alu", "unit": "TFLOP/s", "flops_per_el": {"residual": HEX_FLOPS_RES,
                                                                             "hvp": HEX_FLOPS_HVP},
                         "achieved": {"residual": tf_r, "hvp": tf_h},
                         "peak_measured": peak_meas, "peak_nominal": nominal,
                         "frac_of_measured": {"residual": tf_r / peak_meas, "hvp": tf_h / peak_meas},
                         "frac_of_nominal": {"residual": tf_r / nominal, "hvp": tf_h / nominal},
                         "peak_how": "measured: fem_fp32_fma_rate (8 independent FMA chains per thread, 8 blocks "
                                     "of 256 per SM, best of 5); nominal: SMs x 128 FP32 lanes x 2 x 2.032 GHz"},
            "l2": "flushed before every call",
            "newton_mixed": {"s_per_load_step": statistics.median(times) if times else None, "s_each": times,
                             "newton_iters": newton, "cg_iters": cg,
                             "what": "mixed precision (FP32 CG with FP64 dots, FP64 residual and energy), block "
                                     "Jacobi, relative residual 1e-8, top shear 0.1 in 10 load steps"}}


def sparse_arm(gm, ut, vt, t_hvp_us, flush_l2, peak):
    """Sparse K by colouring (Algorithm 2) on the benchmark mesh: host
    pattern and colouring, the n_colors seeded HVPs plus decompression, and
    the CSR product K v against the HVP (same FP32 u, v; L2 flushed before
    each timed call)."""
    import torch
    t0 = time.perf_counter()
    nnz, nc = gm.sparse_info()
    t_host = time.perf_counter() - t0
    vals = gm.sparse_assemble(ut)
    y = gm.sparse_spmv(vals, vt)
    h = gm.hvp(ut, vt)
    rel = float(torch.linalg.norm(y - h) / torch.linalg.norm(h))

    def timed(fn, reps):
        ts = []
        for k in range(reps):
            flush_l2(k)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            fn()
            b.record()
            b.synchronize()
            ts.append(a.elapsed_time(b) * 1e3)
        return statistics.median(ts)

    t_asm = timed(lambda: gm.sparse_assemble(ut, out=vals), 5)
    t_spmv = timed(lambda: gm.sparse_spmv(vals, vt, out=y), 20)
    nn = gm.n_nodes
    n_blocks = nnz // 9  # node pairs: one node id each
    spmv_bytes = nnz * 4 + n_blocks * 4 + (nn + 1) * 8 + nn * 8 + 2 * gm.n_dofs * 4
    return {"what": "Algorithm 2: greedy distance-2 column colouring, one seeded HVP per colour, "
                    "decompression into CSR; then y = K v (CSR, FP32)",
            "nnz": nnz, "n_colors": nc, "host_pattern_and_colouring_s": t_host,
            "assemble_ms": t_asm / 1e3, "assemble_in_hvps": t_asm / t_hvp_us,
            "spmv_us": t_spmv, "hvp_us": t_hvp_us, "spmv_vs_hvp_rel_err": rel,
            "spmv_roofline": {"bound": "hbm", "bytes": spmv_bytes, "achieved": spmv_bytes / (t_spmv * 1e-6) / 1e9,
                              "peak": peak, "unit": "GB/s",
                              "frac": spmv_bytes / (t_spmv * 1e-6) / 1e9 / peak,
                              "traffic": traffic_for("tet64_spmv_f32", SPMV_SOURCES)}}


def atomic_arm(gm, ut, vt, t_res_us, t_hvp_us, flush_l2):
    """The scatter-add ablation: residual and HVP with one thread per element
    and float atomics (fem_*_atomic) against the tiled, coloured calls timed
    above (same inputs, L2 flushed before each timed call), and the entries
    that change between two atomic runs."""
    import torch
    r = gm.residual_atomic(ut)
    y = gm.hvp_atomic(ut, vt)

    def timed(fn, reps=20):
        ts = []
        for k in range(reps):
            flush_l2(k)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            fn()
            b.record()
            b.synchronize()
            ts.append(a.elapsed_time(b) * 1e3)
        return statistics.median(ts)

    t_r = timed(lambda: gm.residual_atomic(ut, out=r))
    t_h = timed(lambda: gm.hvp_atomic(ut, vt, out=y))
    y2 = gm.hvp_atomic(ut, vt)
    # K itself: element stiffness scattered with atomics against Algorithm 2
    k1 = gm.sparse_assemble_atomic(ut)
    t_k = timed(lambda: gm.sparse_assemble_atomic(ut, out=k1), 5)
    k2 = gm.sparse_assemble_atomic(ut)
    kc = gm.sparse_assemble(ut)
    t_kc = timed(lambda: gm.sparse_assemble(ut, out=kc), 5)
    return {"what": "one thread per element in mesh order, nodal forces added with float atomicAdd "
                    "(same constitutive code); the tiled kernels add in a fixed order",
            "residual_us": t_r, "hvp_us": t_h, "tiled_residual_us": t_res_us, "tiled_hvp_us": t_hvp_us,
            "slowdown_residual": t_r / t_res_us, "slowdown_hvp": t_h / t_hvp_us,
            "hvp_entries_differing_between_two_runs": int((y2 != y).sum()), "n_dofs": gm.n_dofs,
            "K_assembly_atomic_ms": t_k / 1e3, "K_assembly_algorithm2_ms": t_kc / 1e3,
            "K_entries_differing_between_two_runs": int((k2 != k1).sum()), "K_nnz": k1.numel(),
            "K_atomic_vs_algorithm2_rel": float(torch.linalg.norm(k1 - kc) / torch.linalg.norm(kc))}


NCM_H = 32


def ncm_arm(m, gm, ut, vt, t_res_us, t_hvp_us, flush_l2, dev):
    """The neural constitutive model (psi = [NN(I1, J) - NN(3, 1)] + psi_NH,
    a 2 -> 32 -> 32 -> 1 softplus MLP with synthetic weights) on the
    benchmark mesh: residual and HVP calls (each evaluates the network at
    every element first), and one mixed-precision Newton load step of the
    random-moduli mesh with and without the network."""
    import torch
    from paper_2602_12365_b300 import meshgen as mg
    from paper_2602_12365_b300.fem import Mesh

    def timed(fn, reps=20):
        ts = []
        for k in range(reps):
            flush_l2(k)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            fn()
            b.record()
            b.synchronize()
            ts.append(a.elapsed_time(b) * 1e3)
        return statistics.median(ts)

    p = mg.ncm_params(NCM_H, seed=7, amp=0.2)
    gm.set_ncm(NCM_H, p)
    r, y = torch.empty_like(ut), torch.empty_like(ut)
    gm.residual(ut, out=r)
    t_r = timed(lambda: gm.residual(ut, out=r))
    t_h = timed(lambda: gm.hvp(ut, vt, out=y))
    gm.set_ncm(0)
    mn = mg.workload_tet(m.n, seed=101, random_moduli=101)
    gn = Mesh.from_fixture(mn, precision="mixed")
    ubar = torch.as_tensor(mn.ubar.ravel(), dtype=torch.float64, device=dev)
    out = {}
    for arm, net in (("neo_hookean", False), ("ncm", True)):
        gn.set_ncm(NCM_H, p) if net else gn.set_ncm(0)
        u = torch.zeros(mn.n_nodes * 3, dtype=torch.float64, device=dev)
        gn.newton_step(u, ubar, 0.0, 0.0, cg_dtype=torch.float32)  # workspace
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record()
        st = gn.newton_step(u, ubar, 0.0, 0.05, cg_dtype=torch.float32)
        b.record()
        b.synchronize()
        out[arm] = {"s": a.elapsed_time(b) * 1e-3, "newton_iters": st["newton_iters"], "cg_iters": st["cg_iters"],
                    "status": st["status"]}
    return {"what": f"psi = [NN(I1, J) - NN(3, 1)] + psi_NH, NN 2 -> {NCM_H} -> {NCM_H} -> 1 softplus MLP "
                    "(synthetic weights, seed 7), FP32 kernels; each residual / HVP call evaluates the "
                    "network at every element first (the Newton PCG once per solve)",
            "residual_us": t_r, "hvp_us": t_h, "neo_hookean_residual_us": t_res_us,
            "neo_hookean_hvp_us": t_hvp_us, "newton_first_load_step_mixed": out}


def run_ours(args):
    import torch
    world, rank, local = dist_init(args)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_2602_12365_b300 import fem
    from paper_2602_12365_b300.fem import Mesh

    m, u, v = workload(args.n)
    gm = Mesh.from_fixture(m, precision="mixed")
    info = gm.info()
    ut = torch.as_tensor(u, dtype=torch.float32, device=dev)
    vt = torch.as_tensor(v, dtype=torch.float32, device=dev)
    r = torch.empty_like(ut)
    y = torch.empty_like(ut)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    flush_rd = torch.ones(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def flush_l2(k):
        flush.fill_(float(k))
        return flush_rd.sum()

    def warm_up():  # the same work as a timed step, flush included
        for k in range(max(args.warmup, 3)):
            flush_l2(k)
            gm.residual(ut, out=r)
            gm.hvp(ut, vt, out=y)

    warm_up()
    torch.cuda.synchronize()
    assert gm.sync_status() == 0, "device status flagged during warm-up"

    ev_step = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    with ClockSampler(local) as clk:
        # warm up again right before the timed steps, so that the GPU is busy
        # (clocks up) when they start rather than idle since the sampler began
        warm_up()
        barrier(world)
        torch.cuda.synchronize()
        wall0 = time.perf_counter()
        # Host head start: each step costs the host ~150 us of Python, event
        # and launch overhead, more than the GPU's flush before the step, so
        # the GPU would idle inside the timed intervals.  A clock-bounded
        # delay kernel ahead of the first timed event lets the host queue all
        # steps first; the timed intervals then hold GPU work only.
        torch.cuda._sleep(int(2.0e9 * (0.5e-3 * args.steps + 2e-3)))
        # the step: residual then HVP back to back (the HVP's launch overlaps
        # the residual's tail, as in a caller's stream), events around it
        for k in range(args.steps):
            flush_l2(k)
            ev_step[k][0].record(stream)
            gm.residual(ut, out=r)
            gm.hvp(ut, vt, out=y)
            ev_step[k][2].record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - wall0
        # per-call durations for the roofline: the same K steps again with an
        # event between the calls (which costs the step that overlap)
        torch.cuda._sleep(int(2.0e9 * (0.5e-3 * args.steps + 2e-3)))
        for k in range(args.steps):
            flush_l2(k)
            ev[k][0].record(stream)
            gm.residual(ut, out=r)
            ev[k][1].record(stream)
            gm.hvp(ut, vt, out=y)
            ev[k][2].record(stream)
        torch.cuda.synchronize()
    # warm: the same K steps with L2 not flushed (the step's inputs and the
    # element stream partly L2-resident from the previous step)
    ev_w = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    torch.cuda._sleep(int(2.0e9 * (0.5e-3 * args.steps + 2e-3)))
    for k in range(args.steps):
        ev_w[k][0].record(stream)
        gm.residual(ut, out=r)
        ev_w[k][1].record(stream)
        gm.hvp(ut, vt, out=y)
        ev_w[k][2].record(stream)
    torch.cuda.synchronize()
    warm = {"residual_us": statistics.median(e[0].elapsed_time(e[1]) for e in ev_w) * 1e3,
            "hvp_us": statistics.median(e[1].elapsed_time(e[2]) for e in ev_w) * 1e3,
            "l2": "not flushed (warm)"}
    warm["pair_gelem_s"] = m.n_el / ((warm["residual_us"] + warm["hvp_us"]) * 1e-6) / 1e9
    barrier(world)
    t_step = max_over_ranks(sum(e[0].elapsed_time(e[2]) for e in ev_step) / args.steps, world, dev)
    t_res = sum(e[0].elapsed_time(e[1]) for e in ev) / args.steps  # ms
    t_hvp = sum(e[1].elapsed_time(e[2]) for e in ev) / args.steps
    t_res = max_over_ranks(t_res, world, dev)
    t_hvp = max_over_ranks(t_hvp, world, dev)
    flags = gm.sync_status()

    # end to end through the C ABI with host buffers: every step copies its
    # inputs u, v host -> device and its results r, y device -> host.  The
    # steps run as a pipeline, as in a serving loop: two sets of device
    # buffers, the inputs of step k + 1 go up (copy stream) while step k
    # computes, and its results come down (second copy stream) while step
    # k + 1 computes; a buffer set is reused only after its results have
    # reached the host.  Instead of an L2 flush (whose 512 MB of HBM traffic
    # would compete with the copy engines inside the region), consecutive
    # steps run on two device copies of the mesh, the same plan and data:
    # their working sets (records, slots, vectors: ~107 MB each on tet64)
    # add up to more than the 126 MB L2, so a step finds little of its mesh
    # still cached.  The K steps are timed as one region (host head start as
    # above) and ms_per_step = region / K.
    e2e = None
    if not args.no_e2e:
        gms = (gm, Mesh.from_fixture(m, precision="mixed"))
        uh = torch.as_tensor(u, dtype=torch.float32).pin_memory()
        vh = torch.as_tensor(v, dtype=torch.float32).pin_memory()
        hb = [(torch.empty_like(uh).pin_memory(), torch.empty_like(uh).pin_memory()) for _ in range(2)]
        db = [tuple(torch.empty_like(ut) for _ in range(4)) for _ in range(2)]  # u, v, r, y
        s_in, s_out = torch.cuda.Stream(), torch.cuda.Stream()
        ev_in = [torch.cuda.Event() for _ in range(2)]
        ev_done = [torch.cuda.Event() for _ in range(2)]
        ev_out = [torch.cuda.Event() for _ in range(2)]

        def e2e_steps(K, first):
            for k in range(K):
                j = k & 1
                ud, vd, rd, yd = db[j]
                rh, yh = hb[j]
                if k >= 2 or not first:
                    s_in.wait_event(ev_out[j])  # set j's previous results are on the host
                with torch.cuda.stream(s_in):
                    ud.copy_(uh, non_blocking=True)
                    vd.copy_(vh, non_blocking=True)
                    ev_in[j].record(s_in)
                stream.wait_event(ev_in[j])
                gms[j].residual(ud, out=rd, stream=stream)
                gms[j].hvp(ud, vd, out=yd, stream=stream)
                ev_done[j].record(stream)
                s_out.wait_event(ev_done[j])
                with torch.cuda.stream(s_out):
                    rh.copy_(rd, non_blocking=True)
                    yh.copy_(yd, non_blocking=True)
                    ev_out[j].record(s_out)
            for j in range(min(K, 2)):
                stream.wait_event(ev_out[j])  # the region ends when the last results are on the host

        e2e_steps(3, True)
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        torch.cuda._sleep(int(2.0e9 * (0.5e-3 * args.steps + 2e-3)))  # host head start
        a.record(stream)
        e2e_steps(args.steps, False)
        b.record(stream)
        b.synchronize()
        t_e2e = max_over_ranks(a.elapsed_time(b) / args.steps, world, dev)
        assert torch.equal(hb[(args.steps - 1) & 1][1].to(dev), y), "end-to-end result differs from the device run"
        nb = ut.numel() * 4
        e2e = {"value": world * m.n_el / (t_e2e * 1e-3) / 1e9, "unit": "GElem/s",
               "h2d_bytes_per_step": 2 * nb, "d2h_bytes_per_step": 2 * nb,
               "ms_per_step": t_e2e,
               "how": "K steps pipelined (two device buffer sets; H2D of step k+1 and D2H of step k overlap "
                      "compute), each step copying its own inputs and results; consecutive steps on two device "
                      "copies of the mesh, whose working sets together exceed L2 (no flush kernel in the region); "
                      "timed as one region / K"}

    peak, peak_kind = measured_peaks()
    dominant = "hvp" if t_hvp >= t_res else "residual"
    t_dom = t_hvp if dominant == "hvp" else t_res
    b_dom = (B_HVP_PER_EL if dominant == "hvp" else B_RES_PER_EL) * m.n_el
    achieved = b_dom / (t_dom * 1e-3) / 1e9
    tr = traffic_for(f"{WORKLOAD}_{dominant}_f32")
    value = world * m.n_el / (t_step * 1e-3) / 1e9
    launches = fem.KERNELS_PER_CALL
    line = {
        "metric": "residual+HVP GElem/s", "value": value, "unit": "GElem/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": config_dict(m, "1 residual + 1 HVP (FP32 element kernels, FP64 reductions)",
                              {"tiles": info["n_tiles"], "rounds": info["n_rounds"],
                               "round_fill": round(info["round_fill"], 4)}),
        "residual_us": t_res * 1e3, "hvp_us": t_hvp * 1e3,
        "residual_gelem_s": m.n_el / (t_res * 1e-3) / 1e9,
        "hvp_gelem_s": m.n_el / (t_hvp * 1e-3) / 1e9,
        "pair_hbm_frac": (B_RES_PER_EL + B_HVP_PER_EL) * m.n_el / ((t_res + t_hvp) * 1e-3) / 1e9 / peak,
        "roofline": {"bound": "hbm", "kernel": f"fem_{dominant} (tet4, f32)",
                     "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "peak_kind": f"{peak_kind} HBM copy bandwidth",
                     "bytes_per_el": B_HVP_PER_EL if dominant == "hvp" else B_RES_PER_EL,
                     "timed": "whole C-ABI call (all its kernels), CUDA events on its stream, in a second "
                              "pass of the K steps with an event between the two calls (the step time is taken "
                              "without it: it stops the HVP's launch from overlapping the residual's tail)",
                     "traffic": tr},
        "gpu_launches": (launches["residual"] + launches["hvp"]) * args.steps,
        "device_flags": flags,
        "wall_s_timed_region": wall,
    }
    line["clocks"] = clk.summary()
    if e2e:
        line["e2e"] = e2e
    line["warm"] = warm
    if not args.no_ncm and rank == 0:
        line["ncm"] = ncm_arm(m, gm, ut, vt, t_res * 1e3, t_hvp * 1e3, flush_l2, dev)
    if not args.no_sparse and rank == 0:  # per-GPU measurements, reported by rank 0
        line["atomic_ablation"] = atomic_arm(gm, ut, vt, t_res * 1e3, t_hvp * 1e3, flush_l2)
        line["sparse"] = sparse_arm(gm, ut, vt, t_hvp * 1e3, flush_l2, peak)
    if not args.no_hex and rank == 0:
        line["hex128"] = hex_arm(dev, flush_l2, min(args.steps, 20), args.hex_steps)
    if args.newton_steps > 0 and rank == 0:  # a per-GPU measurement, reported by rank 0
        seeds = [int(x) for x in args.newton_seeds.split(",") if x.strip()]
        line["newton"] = newton_arms(args.n, args.newton_steps, seeds, dev)
    # the FP32 path's results at the benchmark's FP64 state (u, v rounded to
    # FP32 on the way in) against the FP64 path on the same GPU (the CPU leg
    # below adds the oracle's own figures)
    u64 = torch.as_tensor(u, dtype=torch.float64, device=dev)
    v64 = torch.as_tensor(v, dtype=torch.float64, device=dev)
    gm.residual(ut, out=r)  # the arms above reuse r and y
    gm.hvp(ut, vt, out=y)
    r64, y64 = gm.residual(u64), gm.hvp(u64, v64)
    e32, e64 = gm.energy(ut), gm.energy(u64)
    rel = lambda a, b: float(torch.linalg.norm(a.double() - b) / torch.linalg.norm(b))  # noqa: E731
    precision = {"state": "the benchmark's FP64 (u, v); FP32 calls receive them rounded to FP32",
                 "residual_f32_vs_f64_gpu": rel(r, r64), "hvp_f32_vs_f64_gpu": rel(y, y64),
                 "energy_f32_vs_f64_gpu": abs(float(e32[0]) - float(e64[0])) / abs(float(e64[0]))}
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_leg(m, u, v, r.double().cpu().numpy(), y.double().cpu().numpy(), r64.cpu().numpy(),
                      y64.cpu().numpy(), float(e32[0]), float(e64[0]))
        line["cpu_baseline"] = cpu.pop("cpu_baseline")
        precision.update(cpu)
    line["precision_error"] = precision
    if rank == 0:
        print(json.dumps(line))


def cpu_info():
    model = None
    try:
        with open("/proc/cpuinfo") as f:
            for ln in f:
                if ln.startswith("model name"):
                    model = ln.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    return model, os.cpu_count()


def cpu_leg(m, u, v, r32, y32, r64, y64, e32, e64):
    """The FP64 CPU oracle (single thread, pinned to one core) on the whole
    workload: one residual + one HVP at the FP64 state, timed, and the same at
    the FP32-rounded state; their outputs give the FP32 and FP64 GPU paths'
    errors against the oracle (precision pattern (1))."""
    import numpy as np
    import oracle
    om = oracle.OracleMesh.from_mesh(m)
    model, ncpu = cpu_info()
    try:
        old = os.sched_getaffinity(0)
        core = min(old)
        os.sched_setaffinity(0, {core})
        pinned = f"core {core} (sched_setaffinity, as taskset -c {core})"
    except (AttributeError, OSError):
        old, pinned = None, "not pinned"
    try:
        ts = []
        t0 = time.perf_counter()
        ro = om.residual(u)
        yo = om.hvp(u, v)
        ts.append(time.perf_counter() - t0)
        u32 = u.astype(np.float32).astype(np.float64)
        v32 = v.astype(np.float32).astype(np.float64)
        t0 = time.perf_counter()
        ro32 = om.residual(u32)
        yo32 = om.hvp(u32, v32)
        ts.append(time.perf_counter() - t0)
        psi = om.energy(u)
        psi32 = om.energy(u32)
    finally:
        if old is not None:
            os.sched_setaffinity(0, old)
    t = min(ts)
    rel = lambda a, b: float(np.linalg.norm(a - b) / np.linalg.norm(b))  # noqa: E731
    out = {"cpu_baseline": {"value": m.n_el / t / 1e9, "unit": "GElem/s", "cores": 1, "kind": "oracle",
                            "sample": f"whole workload, one residual + one HVP, best of 2 ({t:.2f} s each; "
                                      "at the FP64 state and at its FP32 rounding)",
                            "cpu_model": model, "nproc": ncpu, "pinned": pinned},
           "residual_f32_vs_oracle": rel(r32, ro), "hvp_f32_vs_oracle": rel(y32, yo),
           "energy_f32_vs_oracle": abs(e32 - psi) / abs(psi),
           "residual_f32_vs_oracle_at_f32_inputs": rel(r32, ro32), "hvp_f32_vs_oracle_at_f32_inputs": rel(y32, yo32),
           "energy_f32_vs_oracle_at_f32_inputs": abs(e32 - psi32) / abs(psi32),
           "input_rounding_alone": {"residual": rel(ro32, ro), "hvp": rel(yo32, yo),
                                    "what": "oracle at the FP32-rounded state against the oracle at the FP64 state"},
           "residual_f64_vs_oracle": rel(r64, ro), "hvp_f64_vs_oracle": rel(y64, yo),
           "energy_f64_vs_oracle": abs(e64 - psi) / abs(psi)}
    return out


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
