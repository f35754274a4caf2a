#!/usr/bin/env python
"""Benchmark of the RSOT dual + gradient hot path on one GB300 (or N replicas).

Workload (default): unit cube, 32^3 hexes x 6 tets x 4-point rule = 786,432
quadrature points, 65,536 targets from a 4-component mixture, nu ~ U(0.5,1.5)
normalised, eps = 1e-3, dense evaluation (5.154e10 pairs per step).  A step is
one complete dual + gradient evaluation: target prep, pass 1 (log-sum-exp),
combine, pass 2 (gradient), final reductions.

Metric: G pairs/s (pairs = nq * n per dense evaluation), inputs resident in
HBM (`value`), and through the C ABI with host buffers (`e2e`).  L2 is flushed
(256 MiB write) between timed steps; per-step time is taken with CUDA events
on the library's stream, the flush outside them.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

# ex2.approx.f32 results per clock per SM on GB300.  Blackwell-era throughput
# tables give 16 per SM per clock for the special-function unit; GB300 doubles
# it: the probe kernel of librsot (rsot_probe_ex2_rate) measures 9.99e12 ex2/s
# on 152 SMs at ~2.05 GHz, i.e. 32 per SM per clock.  The roofline uses 32.
SFU_EX2_PER_CLK_PER_SM = 32
# FP32 lane-operations (add, mul, fma each one; packed f32x2 instructions two)
# per clock per SM: 4 sub-partitions x 32 lanes
FP32_LANE_OPS_PER_CLK_PER_SM = 128
# FP32 lane-operations per pair of the compensated passes, counted from their
# source: double-float exponent 3 x 12 + 3, shift TwoSum 6, Kahan 4, tail 2-3
COMP_FP32_OPS_PER_PAIR = {"lse_df": 51, "grad_df": 52}
# FP64-pipe operations per pair of the two dense FP64 passes, counted from
# their source (d = 2 / 3): the squared distance (d subtractions, d fused
# multiply-adds), the exponent (one fma; pass 2 one more add), the library's own
# exponential (two range compares, multiply, round, conversion, 2 fma reduction,
# 5 fma + 1 multiply polynomial, 1 fma + 1 add table, 1 multiply scaling: 16),
# then pass 1's compare-and-update (2: the shift subtraction and one of the two
# update forms, plus the compare) and pass 2's accumulation (1):
# pass 1 = 2d + 20, pass 2 = 2d + 19
FP64_OPS_PER_PAIR = {2: 47, 3: 51}
L2_FLUSH_BYTES = 256 << 20


def max_over_ranks(x: float, world: int, device=None) -> float:
    """The maximum of a per-rank time over the ranks of the run (an all-reduce
    on the default process group; the value itself on one rank)."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as tdist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_step: float, steps: int, world: int, seconds: float) -> float:
    """Units per second of the whole job in billions: every rank processes
    units_per_step in each of its steps (weak scaling), timed by the slowest."""
    return units_per_step * steps * world / seconds / 1e9


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--mesh", type=int, default=32, help="hexes per side (32 -> 786,432 points)")
    ap.add_argument("--targets", type=int, default=65536)
    ap.add_argument("--eps", type=float, default=1e-3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-trunc", action="store_true")
    ap.add_argument("--no-fp32-compare", action="store_true")
    ap.add_argument("--no-compensated", action="store_true")
    ap.add_argument("--pair-kernel", choices=["auto", "tensor", "fp32"], default="auto",
                    help="dense workload: pair kernel of the timed evaluations")
    ap.add_argument("--tail", type=float, default=0.0,
                    help="multilevel: truncation tail of every evaluation (0: dense)")
    ap.add_argument("--workload", choices=["dense", "solve", "batch", "multilevel", "warmstart",
                                           "maps", "barycenter", "mlp", "cutoffs"],
                    default="dense",
                    help="dense: dual+grad throughput (default); the others time solves")
    ap.add_argument("--problems", type=int, default=32, help="batch: problems (seeds 1000..)")
    ap.add_argument("--plain-problems", type=int, default=8,
                    help="batch: problems also solved by the plain FP64 path")
    ap.add_argument("--train-seeds", type=int, default=10000)
    ap.add_argument("--eval-seeds", type=int, default=512)
    ap.add_argument("--epochs", type=int, default=8)
    ap.add_argument("--mlp-rows", type=int, default=65536, help="mlp: rows per gradients call")
    ap.add_argument("--no-solve", action="store_true",
                    help="dense workload: skip the solve-time object (cube solve and the "
                         "warm-started vs plain FP64 comparison)")
    ap.add_argument("--compare-problems", type=int, default=16,
                    help="dense workload: held-out warm-start problems solved by both arms")
    ap.add_argument("--no-oracle-check", action="store_true",
                    help="dense workload: skip the oracle gradients at the solves' results")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class Clocks:
    """nvidia-smi sampling during the timed region (recipe's clocks line)."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "25"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
            # the timed region starts once the sampler writes (a short region
            # still gets several samples); at most 2 s
            t0 = time.perf_counter()
            while time.perf_counter() - t0 < 2.0 and self.proc.poll() is None:
                if os.path.getsize(self.path) > 0:
                    break
                time.sleep(0.01)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [t.strip() for t in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.remove(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


def kernel_source_hash():
    """Hash of the sources the dense kernels are built from (their file and the
    shared device headers)."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2507_23602_gb300", "csrc")
    for f in sorted(os.listdir(csrc)):
        if f == "rsot_dense.cu" or f.endswith(".cuh"):
            h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:16]


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def traffic_for(kernel, workload):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on
    the current kernel sources (else None)."""
    try:
        t = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
    except Exception:
        return None
    e = t.get(workload, {}).get(kernel)
    if not e or e.get("source_hash") != kernel_source_hash():
        return None
    return e.get("dram_bytes_per_launch")


def cpu_baseline(p, psi, target_seconds=12.0):
    """The FP64 oracle, as it stands, on a bounded sample of the workload:
    the first S quadrature points against all targets, one dense evaluation."""
    import oracle
    cores = oracle.threads_used()
    s0 = min(p.nq, max(256, cores * 64))
    t = time.perf_counter()
    oracle.dual_grad(p.x[:s0], p.mass[:s0], p.y, p.nu, psi, p.eps)
    dt0 = time.perf_counter() - t
    s = int(min(p.nq, max(s0, s0 * target_seconds / max(dt0, 1e-3))))
    t = time.perf_counter()
    oracle.dual_grad(p.x[:s], p.mass[:s], p.y, p.nu, psi, p.eps)
    dt = time.perf_counter() - t
    pairs = s * p.n
    # the same oracle on one thread, on a sample of about 5 s
    s1 = max(16, min(p.nq, int(s * 5.0 / max(dt * cores, 1e-3))))
    t = time.perf_counter()
    oracle.dual_grad(p.x[:s1], p.mass[:s1], p.y, p.nu, psi, p.eps, threads=1)
    dt1 = time.perf_counter() - t
    return {"value": pairs / dt / 1e9, "unit": "G pairs/s", "cores": cores, "kind": "oracle",
            "sample": f"dense FP64 evaluation of quadrature points 0..{s - 1} of {p.nq} against all "
                      f"{p.n} targets ({pairs:.3e} pairs, {dt:.1f} s)",
            "single_thread": {"value": s1 * p.n / dt1 / 1e9, "unit": "G pairs/s", "cores": 1,
                              "sample": f"points 0..{s1 - 1} ({s1 * p.n:.3e} pairs, {dt1:.1f} s)"}}


def run_reference(args, p, psi, workload):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle
    cores = oracle.threads_used()
    # calibrate one step to ~ (a few minutes / (steps + warmup))
    budget = 150.0 / max(1, args.steps + args.warmup)
    s0 = min(p.nq, max(256, cores * 64))
    t = time.perf_counter()
    oracle.dual_grad(p.x[:s0], p.mass[:s0], p.y, p.nu, psi, p.eps)
    dt0 = time.perf_counter() - t
    s = int(min(p.nq, max(s0, s0 * budget / max(dt0, 1e-3))))
    for _ in range(args.warmup):
        oracle.dual_grad(p.x[:s], p.mass[:s], p.y, p.nu, psi, p.eps)
    times = []
    for _ in range(args.steps):
        t = time.perf_counter()
        oracle.dual_grad(p.x[:s], p.mass[:s], p.y, p.nu, psi, p.eps)
        times.append(time.perf_counter() - t)
    ms = 1e3 * sum(times) / len(times)
    val = s * p.n / (ms * 1e-3) / 1e9
    sample = f"each step: dense FP64 oracle evaluation of points 0..{s - 1} of {p.nq} x {p.n} targets"
    print(json.dumps({
        "impl": "reference", "metric": "dual+grad G pairs/s (dense)", "value": val,
        "unit": "G pairs/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload, "sample_points": s},
        "cpu_baseline": {"value": val, "unit": "G pairs/s", "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": val, "unit": "G pairs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def solve_line(metric, value, unit, workload, extra, args, higher=False):
    out = {"metric": metric, "value": value, "unit": unit, "n_gpus": 1, "steps": 1,
           "warmup": 0, "ms_per_step": value * 1e3 if unit == "s" else None,
           "higher_is_better": higher, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
           "data": "synthetic", "config": {"workload": workload}}
    out.update(extra)
    print(json.dumps(out))


def run_solve_workloads(args):
    """Solve-time metrics (time to ||grad J||_1 <= tol): mixed with the
    refinement on compensated evaluations against plain FP64, on the GPU."""
    import numpy as np
    import torch
    import rsot_inputs as ri
    import paper_2507_23602_gb300 as rs
    torch.cuda.set_device(0)
    if args.workload == "solve":
        res = {}
        p = ri.small_2d()
        P = rs.Problem(p.x, p.mass, p.y, p.nu)
        for name, prec in (("fp64", rs.FP64), ("mixed", rs.MIXED)):
            t = time.perf_counter()
            _, st = P.solve(eps=p.eps, tol_l1=1e-8, precision=prec, raise_on_error=False)
            res["small_2d_" + name] = {"seconds": time.perf_counter() - t, "iters": st.iters,
                                       "evals": st.evals, "grad_l1": st.grad_l1, "status": st.status}
        P.close()
        q = ri.cube_3d(mesh_n=args.mesh, n_targets=args.targets, eps=args.eps)
        Q = rs.Problem(q.x, q.mass, q.y, q.nu)
        # dense, and truncated at tail 1e-12 (psi-aware cutoffs; the certified stop
        # holds for the untruncated J)
        for name, tail in (("cube_mixed", 0.0), ("cube_mixed_tail", 1e-12)):
            t = time.perf_counter()
            _, st = Q.solve(eps=q.eps, eps_start=0.1, eps_factor=0.5, tol_l1=1e-6, precision=rs.MIXED,
                            raise_on_error=False, max_iter=20000, tail=tail)
            res[name] = {"seconds": time.perf_counter() - t, "iters": st.iters, "evals": st.evals,
                         "grad_l1": st.grad_l1, "status": st.status, "tail": tail}
        mixed_s = res["cube_mixed"]["seconds"]
        Q.close()
        solve_line("solve time to ||grad||_1<=1e-6 (cube, eps 0.1->1e-3, mixed + compensated correction)",
                   mixed_s, "s", f"cube-{q.nq}x{q.n}-solve", {"results": res}, args)
        return
    if args.workload == "batch":
        seeds = list(range(1000, 1000 + args.problems))
        probs = [ri.batch_problem(s) for s in seeds]
        eps = np.array([p.eps for p in probs])
        B = rs.Batch([(p.x, p.mass, p.y, p.nu) for p in probs])
        psi0 = np.zeros(B.total)
        choice = B.tune(psi0, eps)
        psi, st = B.solve(eps, eps_start=0.1, eps_factor=0.5, tol_l1=1e-6, precision=rs.MIXED,
                          raise_on_error=False)
        B.close()
        k = min(args.plain_problems, len(probs))
        sub = probs[:k]
        B2 = rs.Batch([(p.x, p.mass, p.y, p.nu) for p in sub])
        _, st_m = B2.solve(eps[:k], eps_start=0.1, eps_factor=0.5, tol_l1=1e-6, precision=rs.MIXED,
                           raise_on_error=False)
        _, st_p = B2.solve(eps[:k], eps_start=0.1, eps_factor=0.5, tol_l1=1e-6, precision=rs.FP64,
                           raise_on_error=False)
        B2.close()
        pairs = sum(p.nq * p.n for p in probs)
        clean = lambda s: {k2: (v.tolist() if hasattr(v, "tolist") else v) for k2, v in s.items()
                           if k2 not in ("grad_l1", "statuses")}
        solve_line("batched solve time to ||grad||_1<=1e-6 (mixed + compensated correction)",
                   st["seconds"], "s", f"batch-{len(probs)}-problems",
                   {"pairs_per_round_all": pairs, "item_exp": choice, "batch": clean(st),
                    "subset_problems": k, "subset_mixed_batched": clean(st_m),
                    "subset_plain_fp64": clean(st_p),
                    "subset_speedup": st_p["seconds"] / max(st_m["seconds"], 1e-9)}, args)
        return
    if args.workload == "multilevel":
        d = 3
        mix = ri.random_mixture(3, 5, 3)
        ns = [9, 18, 35, 70] if args.mesh >= 32 else [4, 8, 16]
        src = []
        for n in ns:
            v, c = ri.unit_cube_tet_mesh(n)
            src.append(ri.source_measure(v, c, ri.tet_rule_deg2(), ri.mixture_density(mix, v)))
        ysamp = ri.sample_mixture(ri.random_mixture(3, 4, 6), 1 << 20, 6)
        wsamp = np.full(1 << 20, 1.0 / (1 << 20))
        t = time.perf_counter()
        levels = []
        for k in (1 << 12, 1 << 14, 1 << 16):
            C, W, _ = rs.kmeans(ysamp, wsamp, k, iters=10, seed=6)
            keep = W > 0
            levels.append((C[keep], W[keep] / W[keep].sum()))
        t_km = time.perf_counter() - t
        L = max(len(src), len(levels)) - 1
        eps_levels = [args.eps * 2 ** (L - l) for l in range(L + 1)]
        psi, st = rs.multilevel_solve(src, levels, eps_levels, tol_l1=1e-6, eps_start=0.1,
                                      eps_factor=0.5, precision=rs.MIXED, raise_on_error=False,
                                      tail=args.tail)
        solve_line("multilevel solve time to ||grad||_1<=1e-6 (combined source/target, Sec. 5.3)",
                   st["total_seconds"], "s",
                   f"multilevel-{src[-1][0].shape[0]}pts-{levels[-1][0].shape[0]}tgt",
                   {"kmeans_seconds": t_km, "stats": st, "tail": args.tail,
                    "levels_points": [s[0].shape[0] for s in src],
                    "levels_targets": [t2[0].shape[0] for t2 in levels]}, args)
        return
    if args.workload == "maps":
        # transport maps (Sec. 6.3) and conditional centroids (Eq. barycenter_fixed_point)
        p = ri.cube_3d(mesh_n=args.mesh, n_targets=args.targets, eps=args.eps)
        psi = 0.005 * np.random.default_rng(2024).standard_normal(p.n)
        P = rs.Problem(p.x, p.mass, p.y, p.nu)
        for _ in range(max(1, args.warmup)):
            P.transport_maps(psi, p.eps)
            P.centroids(psi, p.eps)
        P.kernel_timing(True)
        for _ in range(args.steps):
            P.transport_maps(psi, p.eps)
            P.centroids(psi, p.eps)
        kt = {k: v[0] / v[1] for k, v in P.kernel_times().items()}
        P.kernel_timing(False)
        P.close()
        pairs = p.nq * p.n
        out = {"metric": "transport maps G pairs/s (T_bary and modal map in one pass)",
               "value": pairs / (kt["maps"] * 1e-3) / 1e9, "unit": "G pairs/s", "n_gpus": 1,
               "steps": args.steps, "warmup": args.warmup, "ms_per_step": kt["maps"],
               "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
               "data": "synthetic", "config": {"workload": f"cube-{p.nq}x{p.n}-maps-eps{args.eps:g}"},
               "centroids": {"value": pairs / (kt["centroids"] * 1e-3) / 1e9, "unit": "G pairs/s",
                             "ms": kt["centroids"]},
               "per_kernel_ms": kt}
        print(json.dumps(out))
        return
    if args.workload == "barycenter":
        # damped Lloyd barycenter (Sec. 6.2) of three 3-D mixture sources on 16^3 tet meshes
        v, c = ri.unit_cube_tet_mesh(16)
        srcs = []
        for s in range(3):
            mix = ri.random_mixture(3, 3, 40 + s)
            srcs.append(ri.source_measure(v, c, ri.tet_rule_deg2(), ri.mixture_density(mix, v)))
        n = 4096
        y0 = np.random.default_rng(43).uniform(0.25, 0.75, (n, 3))
        nu = np.full(n, 1.0 / n)
        t = time.perf_counter()
        y, st = rs.barycenter(srcs, np.full(3, 1.0 / 3), y0, nu, theta=0.5, max_iter=30,
                              tol_rms=1e-4, eps=2e-3, eps_start=0.1, tol_l1=1e-6,
                              raise_on_error=False)
        wall = time.perf_counter() - t
        solve_line("barycenter wall time (damped Lloyd, 3 sources x 98,304 points, 4,096 support points)",
                   wall, "s", "barycenter-3x98304-4096-eps0.002",
                   {"stats": st, "seconds_per_iteration": wall / max(1, st["iterations"])}, args)
        return
    if args.workload == "mlp":
        # the warm-start network's training step (forward, back-propagation, weight
        # gradients) on device-resident rows, with each GEMM kernel; value: GEMM
        # FLOP/s of the whole gradients call (host copy of the gradient included)
        rows, in_dim, w = args.mlp_rows, 18, 256
        in_pad = 32
        flops = 2.0 * rows * (2 * in_pad * w + 6 * w * w)
        rng = np.random.default_rng(0)
        x = torch.tensor(rng.normal(0, 1, (rows, in_dim)).astype(np.float32), device="cuda")
        yv = torch.tensor(rng.normal(0, 1, rows).astype(np.float32), device="cuda")
        res = {}
        for name, kind in (("tcgen05", rs.GEMM_TCGEN05), ("tcgen05_cpasync", rs.GEMM_TCGEN05_CPASYNC),
                           ("mma_sync", rs.GEMM_MMA_SYNC)):
            net = rs.MLP(in_dim, w, seed=1)
            net.set_gemm_kernel(kind)
            for _ in range(max(3, args.warmup)):
                net.gradients(x, yv)
            a = torch.cuda.Event(enable_timing=True)
            b_ = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            a.record()
            for _ in range(args.steps):
                net.gradients(x, yv)
            b_.record()
            torch.cuda.synchronize()
            ms = a.elapsed_time(b_) / args.steps
            res[name] = {"ms_per_step": ms, "tflops": flops / (ms * 1e-3) / 1e12}
            if name == "tcgen05":
                # the training step itself: gradients (no host copy), Adam, BF16 weights
                for _ in range(max(3, args.warmup)):
                    net.train_step(x, yv, 1e-4)
                torch.cuda.synchronize()
                a.record()
                for _ in range(args.steps):
                    net.train_step(x, yv, 1e-4)
                b_.record()
                torch.cuda.synchronize()
                ms_t = a.elapsed_time(b_) / args.steps
                res["train_step"] = {"ms_per_step": ms_t, "tflops": flops / (ms_t * 1e-3) / 1e12,
                                     "note": "gradients without the host copy, Adam on the FP32 "
                                             "master weights, BF16 weight refresh"}
            net.close()
        peak = measured_peaks().get("bf16_tflops")
        out = {"metric": "MLP training step TFLOP/s (GEMM FLOPs per gradients call, tcgen05 GEMMs, TMA operands)",
               "value": res["tcgen05"]["tflops"], "unit": "TFLOP/s", "n_gpus": 1, "steps": args.steps,
               "warmup": max(3, args.warmup), "ms_per_step": res["tcgen05"]["ms_per_step"],
               "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16",
               "data": "synthetic",
               "config": {"workload": f"mlp-{in_dim}x{w}x3-rows{rows}", "flops_per_step": flops},
               "tcgen05_cpasync": res["tcgen05_cpasync"], "mma_sync": res["mma_sync"],
               "train_step": res["train_step"],
               "roofline": {"bound": "tensor", "unit": "TFLOP/s", "achieved": res["tcgen05"]["tflops"],
                            "peak": peak, "frac": (res["tcgen05"]["tflops"] / peak) if peak else None,
                            "note": "whole call (activation writes, column sums, host copy of the "
                                    "gradient included), not the GEMM kernels alone"}}
        print(json.dumps(out))
        return
    if args.workload == "cutoffs":
        # the paper's truncation strategies (Sec. 4.1, Sec. 6 truncation table) on the
        # cube: mixed L-BFGS solves to ||g||_1 <= 1e-5 (the mixed floor; no
        # refinement, so the solve runs on the truncated functional throughout),
        # then E_rel = |J~(psi) - J_none| / |J_none| from FP64 evaluations of the
        # truncated functional at each result (its cutoff recomputed there) against
        # the dense FP64 functional at the untruncated solve's result
        import math as _m
        q = ri.cube_3d(mesh_n=args.mesh, n_targets=args.targets, eps=args.eps)
        Q = rs.Problem(q.x, q.mass, q.y, q.nu)
        modes = [("none", {}), ("psi-aware tail", {"tail": 1e-12}),
                 ("pointwise", {"delta_pw": 1e-12}), ("pointwise", {"delta_pw": 1e-10}),
                 ("pointwise", {"delta_pw": 1e-7}),
                 ("integral", {"tau_int": 1e-6}), ("integral", {"tau_int": 1e-5}),
                 ("integral", {"tau_int": 1e-4}),
                 ("geometric", {"tau_geom": 1e-6}), ("geometric", {"tau_geom": 1e-5}),
                 ("geometric", {"tau_geom": 1e-4})]
        out = {}
        for eps_f in (1e-2, 1e-3):
            rows, J_none = [], None
            for name, kw in modes:
                t = time.perf_counter()
                psi_m, st = Q.solve(eps=eps_f, eps_start=0.1, eps_factor=0.5, tol_l1=1e-5,
                                    precision=rs.MIXED, refine_fp64=False, max_iter=5000,
                                    raise_on_error=False, **kw)
                wall = time.perf_counter() - t
                Jd, _, _ = Q.eval(psi_m, eps_f, 0.0, rs.FP64)
                if name == "none":
                    Jt, J_none = Jd, Jd
                elif name == "psi-aware tail":
                    Jt, _, _ = Q.eval_tail(psi_m, eps_f, kw["tail"], rs.FP64)
                else:
                    if name == "pointwise":
                        C = Q.truncation_cutoff(psi_m, eps_f, rs.CUTOFF_POINTWISE, kw["delta_pw"])
                    elif name == "integral":
                        lnD = Q.log_integrated_D()          # of the dense FP64 evaluation above
                        C = Q.truncation_cutoff(psi_m, eps_f, rs.CUTOFF_INTEGRAL, kw["tau_int"], J=Jd, lnD=lnD)
                    else:
                        C = Q.truncation_cutoff(psi_m, eps_f, rs.CUTOFF_GEOMETRIC, kw["tau_geom"], J=Jd)
                    Jt, _, _ = Q.eval(psi_m, eps_f, _m.sqrt(2.0 * C) if C > 0 else 1e-150, rs.FP64,
                                      allow_empty=True)
                param = next(iter(kw.values()), None)
                rows.append({"strategy": name, "param": param, "seconds": wall, "iters": st.iters,
                             "evals": st.evals, "converged": st.status == 0, "status": st.status,
                             "grad_l1": st.grad_l1,
                             "kept_fraction": st.pairs / max(1, st.evals * q.nq * q.n),
                             "J_trunc_fp64": Jt, "J_dense_fp64": Jd,
                             "E_rel": abs(Jt - J_none) / abs(J_none)})
                sys.stderr.write(f"[bench] eps {eps_f:g} {name} {param}: {wall:.2f} s, "
                                 f"{st.iters} it, kept {rows[-1]['kept_fraction']:.3f}, "
                                 f"E_rel {rows[-1]['E_rel']:.2e}\n")
            out[f"eps_{eps_f:g}"] = rows
        Q.close()
        solve_line("solve time by truncation strategy (cube, mixed to ||g||_1 <= 1e-5)",
                   out["eps_0.001"][0]["seconds"], "s", f"cube-{q.nq}x{q.n}-cutoffs",
                   {"results": out,
                    "note": "eps 1e-2 from eps_start 0.1 (x0.5 stages), eps 1e-3 likewise; E_rel "
                            "as the paper's truncation table: the truncated functional at the "
                            "strategy's result against the untruncated one at its own result, "
                            "both FP64"}, args)
        return
    if args.workload == "warmstart":
        from paper_2507_23602_gb300 import warmstart as ws
        X, Y, t_gen = ws.generate(list(range(10000, 10000 + args.train_seeds)))
        net, hist, t_train = ws.train(X, Y, epochs=args.epochs)
        res = ws.evaluate(net, list(range(20000, 20000 + args.eval_seeds)))
        solve_line("warm-started solve time to ||grad||_1<=1e-6 (held-out problems)",
                   res["warm_seconds"], "s", f"warmstart-{args.eval_seeds}-heldout",
                   {"plain_seconds": res["plain_seconds"], "results": res,
                    "train_samples": int(X.shape[0]), "gen_seconds": t_gen,
                    "train_seconds": t_train, "loss_history": hist,
                    "speedup": res["plain_seconds"] / max(res["warm_seconds"], 1e-9)}, args)
        net.close()
        return


def eval_roofline_seconds(pairs_prec, sms, sm_mhz, dfma_per_s=None, d=3):
    """Roofline time of a solve's evaluations: per precision, the algorithmic
    work of its pairs over its binding unit's peak -- mixed: 2 ex2 per pair on
    the SFU; compensated: the FP32 lane-ops per pair of both passes; FP64: the
    FP64 operations per pair of both passes at the measured DFMA rate (None when
    the FP64 rate is not known).  Index = rsot_precision (FP64, MIXED,
    COMPENSATED)."""
    clk = sm_mhz * 1e6
    t = 2.0 * pairs_prec[1] / (SFU_EX2_PER_CLK_PER_SM * sms * clk)
    t += pairs_prec[2] * sum(COMP_FP32_OPS_PER_PAIR.values()) / (FP32_LANE_OPS_PER_CLK_PER_SM * sms * clk)
    if pairs_prec[0]:
        if not dfma_per_s:
            return None
        t += pairs_prec[0] * FP64_OPS_PER_PAIR[d] / dfma_per_s
    return t


def warmstart_network(args, log):
    """The warm-start network trained on the batched solver's potentials of
    args.train_seeds problems (seeds 10000..), cached under the temp directory
    by a hash of the library sources and the training settings; returns
    (net, info)."""
    import numpy as np
    import paper_2507_23602_gb300 as rs
    from paper_2507_23602_gb300 import warmstart as ws
    h = hashlib.sha256()
    for d in (os.path.join(ROOT, "paper_2507_23602_gb300", "csrc"),):
        for f in sorted(os.listdir(d)):
            h.update(open(os.path.join(d, f), "rb").read())
    for f in (os.path.join(ROOT, "paper_2507_23602_gb300", "warmstart.py"),
              os.path.join(ROOT, "rsot_inputs", "__init__.py")):
        h.update(open(f, "rb").read())
    h.update(f"{args.train_seeds}-{args.epochs}".encode())
    path = os.path.join(tempfile.gettempdir(), f"rsot_warmstart_{h.hexdigest()[:16]}.npz")
    if os.path.exists(path):
        z = np.load(path)
        net = rs.MLP(ws.IN_DIM, 256, seed=0)
        net.set_params(z["params"])
        info = {k: float(z[k]) for k in ("gen_seconds", "train_seconds", "samples")}
        info.update({"cached": True, "loss_history": z["loss"].tolist()})
        return net, info
    X, Y, t_gen = ws.generate(list(range(10000, 10000 + args.train_seeds)))
    log(f"warm start: {X.shape[0]} training rows generated in {t_gen:.1f} s")
    net, hist, t_train = ws.train(X, Y, epochs=args.epochs)
    log(f"warm start: trained in {t_train:.1f} s, loss {hist[0]:.3e} -> {hist[-1]:.3e}")
    np.savez(path, params=net.params(), gen_seconds=t_gen, train_seconds=t_train,
             samples=float(X.shape[0]), loss=np.array(hist))
    return net, {"gen_seconds": t_gen, "train_seconds": t_train, "samples": float(X.shape[0]),
                 "cached": False, "loss_history": hist}


def solve_metrics(args, P, p, dev, dfma_per_s):
    """The metric's solve-time half: (a) the cube solve eps 0.1 -> 1e-3 to
    ||grad J||_1 <= 1e-6 (mixed evaluations, refinement on compensated
    evaluations with the certified stop); (b) on the same held-out warm-start
    problems (d = 2, 4,096 targets, eps = 5e-3), the warm-started mixed batched
    solve against the plain FP64 GPU solve from psi = 0 with the eps-schedule.
    Each with wall time, iterations / rounds, converged count, the oracle's
    ||grad J||_1 at the returned potential and the roofline fraction
    (evaluations' roofline time / wall)."""
    import numpy as np
    import torch
    import paper_2507_23602_gb300 as rs
    from paper_2507_23602_gb300 import warmstart as ws
    import rsot_inputs as ri

    def log(msg):
        sys.stderr.write(f"[bench] {msg}\n")

    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    sm_max = float(measured_peaks().get("sm_max_mhz", 2070.0))
    out = {"tol_l1": 1e-6,
           "roofline_basis": f"evaluations' roofline time / wall: mixed 2 ex2 per pair at "
                             f"{SFU_EX2_PER_CLK_PER_SM} ex2/clk/SM, compensated "
                             f"{sum(COMP_FP32_OPS_PER_PAIR.values())} FP32 lane-ops per pair at "
                             f"{FP32_LANE_OPS_PER_CLK_PER_SM}/clk/SM, FP64 {FP64_OPS_PER_PAIR} (by d) "
                             f"FP64-pipe ops per pair at the measured DFMA rate "
                             f"({dfma_per_s:.4g}/s); {sms} SMs x {sm_max:.0f} MHz"}
    # (a) cube solve
    torch.cuda.synchronize()
    t = time.perf_counter()
    psi_c, st = P.solve(eps=p.eps, eps_start=0.1, eps_factor=0.5, tol_l1=1e-6, precision=rs.MIXED,
                        raise_on_error=False, max_iter=20000)
    wall = time.perf_counter() - t
    rt = eval_roofline_seconds(st.pairs_prec, sms, sm_max, dfma_per_s)
    out["cube"] = {"workload": f"cube-{p.nq}x{p.n}, eps 0.1 -> {p.eps:g} (x0.5), tol 1e-6",
                   "seconds": wall, "iters": st.iters, "evals": st.evals, "stages": st.stages,
                   "status": st.status, "converged": int(st.status == 0),
                   "grad_l1_reported": st.grad_l1,
                   "certified_grad_l1_bound": st.grad_l1 + rs.COMPENSATED_GRAD_REL * float(p.mass.sum()),
                   "evals_by_precision": dict(zip(("fp64", "mixed", "compensated"), st.evals_prec)),
                   "pairs_by_precision": dict(zip(("fp64", "mixed", "compensated"), st.pairs_prec)),
                   "roofline_seconds": rt, "roofline_frac": (rt / wall) if rt else None}
    log(f"cube solve {wall:.2f} s, {st.iters} iterations, status {st.status}")

    # (b) warm-started mixed batched vs plain FP64 on the same held-out problems
    net, info = warmstart_network(args, log)
    seeds = list(range(20000, 20000 + args.compare_problems))
    probs = [ri.warmstart_problem(sd) for sd in seeds]
    B = rs.Batch([(q.x, q.mass, q.y, q.nu) for q, _ in probs])
    epsv = np.full(len(probs), probs[0][0].eps)
    try:
        torch.cuda.synchronize()
        t = time.perf_counter()
        psi0 = np.concatenate([ws.predict(net, th, q.y, q.nu) for q, th in probs])
        t_pred = time.perf_counter() - t
        psi_w, sw = B.solve(epsv, psi0=psi0, eps_start=0.0, tol_l1=1e-6, precision=rs.MIXED,
                            refine_fp64=True, raise_on_error=False)
        wall_w = time.perf_counter() - t
        log(f"warm-started mixed batched: {wall_w:.2f} s, {sw['converged']}/{len(probs)} converged")
        t = time.perf_counter()
        psi_p, sp = B.solve(epsv, eps_start=0.1, eps_factor=0.5, tol_l1=1e-6, precision=rs.FP64,
                            raise_on_error=False)
        wall_p = time.perf_counter() - t
        log(f"plain FP64: {wall_p:.2f} s, {sp['converged']}/{len(probs)} converged")
    finally:
        B.close()
        net.close()

    def arm(st_, wall_):
        rt_ = eval_roofline_seconds(st_["pairs_prec"], sms, sm_max, dfma_per_s, d=2)
        return {"seconds": wall_, "rounds": st_["rounds"], "evals": st_["evals"],
                "converged": st_["converged"], "max_grad_l1_reported": st_["max_grad_l1"],
                "evals_by_precision": dict(zip(("fp64", "mixed", "compensated"), st_["evals_prec"])),
                "pairs_by_precision": dict(zip(("fp64", "mixed", "compensated"), st_["pairs_prec"])),
                "roofline_seconds": rt_, "roofline_frac": (rt_ / wall_) if rt_ else None}

    cmp_ = {"workload": f"{len(probs)} held-out problems (seeds {seeds[0]}..{seeds[-1]}): d = 2, "
                        f"{probs[0][0].nq} points x {probs[0][0].n} targets, eps {epsv[0]:g}",
            "warm_started_mixed_batched": arm(sw, wall_w),
            "plain_fp64_gpu": arm(sp, wall_p),
            "speedup": wall_p / max(wall_w, 1e-9),
            "network": dict(info, predict_seconds=t_pred,
                            note="trained before the timed solves on the batched solver's "
                                 "potentials; its time is reported here, not in either arm")}
    cmp_["warm_started_mixed_batched"]["predict_seconds_included"] = t_pred
    out["warm_vs_plain_fp64"] = cmp_

    # oracle gradients at the returned potentials (after every timed solve)
    if not args.no_oracle_check:
        import oracle
        t = time.perf_counter()
        _, go, _, _ = oracle.dual_grad(p.x, p.mass, p.y, p.nu, psi_c, p.eps)
        out["cube"]["oracle_grad_l1"] = float(np.abs(go).sum())
        for key, psi_all in (("warm_started_mixed_batched", psi_w), ("plain_fp64_gpu", psi_p)):
            mx, off = 0.0, 0
            for q, _ in probs:
                _, gq, _, _ = oracle.dual_grad(q.x, q.mass, q.y, q.nu, psi_all[off:off + q.n], q.eps)
                mx = max(mx, float(np.abs(gq).sum()))
                off += q.n
            cmp_[key]["oracle_max_grad_l1"] = mx
        out["oracle_check_seconds"] = time.perf_counter() - t
    return out


def main():
    args = parse()
    rank, world, local = dist_env()
    import numpy as np
    import rsot_inputs as ri
    if args.workload != "dense":
        if rank == 0 and args.impl == "ours":
            run_solve_workloads(args)
        return

    p = ri.cube_3d(mesh_n=args.mesh, n_targets=args.targets, eps=args.eps)
    psi = 0.005 * np.random.default_rng(2024).standard_normal(p.n)
    workload = f"cube-{p.nq}x{p.n}-dense-eps{args.eps:g}"
    if args.impl == "reference":
        run_reference(args, p, psi, workload)
        return

    import torch
    import paper_2507_23602_gb300 as rs
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as tdist
        tdist.init_process_group("nccl", device_id=dev)

    def barrier():
        if world > 1:
            import torch.distributed as tdist
            tdist.barrier()
        torch.cuda.synchronize()

    P = rs.Problem(p.x, p.mass, p.y, p.nu, stream=torch.cuda.current_stream())
    kind = {"auto": rs.PAIRS_AUTO, "tensor": rs.PAIRS_TENSOR, "fp32": rs.PAIRS_FP32}[args.pair_kernel]
    P.set_pair_kernel(kind)
    psi_d = torch.tensor(psi, device=dev)
    grad_d = torch.empty(p.n, dtype=torch.float64, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    pairs = p.nq * p.n

    for _ in range(args.warmup):
        P.eval(psi_d, p.eps, 0.0, rs.MIXED, grad_out=grad_d)

    clocks = Clocks(local)
    P.kernel_timing(True)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    barrier()
    clocks.start()
    wall0 = time.perf_counter()
    for k in range(args.steps):
        flush.zero_()
        starts[k].record()
        P.eval(psi_d, p.eps, 0.0, rs.MIXED, grad_out=grad_d)
        ends[k].record()
    barrier()
    wall = time.perf_counter() - wall0
    clk = clocks.stop()
    ktimes = P.kernel_times()
    P.kernel_timing(False)
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    total_s = max_over_ranks(sum(step_ms) / 1e3, world, dev)
    value = whole_job_rate(pairs, args.steps, world, total_s)
    ms_per_step = 1e3 * total_s / args.steps

    # the same evaluation with the other pair form (the tensor-core exponents,
    # opt-in, when the headline runs the default FP32 form): reported beside the
    # headline for comparison, not part of it
    fp32_pairs = None
    if not args.no_fp32_compare:
        other = rs.PAIRS_TENSOR if kind != rs.PAIRS_TENSOR else rs.PAIRS_FP32
        P.set_pair_kernel(other)
        for _ in range(max(1, args.warmup)):
            P.eval(psi_d, p.eps, 0.0, rs.MIXED, grad_out=grad_d)
        P.kernel_timing(True)
        fms = []
        for _ in range(args.steps):
            flush.zero_()
            a = torch.cuda.Event(enable_timing=True)
            b_ = torch.cuda.Event(enable_timing=True)
            a.record()
            P.eval(psi_d, p.eps, 0.0, rs.MIXED, grad_out=grad_d)
            b_.record()
            torch.cuda.synchronize()
            fms.append(a.elapsed_time(b_))
        fk = P.kernel_times()
        P.kernel_timing(False)
        P.set_pair_kernel(kind)
        fp32_pairs = {"pair_kernel": "tensor (opt-in)" if other == rs.PAIRS_TENSOR else "fp32",
                      "value": pairs / (sum(fms) / len(fms) * 1e-3) / 1e9, "unit": "G pairs/s",
                      "ms_per_step": sum(fms) / len(fms),
                      "per_kernel_ms": {k: v[0] / v[1] for k, v in fk.items()}}

    # the compensated evaluation (double-float pair exponents, certified gradient
    # bound): a secondary line, with its own roofline on the FP32 pipe
    comp = None
    if not args.no_compensated:
        for _ in range(max(1, min(args.warmup, 2))):
            P.eval(psi_d, p.eps, 0.0, rs.COMPENSATED, grad_out=grad_d)
        P.kernel_timing(True)
        cms = []
        for _ in range(max(1, min(args.steps, 3))):
            flush.zero_()
            a = torch.cuda.Event(enable_timing=True)
            b_ = torch.cuda.Event(enable_timing=True)
            a.record()
            P.eval(psi_d, p.eps, 0.0, rs.COMPENSATED, grad_out=grad_d)
            b_.record()
            torch.cuda.synchronize()
            cms.append(a.elapsed_time(b_))
        ck = {k: v[0] / v[1] for k, v in P.kernel_times().items()}
        P.kernel_timing(False)
        sms_c = torch.cuda.get_device_properties(dev).multi_processor_count
        sm_max_c = float(measured_peaks().get("sm_max_mhz", 2070.0))
        peak_ops = FP32_LANE_OPS_PER_CLK_PER_SM * sms_c * sm_max_c * 1e6 / 1e12
        dom_c = max(("lse_df", "grad_df"), key=lambda k: ck.get(k, 0.0))
        ops = COMP_FP32_OPS_PER_PAIR[dom_c] * pairs
        ach = ops / (ck[dom_c] * 1e-3) / 1e12
        comp = {"metric": "dual+grad G pairs/s (dense, compensated: double-float pair exponents)",
                "value": pairs / (sum(cms) / len(cms) * 1e-3) / 1e9, "unit": "G pairs/s",
                "ms_per_step": sum(cms) / len(cms), "per_kernel_ms": ck,
                "grad_l1_error_bound": rs.COMPENSATED_GRAD_REL * float(p.mass.sum()),
                "roofline": {"bound": "alu", "unit": "T FP32 lane-ops/s", "kernel": dom_c,
                             "achieved": ach, "peak": peak_ops, "frac": ach / peak_ops,
                             "peak_basis": f"{FP32_LANE_OPS_PER_CLK_PER_SM} FP32 lane-ops/clk/SM x "
                                           f"{sms_c} SMs x {sm_max_c:.0f} MHz; "
                                           f"{COMP_FP32_OPS_PER_PAIR[dom_c]} lane-ops per pair",
                             "traffic": None}}
        # the same evaluation truncated at tail 1e-12 (psi-aware cutoffs, block-skip
        # passes keeping exactly the FP64 path's pairs), at the bench potential
        P.eval_tail(psi_d, p.eps, 1e-12, rs.COMPENSATED, grad_out=grad_d)
        P.kernel_timing(True)
        tms, tpairs = [], 0
        for _ in range(max(1, min(args.steps, 3))):
            flush.zero_()
            a = torch.cuda.Event(enable_timing=True)
            b_ = torch.cuda.Event(enable_timing=True)
            a.record()
            _, _, tpairs = P.eval_tail(psi_d, p.eps, 1e-12, rs.COMPENSATED, grad_out=grad_d)
            b_.record()
            torch.cuda.synchronize()
            tms.append(a.elapsed_time(b_))
        tk = {k: v[0] / v[1] for k, v in P.kernel_times().items()}
        P.kernel_timing(False)
        comp["truncated_tail_1e-12"] = {"ms_per_step": sum(tms) / len(tms), "pairs_per_step": tpairs,
                                        "kept_fraction": tpairs / pairs, "per_kernel_ms": tk,
                                        "dense_equivalent": pairs / (sum(tms) / len(tms) * 1e-3) / 1e9,
                                        "unit": "G pairs/s"}

    # truncated evaluations at tail 1e-12 (secondary line, same workload): the
    # psi-aware cutoffs per pair (rsot_eval_dual_grad_tail) and the global tail
    # radius, at the solved potential (mixed solve to ||g||_1 <= 1e-5, eps
    # 0.1 -> eps: the regime in which a solver evaluates truncated) and at the
    # bench potential
    trunc = None
    if not args.no_trunc:
        def timed(fn):
            for _ in range(max(1, args.warmup)):
                fn()
            P.kernel_timing(True)
            tms, tp = [], 0
            for _ in range(args.steps):
                flush.zero_()
                a = torch.cuda.Event(enable_timing=True)
                b_ = torch.cuda.Event(enable_timing=True)
                a.record()
                _, _, tp = fn()
                b_.record()
                torch.cuda.synchronize()
                tms.append(a.elapsed_time(b_))
            tk = P.kernel_times()
            P.kernel_timing(False)
            return sum(tms) / len(tms), tp, tk

        sms_t = torch.cuda.get_device_properties(dev).multi_processor_count
        sfu_peak = SFU_EX2_PER_CLK_PER_SM * sms_t * float(measured_peaks().get("sm_max_mhz", 2070.0)) * 1e6
        hbm_peak = float(measured_peaks().get("hbm_gbs", 6800.0))

        def trunc_roofline(t_ms, tp):
            # SFU: two ex2 per kept pair (one per pass); HBM: the algorithmic bytes of
            # one evaluation (point stream x' + m + result, target records, the
            # gradient) -- both fractions, the larger one naming the binding unit
            ex2 = 2.0 * tp / (t_ms * 1e-3)
            by = p.nq * (8 * p.x.shape[1] + 16) + p.n * (16 + 8 + 8)
            gbs = by / (t_ms * 1e-3) / 1e9
            r = {"sfu": {"achieved_ex2_per_s": ex2, "peak": sfu_peak, "frac": ex2 / sfu_peak},
                 "hbm": {"achieved_gbs": gbs, "peak": hbm_peak, "frac": gbs / hbm_peak,
                         "algorithmic_bytes": by}}
            r["binds"] = "sfu" if r["sfu"]["frac"] >= r["hbm"]["frac"] else "hbm"
            return r

        def trunc_at(psi_t):
            t_ms, tp, tk = timed(lambda: P.eval_tail(psi_t, p.eps, 1e-12, rs.MIXED, grad_out=grad_d))
            R = P.radius_for_tail(psi_t, p.eps, 1e-12)
            r_ms, rp, rk = timed(lambda: P.eval(psi_t, p.eps, R, rs.MIXED, grad_out=grad_d))
            return {"value": tp / (t_ms * 1e-3) / 1e9, "unit": "G pairs/s",
                    "dense_equivalent": pairs / (t_ms * 1e-3) / 1e9, "pairs_per_step": tp,
                    "kept_fraction": tp / pairs, "ms_per_step": t_ms,
                    "roofline": trunc_roofline(t_ms, tp),
                    "per_kernel_ms": {k: v[0] / v[1] for k, v in tk.items()},
                    "gpu_launches": int(sum(v[1] for v in tk.values())),
                    "global_radius": {"radius": R, "pairs_per_step": rp, "kept_fraction": rp / pairs,
                                      "ms_per_step": r_ms, "value": rp / (r_ms * 1e-3) / 1e9,
                                      "dense_equivalent": pairs / (r_ms * 1e-3) / 1e9,
                                      "per_kernel_ms": {k: v[0] / v[1] for k, v in rk.items()}}}
        t0s = time.perf_counter()
        psi_sol, st_sol = P.solve(eps=p.eps, eps_start=0.1, eps_factor=0.5, tol_l1=1e-5,
                                  precision=rs.MIXED, refine_fp64=False, raise_on_error=False,
                                  max_iter=20000)
        solve_s = time.perf_counter() - t0s
        trunc = {"metric": "dual+grad G pairs/s (truncated at tail 1e-12, psi-aware cutoffs, at the "
                           "solved potential; pairs counted by the kernel)", "tail": 1e-12}
        trunc.update(trunc_at(torch.tensor(psi_sol, device=dev)))
        trunc["solution"] = {"seconds": solve_s, "iters": st_sol.iters, "grad_l1": st_sol.grad_l1,
                             "status": st_sol.status}
        trunc["at_bench_psi"] = trunc_at(psi_d)

    # end to end through the C ABI with host buffers (pinned), copies included
    e2e = None
    if not args.no_e2e:
        psi_h = torch.tensor(psi, dtype=torch.float64).pin_memory()
        grad_h = torch.empty(p.n, dtype=torch.float64).pin_memory()
        for _ in range(max(1, args.warmup)):
            P.eval(psi_h, p.eps, 0.0, rs.MIXED, grad_out=grad_h)
        e2e_s = 0.0
        for _ in range(args.steps):
            flush.zero_()
            torch.cuda.synchronize()
            t = time.perf_counter()
            P.eval(psi_h, p.eps, 0.0, rs.MIXED, grad_out=grad_h)
            e2e_s += time.perf_counter() - t
        e2e_s = max_over_ranks(e2e_s, world, dev)
        e2e = {"value": whole_job_rate(pairs, args.steps, world, e2e_s), "unit": "G pairs/s",
               "h2d_bytes_per_step": p.n * 8, "d2h_bytes_per_step": p.n * 8 + 48}

    if rank != 0:
        P.close()
        return

    # roofline of the dominant kernel (exponential-bound: 1 ex2 per pair per pass)
    dom = max(ktimes, key=lambda k: ktimes[k][0])
    tot_ms, launches = ktimes[dom]
    per_launch_s = tot_ms / launches / 1e3
    ex2_per_launch = pairs if dom in ("lse_mixed", "grad_mixed", "lse_tc", "grad_tc") else float("nan")
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    peaks = measured_peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    peak = SFU_EX2_PER_CLK_PER_SM * sms * sm_max * 1e6 / 1e9
    achieved = ex2_per_launch / per_launch_s / 1e9
    try:
        probe = rs.probe_ex2_rate() / 1e9
    except Exception:
        probe = None
    roof = {"bound": "alu", "unit": "Gex2/s", "kernel": dom, "achieved": achieved, "peak": peak,
            "frac": achieved / peak,
            "peak_basis": f"{SFU_EX2_PER_CLK_PER_SM} ex2/clk/SM x {sms} SMs x {sm_max:.0f} MHz "
                          "(unit count measured by the ex2 probe, at the maximum SM clock)",
            "probe_ex2_gps": probe,
            "frac_of_probe": (achieved / probe) if probe else None,
            "traffic": traffic_for(dom, workload),
            "per_kernel_ms": {k: v[0] / v[1] for k, v in ktimes.items()}}
    if clk and clk.get("sm_mhz"):
        roof["frac_at_measured_clock"] = achieved / (SFU_EX2_PER_CLK_PER_SM * sms * clk["sm_mhz"] * 1e6 / 1e9)

    # the metric's solve-time half (after every timed evaluation above)
    solve = None
    dfma = rs.probe_dfma_rate()
    if not args.no_solve and world == 1:
        solve = solve_metrics(args, P, p, dev, dfma)

    out = {
        "metric": "dual+grad G pairs/s (dense)", "value": value, "unit": "G pairs/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": workload, "nq": p.nq, "n": p.n, "eps": p.eps,
                   "pairs_per_step": pairs, "precision": "mixed (f32 pairs, f64 reductions)",
                   "pair_kernel": args.pair_kernel + (" (FP32 pair arithmetic for evaluations "
                                                      "returned to the caller)"
                                                      if args.pair_kernel == "auto" else ""),
                   "l2": "flushed between steps (256 MiB write, outside the step events)",
                   "parallelism": "replicas" if world > 1 else "single"},
        "roofline": roof,
        "e2e": e2e,
        "truncated": trunc,
        "other_pair_kernel": fp32_pairs,
        "compensated": comp,
        "solve": solve,
        "gpu_launches": int(sum(v[1] for v in ktimes.values())),
        "clocks": clk,
        "wall_s_timed_region": wall,
    }
    if world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(p, psi)
    print(json.dumps(out))
    P.close()


if __name__ == "__main__":
    main()
