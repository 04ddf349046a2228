#!/usr/bin/env python
"""Benchmark: IFMM factorization + preconditioned GMRES solve on one GB300.

One step = ifmm_factor (operator initialisation, leaf-to-root elimination with
colors, recompression, top-level explicit inverse) followed by bem_gmres (GMRES(30) to a true
relative residual of 1e-8, right-preconditioned by the IFMM solve, direct-sum
matvec), on the 131,072-point bumpy-sphere workload (depth 6, Chebyshev order 4,
eps = 1e-6, sigma = 3).  The tree and coloring (host, built once) and the points
and right-hand side are resident on the device before timing starts.

The JSON line reports seconds per step in the mixed-precision mode (pivots and
GMRES in FP64, Schur updates and recompression in FP32, FP64-accurate
double-float matvec) and, as "fp64", the plain FP64 mode on the same GPU.

--impl reference times the CPU oracle on a bounded sample of the same workload.
With torchrun (N > 1 ranks) each rank factors and solves its own replica of the
problem (replicas only: one problem does not shard), rank 0 prints the line.
"""

from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
# ALU peaks from unit counts and the 2070 MHz maximum SM clock (152 SMs):
# FP32: 128 lanes x 2 flop per clock; FP64: 2 DFMA x 2 flop per clock per SM.
ALU_PEAK_TFLOPS = {"fp32": 152 * 128 * 2 * 2.070e9 / 1e12, "fp64": 152 * 2 * 2 * 2.070e9 / 1e12}
METRIC = "IFMM factor+solve s at N=131k, eps=1e-6: mixed/learned vs plain FP64, same GB300"


def max_over_ranks(value: float, dist, device) -> float:
    """The largest per-rank value (each rank times its own replica; the job takes
    as long as the slowest).  dist None: a single process."""
    if dist is None:
        return float(value)
    import torch

    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="bumpy131k")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "bf16", "fp64"])
    ap.add_argument("--rank-mode", default="svd", choices=["svd", "learned"])
    ap.add_argument("--no-fp64", action="store_true", help="skip the plain FP64 comparison step")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    return ap.parse_args()


class Clocks:
    """nvidia-smi samples during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["active", "hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names[1:], f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def oracle_sample_seconds(workload_name: str, budget_s: float = 25.0):
    """The CPU oracle (as it stands) on a bounded sample of the workload: the same
    surface family and parameters at a smaller N with the same points per leaf,
    single-threaded BLAS, scaled linearly to the full N (the IFMM is O(N))."""
    code = r"""
import os, sys, time, json
sys.path.insert(0, %r)
from paper_1905_10602_gb300.workloads import WORKLOADS, surface, point_source_rhs
from oracle.ifmm import IFMMOracle
from oracle.dense import direct_matvec
from oracle.gmres import gmres
w = WORKLOADS[%r]
n, depth = %d, %d
pts = surface(w.shape, n, w.seed)
b = point_source_rhs(pts)
t0 = time.perf_counter()
o = IFMMOracle(pts, depth, w.cheb_order, w.eps, w.sigma).factor()
x, its, rel = gmres(lambda v: direct_matvec(pts, v), b, precond=o.solve, tol=1e-8)
t = time.perf_counter() - t0
print(json.dumps({"t": t, "n": n, "depth": depth, "its": its, "rel": rel}))
"""
    from paper_1905_10602_gb300.workloads import WORKLOADS

    w = WORKLOADS[workload_name]
    # same mean points per leaf: drop two levels per factor 16 in N
    n_s, d_s = w.n // 32, max(2, w.depth - 2)
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    out = subprocess.run([sys.executable, "-c", code % (ROOT, workload_name, n_s, d_s)], capture_output=True, text=True,
                         env=env, timeout=max(120, 10 * budget_s))
    if out.returncode != 0:
        raise RuntimeError(out.stderr[-2000:])
    r = json.loads(out.stdout.strip().splitlines()[-1])
    scaled = r["t"] * w.n / r["n"]
    return scaled, {"value": scaled, "unit": "s", "cores": 1, "kind": "oracle",
                    "sample": f"{w.shape} N={r['n']} depth {r['depth']} (same eps, order, sigma, points per leaf), "
                              f"factor + GMRES(30) to 1e-8 in {r['t']:.1f} s on 1 host core, x{w.n // r['n']} "
                              f"(work linear in N)"}


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    from paper_1905_10602_gb300.workloads import WORKLOADS

    times = []
    info = None
    for _ in range(args.warmup):
        oracle_sample_seconds(args.workload)
    for _ in range(args.steps):
        t, info = oracle_sample_seconds(args.workload)
        times.append(t)
    v = sum(times) / len(times)
    w = WORKLOADS[args.workload]
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": v * 1e3, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"{w.name}: {w.shape} N={w.n}, depth {w.depth}, Chebyshev {w.cheb_order}, "
                                   f"eps {w.eps}, sigma {w.sigma}", "global_batch": world},
            "cpu_baseline": dict(info, value=v),
            "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import numpy as np
    import torch

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_1905_10602_gb300 import build as _build

    _build.build()
    from paper_1905_10602_gb300 import ifmm
    from paper_1905_10602_gb300.workloads import WORKLOADS

    if args.workload == "batch64":
        return run_batch(args, rank, world, dist, ifmm, torch)
    w = WORKLOADS[args.workload]
    pts = w.points()
    b_host = w.rhs(pts)
    tree = ifmm.ifmm_build_tree(pts, w.depth)
    ifmm.ifmm_color(tree, w.sigma)
    b = torch.from_numpy(b_host).cuda()
    stream = torch.cuda.current_stream()
    sptr = __import__("ctypes").c_void_p(stream.cuda_stream)

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
            torch.cuda.synchronize()

    def step(prec, arith, rank_mode="svd"):
        k = ifmm.default_kernel(w.n, arith)
        f = ifmm.ifmm_factor(tree, w.cheb_order, w.eps, kernel=k, precision=prec, rank_mode=rank_mode, stream=sptr)
        x, its, rel = ifmm.bem_gmres(tree, b, precond=f, restart=30, tol=1e-8, kernel=k, stream=sptr)
        return f, its, rel

    arith = "fp64" if args.precision == "fp64" else "df"
    for _ in range(args.warmup):
        step(args.precision, arith, args.rank_mode)
    barrier()
    clocks = Clocks(local)
    clocks.start()
    ifmm.ifmm_profile(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    last = None
    for _ in range(args.steps):
        last = step(args.precision, arith, args.rank_mode)
    e1.record(stream)
    barrier()
    prof = ifmm.ifmm_profile_query()
    ifmm.ifmm_profile(False)
    clk = clocks.stop()
    ms = e0.elapsed_time(e1) / args.steps
    ms = max_over_ranks(ms, dist, "cuda")
    fact, its, rel = last
    stats = ifmm.ifmm_fact_stats(fact)
    # kernels the library launched (every launch is counted as it is issued;
    # a solve-graph replay counts its kernel nodes)
    launches = prof.pop("kernels", (0, 0.0))[0] // args.steps
    # dominant kernel of the step and its roofline (ALU-bound dense kernels)
    flops_of = {"svd_fp32": stats["flops_svd"], "svd_fp64": stats["flops_svd"], "qr_fp32": stats["flops_qr"],
                "qr_fp64": stats["flops_qr"], "gemm_fp32": stats["flops_gemm"], "gemm_fp64": stats["flops_gemm"],
                "gauss_jordan": stats["flops_inv"], "gauss_jordan_big": stats["flops_lu"]}
    # the shared-memory and global-memory QR kernels share one work counter (the
    # cluster launches are counted, and timed inside the qr_* regions)
    for g in ("fp32", "fp64"):
        prof.pop(f"qr_cluster_{g}", None)
        if f"qr_global_{g}" in prof:
            n1, m1 = prof.get(f"qr_{g}", (0, 0.0))
            n2, m2 = prof.pop(f"qr_global_{g}")
            prof[f"qr_{g}"] = (n1 + n2, m1 + m2)
    top = max(prof.items(), key=lambda kv: kv[1][1])
    kname, (klaunch, kms) = top
    kms /= args.steps
    roof = None
    if kname in flops_of:
        kind = "fp64" if (kname.endswith("fp64") or kname.startswith("gauss")) else "fp32"
        achieved = flops_of[kname] / (kms / 1e3) / 1e12
        peak = ALU_PEAK_TFLOPS[kind]
        roof = {"bound": "alu", "kernel": kname, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": None, "launches_per_step": klaunch // args.steps,
                "ms_per_step": kms, "peak_note": f"{kind} FMA units x 2070 MHz (derived)"}
    elif kname == "matvec":
        pairs = float(w.n) * w.n
        roof = {"bound": "alu", "kernel": kname, "achieved": None, "peak": None, "unit": "TFLOP/s", "frac": None,
                "traffic": None, "ms_per_step": kms, "pairs_per_s": pairs * (klaunch // args.steps) / (kms / 1e3)}
    out = {"metric": METRIC, "value": ms / 1e3, "unit": "s", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
           "dtype": "f32" if args.precision == "fp32" else ("bf16" if args.precision == "bf16" else "f64"),
           "data": "synthetic",
           "config": {"workload": f"{w.name}: {w.shape} N={w.n}, depth {w.depth}, Chebyshev order {w.cheb_order}, "
                                  f"eps {w.eps}, sigma {w.sigma}, GMRES(30) to 1e-8",
                      "precision": args.precision, "rank_mode": args.rank_mode, "matvec": arith,
                      "global_batch": world, "l2": "working set > L2 (factor of several GB written every step)"},
           "gmres": {"iterations": its, "relres": rel},
           "factor_s": stats["time_factor"], "gpu_launches": int(launches),
           "kernels": {k: {"launches_per_step": n // args.steps, "ms_per_step": m / args.steps}
                       for k, (n, m) in prof.items() if n},
           "roofline": roof, "clocks": clk}
    # plain FP64 on the same GPU (one step, untimed by the events above)
    if not args.no_fp64 and args.precision != "fp64":
        barrier()
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        f64, its64, rel64 = step("fp64", "fp64")
        s1.record(stream)
        barrier()
        out["fp64"] = {"value": s0.elapsed_time(s1) / 1e3, "unit": "s", "gmres_iterations": its64, "relres": rel64,
                       "factor_s": ifmm.ifmm_fact_stats(f64)["time_factor"]}
        out["speedup_vs_fp64"] = out["fp64"]["value"] / out["value"]
    # end to end through the C ABI with host buffers
    if not args.no_e2e:
        barrier()
        t0 = time.perf_counter()
        tr = ifmm.ifmm_build_tree(pts, w.depth)
        ifmm.ifmm_color(tr, w.sigma)
        k = ifmm.default_kernel(w.n, arith)
        f = ifmm.ifmm_factor(tr, w.cheb_order, w.eps, kernel=k, precision=args.precision, rank_mode=args.rank_mode)
        xh, _, _ = ifmm.bem_gmres(tr, b_host, precond=f, tol=1e-8, kernel=k)
        torch.cuda.synchronize()
        te = time.perf_counter() - t0
        n = w.n
        out["e2e"] = {"value": te, "unit": "s", "h2d_bytes_per_step": int(n * (3 * 8 + 6 * 4 + 4 + 8)),
                      "d2h_bytes_per_step": int(n * 8),
                      "note": "tree + coloring + factor + GMRES from host points and host b to host x"}
    if rank == 0 and not args.no_cpu and world == 1:
        try:
            _, out["cpu_baseline"] = oracle_sample_seconds(args.workload)
        except Exception as e:  # the oracle leg must not hide the GPU result
            out["cpu_baseline"] = {"value": None, "error": str(e)[:200]}
    if rank == 0:
        print(json.dumps(out), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def run_batch(args, rank, world, dist, ifmm, torch):
    """64 independent problems (N log-uniform in [4096, 65536], spheres / tori /
    bumpy spheres, order 4, eps 1e-6) factored and solved together per step."""
    from paper_1905_10602_gb300.workloads import batch_workloads

    ws = batch_workloads(64, 5)
    trees, bs = [], []
    for w in ws:
        pts = w.points()
        t = ifmm.ifmm_build_tree(pts, w.depth)
        ifmm.ifmm_color(t, w.sigma)
        trees.append(t)
        bs.append(w.rhs(pts))
    arith = "fp64" if args.precision == "fp64" else "df"
    ks = [ifmm.default_kernel(w.n, arith) for w in ws]

    def step():
        fs = ifmm.ifmm_factor_batched(trees, 4, 1e-6, precision=args.precision, nworkers=8, kernels=ks)
        xs, its, rel = ifmm.bem_gmres_batched(trees, bs, fs, kernels=ks, nworkers=8)
        return its, rel

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    clocks = Clocks(int(os.environ.get("LOCAL_RANK", "0")))
    clocks.start()
    ifmm.ifmm_profile(False)  # launch counts only (no per-launch events)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        its, rel = step()
    torch.cuda.synchronize()
    dt = (time.perf_counter() - t0) / args.steps
    launches = ifmm.ifmm_profile_query().get("kernels", (0, 0.0))[0] // args.steps
    clk = clocks.stop()
    dt = max_over_ranks(dt, dist, "cuda")
    out = {"metric": METRIC + " (64-problem batch)", "value": dt, "unit": "s", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": False, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32" if args.precision != "fp64" else "f64", "data": "synthetic",
           "config": {"workload": "64 problems, N log-uniform in [4096, 65536], sphere/torus/bumpy, order 4, eps 1e-6, "
                                  "GMRES(30) to 1e-8, 8 worker streams", "precision": args.precision,
                      "global_batch": 64 * world},
           "problems_per_s": 64 * world / dt, "max_gmres_iterations": max(its), "max_relres": max(rel),
           "timing": "host wall clock around the batched calls (several streams)", "gpu_launches": int(launches),
           "clocks": clk}
    if rank == 0:
        print(json.dumps(out), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
