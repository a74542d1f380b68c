"""Benchmark: solves/s of a sequence of Poisson solves to rtol 1e-8 (one step = one
time step's solve through the whole hot path: condensation, deflated/recycled PCG
with BDDC, interior recovery, recycling update).

Default workload: 128^3 graded Q1 mesh (aspect 40), 4096 subdomains of 8^3
elements, three-level BDDC, B4 recycling with k = 40; the headline arm runs the
mixed-precision path (df64 Schur operator, FP32 BDDC, flexible PCG, FP64 Krylov),
and the plain FP64 PCG-BDDC arm (no deflation) runs on the same GPU for the ratio.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]

Multi-GPU (torchrun): every rank solves an independent sequence (its own RHS
seed) on its own GPU; the path has no data exchange between sequences, so the
ranks share nothing but the start/stop barrier and the max-over-ranks timing.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from workload import WORKLOADS, load_sequence, workload_mesh  # noqa: E402

METRIC = "solves/s to rtol 1e-8 at 128^3: recycled mixed-prec vs plain FP64; %HBM peak"


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled during the timed region."""

    def __init__(self, index: int):
        self.index = index
        self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.proc = None

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.file, stderr=subprocess.DEVNULL)
        except (FileNotFoundError, OSError):
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        self.file.flush()
        self.file.seek(0)
        sm, mx, reasons = [], [], set()
        for line in self.file:
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
            for name, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def solver_options(wl, mixed: bool) -> dict:
    """Options of a workload: the mixed-precision arm and the plain FP64 arm share mesh,
    partition and constraints (adaptive ones included)."""
    o = dict(levels=wl["levels"], coarse_group=4, use_corners=wl["corners"], use_edges=wl["edges"],
             use_faces=wl["faces"], weights="diag", adaptive=wl.get("adaptive", 0), tau=wl.get("tau", 10.0),
             max_eig_per_face=10, maxit=500)
    if mixed:
        o.update(schur_prec="df64", precond_prec="fp32", flexible=1)
    else:
        o.update(schur_prec="fp64", precond_prec="fp64", flexible=0)
    return o


def run_arm(torch, solver, F_dev, warmup, steps, k, strategy, rtol, world, dist, prof=False):
    """W untimed solves then K timed solves; returns (seconds, stats list, profile)."""
    rec = solver.recycler(k, strategy)
    x = torch.empty(solver.n_free, dtype=torch.float64, device=F_dev.device)
    for t in range(warmup):
        solver.solve(F_dev[t], rec, rtol, out=x)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    if prof:
        solver.profile(True, read=True)  # reset counters, start timing
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stats = []
    torch.cuda.synchronize()
    e0.record(stream)
    for t in range(warmup, warmup + steps):
        _, st = solver.solve(F_dev[t], rec, rtol, out=x)
        stats.append(st)
    e1.record(stream)
    torch.cuda.synchronize()
    sec = e0.elapsed_time(e1) / 1e3
    pr = solver.profile(False, read=True) if prof else None
    if dist:
        t_ = torch.tensor([sec], device=F_dev.device)
        dist.all_reduce(t_, op=dist.ReduceOp.MAX)
        sec = float(t_.item())
    rec.close()
    return sec, stats, pr


def run_e2e(torch, solver, F_host, warmup, steps, k, strategy, rtol):
    """Same metric through the public API from pinned host buffers (H2D of f, solve, D2H of x) per step."""
    rec = solver.recycler(k, strategy)
    n = solver.n_free
    f_dev = torch.empty(n, dtype=torch.float64, device="cuda")
    x_dev = torch.empty(n, dtype=torch.float64, device="cuda")
    x_host = torch.empty(n, dtype=torch.float64).pin_memory()
    for t in range(warmup):
        f_dev.copy_(F_host[t], non_blocking=True)
        solver.solve(f_dev, rec, rtol, out=x_dev)
        x_host.copy_(x_dev, non_blocking=True)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for t in range(warmup, warmup + steps):
        f_dev.copy_(F_host[t], non_blocking=True)
        solver.solve(f_dev, rec, rtol, out=x_dev)
        x_host.copy_(x_dev, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    rec.close()
    return e0.elapsed_time(e1) / 1e3, n * 8, n * 8


def cpu_baseline(mesh, seed, nsolve=2, sequence=500):
    """The oracle (nested-dissection multifrontal sparse Cholesky, FP64) on the host cores:
    factorization once, then per-step triangular solves; solves/s of a sequence of `sequence`
    steps with the factorization amortized over it."""
    from oracle import cholesky, q1
    cores = os.cpu_count()
    t0 = time.perf_counter()
    K = q1.assemble(mesh)
    ch = cholesky.factor_mesh(mesh, K)
    t_fac = time.perf_counter() - t0
    F = load_sequence(mesh, seed, nsolve)
    t0 = time.perf_counter()
    for f in F:
        ch.solve(f)
    t_sol = (time.perf_counter() - t0) / nsolve
    rate = sequence / (t_fac + sequence * t_sol)
    return {"value": rate, "unit": "solves/s", "cores": cores, "kind": "oracle",
            "sample": f"assembly+factorization ({t_fac:.1f} s) and {nsolve} triangular-solve steps "
                      f"({t_sol:.2f} s each) of the same system; rate amortizes the factorization over a "
                      f"{sequence}-step sequence",
            "factor_s": t_fac, "solve_s": t_sol}


def reference_arm(args, wl, world, rank):
    """The oracle as the reference arm: sparse-Cholesky solves per step on the host cores."""
    if rank != 0:
        return
    from oracle import cholesky, q1
    mesh = workload_mesh(args.workload)
    t0 = time.perf_counter()
    ch = cholesky.factor_mesh(mesh, q1.assemble(mesh))
    t_fac = time.perf_counter() - t0
    F = load_sequence(mesh, wl["seed"], args.warmup + args.steps)
    for t in range(args.warmup):
        ch.solve(F[t])
    t0 = time.perf_counter()
    for t in range(args.warmup, args.warmup + args.steps):
        ch.solve(F[t])
    sec = time.perf_counter() - t0
    value = args.steps / sec
    cores = os.cpu_count()
    line = {"metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * sec / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": args.workload, "n": wl["n"], "subdomains": (wl["n"] // wl["sub"]) ** 3,
                       "rtol": wl["rtol"], "method": "sparse Cholesky (oracle), exact solve per step"},
            "cpu_baseline": {"value": value, "unit": "solves/s", "cores": cores, "kind": "oracle",
                             "sample": f"{args.steps} triangular-solve steps after a {t_fac:.1f} s factorization "
                                       "(setup excluded, as for the GPU arm)"},
            "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "setup_s": t_fac}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="graded128", choices=sorted(WORKLOADS))
    ap.add_argument("--no-plain", action="store_true", help="skip the plain FP64 arm")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--rtol", type=float, default=None)
    args = ap.parse_args()
    wl = WORKLOADS[args.workload]
    world, rank, local = dist_env()
    if args.impl == "reference":
        reference_arm(args, wl, world, rank)
        return

    import torch
    import paper_2412_17543_gb300 as pkg
    dist = None
    if world > 1:
        import torch.distributed as tdist
        tdist.init_process_group("nccl")
        dist = tdist
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    rtol = args.rtol if args.rtol is not None else wl["rtol"]
    k = wl["k"]
    mesh = workload_mesh(args.workload)
    seed = wl["seed"] + 1000 * rank
    nsteps = args.warmup + args.steps
    t0 = time.perf_counter()
    F_host = torch.from_numpy(load_sequence(mesh, seed, nsteps))
    t_rhs = time.perf_counter() - t0
    F_dev = F_host.to(dev)

    t0 = time.perf_counter()
    mixed = pkg.Solver(mesh, **solver_options(wl, True))
    setup_mixed = time.perf_counter() - t0
    hbm, peak_kind = peaks()
    with ClockSampler(local) as clk:
        sec, stats, (prof, launches) = run_arm(torch, mixed, F_dev, args.warmup, args.steps, k, "B4", rtol, world,
                                               dist, prof=True)
    clocks = clk.summary()
    total_solves = args.steps * world
    value = total_solves / sec
    its = [s["iters"] for s in stats]

    plain = None
    if not args.no_plain:
        t0 = time.perf_counter()
        ps = pkg.Solver(mesh, **solver_options(wl, False))
        setup_plain = time.perf_counter() - t0
        psec, pstats, _ = run_arm(torch, ps, F_dev, args.warmup, args.steps, 0, "B4", rtol, world, dist)
        pits = [s["iters"] for s in pstats]
        plain = {"value": args.steps * world / psec, "unit": "solves/s", "ms_per_step": 1e3 * psec / args.steps,
                 "iters_min_max_avg": [min(pits), max(pits), sum(pits) / len(pits)], "setup_s": setup_plain,
                 "options": "FP64 Schur operator and BDDC, no deflation, x_prev initial guess, ||r||/||b|| stop"}
        ps.close()
        del ps

    e2e = None
    if not args.no_e2e:
        Fp = F_host.pin_memory()
        esec, h2d, d2h = run_e2e(torch, mixed, Fp, args.warmup, args.steps, k, "B4", rtol)
        e2e = {"value": args.steps * world / esec, "unit": "solves/s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h}

    kii = prof["symv_KIIinv"]
    kii_ms = kii[0] / max(kii[1], 1)
    achieved = kii[2] / (kii_ms / 1e3) / 1e9 if kii[1] else None
    roof = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
            "frac": (achieved / hbm) if achieved else None, "traffic": None,
            "kernel": "k_symv<DF64> (batched K_II^{-1} GEMV)", "peak_kind": f"{peak_kind} hbm_gbs",
            "alg_bytes_per_launch": kii[2], "avg_launch_ms": kii_ms, "launches": kii[1]}
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = cpu_baseline(mesh, wl["seed"])

    if rank == 0:
        per_kernel = {name: {"ms_total": v[0], "launches": v[1], "avg_ms": (v[0] / v[1]) if v[1] else None}
                      for name, v in prof.items()}
        line = {"metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": 1e3 * sec / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64 (df64 Schur, f32 BDDC)", "data": "synthetic",
                "config": {"workload": args.workload, "n": wl["n"], "subdomains": (wl["n"] // wl["sub"]) ** 3,
                           "levels": wl["levels"], "coarse_group": 4, "k": k, "strategy": "B4", "rtol": rtol,
                           "adaptive": bool(wl.get("adaptive", 0)), "tau": wl.get("tau"),
                           "n_adaptive": mixed.info["n_adaptive"], "grading_ratio": mesh.info["ratio"],
                           "max_aspect": mesh.info["max_aspect"], "n_free": mixed.n_free,
                           "n_gamma": mixed.n_gamma, "n_coarse": mixed.info["n_coarse"],
                           "l2": "operators of 3.1 GB stream from HBM every iteration (inputs larger than L2)",
                           "rhs_seed": seed},
                "iters_min_max_avg": [min(its), max(its), sum(its) / len(its)],
                "frozen_at_end": bool(stats[-1]["frozen"]),
                "setup_s": setup_mixed, "rhs_gen_s": t_rhs,
                "plain_fp64": plain,
                "speedup_vs_plain": (value / plain["value"]) if plain else None,
                "e2e": e2e, "roofline": roof, "cpu_baseline": cpu, "clocks": clocks,
                "gpu_launches": launches, "kernels": per_kernel}
        print(json.dumps(line), flush=True)
    mixed.close()
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
