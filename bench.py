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


def run_arm(torch, solver, F_dev, warmup, steps, k, strategy, rtol, world, dist, prof=False, capture=(),
            keep_state=None):
    """W untimed solves then K timed solves; returns (seconds, stats list, (profile, kernel launches)).

    Without prof the solves run as the library runs them by default: each PCG loop is one
    CUDA-graph launch. With prof, CUDA events bracket every operator application, which
    needs the host-issued form of the same loop (same kernels, identical results).
    capture: step indices whose solutions are copied to the host after the timed region
    (into the dict keep_state["x"]); keep_state["recycle"] receives the recycle state."""
    rec = solver.recycler(k, strategy)
    x = torch.empty(solver.n_free, dtype=torch.float64, device=F_dev.device)
    for t in range(warmup):
        solver.solve(F_dev[t], rec, rtol, out=x)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    solver.profile(prof, read=True)  # resets the counters; prof: starts event timing
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stats = []
    torch.cuda.synchronize()
    kept = {}
    e0.record(stream)
    for t in range(warmup, warmup + steps):
        _, st = solver.solve(F_dev[t], rec, rtol, out=x)
        stats.append(st)
        if t in capture:
            kept[t] = x.clone()
    e1.record(stream)
    torch.cuda.synchronize()
    sec = e0.elapsed_time(e1) / 1e3
    pr = solver.profile(False, read=True)
    if keep_state is not None:
        keep_state["x"] = {t: v.cpu().numpy() for t, v in kept.items()}
        keep_state["recycle"] = rec.state()
    sec = max_over_ranks(torch, sec, dist, F_dev.device)
    rec.close()
    return sec, stats, pr


class CopyPipeline:
    """Steps t0 .. t1-1 of an end-to-end run: each step copies its input from pinned host
    memory to the device, runs `solve(f_dev, x_dev)` (a public-API call that returns when its
    work is done) and copies the result back to pinned host memory. The copies run on a
    second stream with two device buffers each way, so the next step's input goes up and
    the previous result comes down while a solve runs; run() returns with all of it ordered
    before the current stream's next work."""

    def __init__(self, torch, F_host, solve):
        self.torch, self.F, self.solve = torch, F_host, solve
        shape, dev = F_host[0].shape, torch.device("cuda", torch.cuda.current_device())
        self.f_dev = [torch.empty(shape, dtype=torch.float64, device=dev) for _ in range(2)]
        self.x_dev = [torch.empty(shape, dtype=torch.float64, device=dev) for _ in range(2)]
        self.x_host = [torch.empty(shape, dtype=torch.float64).pin_memory() for _ in range(2)]
        self.cs = torch.cuda.Stream()

    def run(self, t0, t1, e_start=None):
        torch, cs = self.torch, self.cs
        stream = torch.cuda.current_stream()
        if e_start is not None:
            cs.wait_event(e_start)
        up = [torch.cuda.Event() for _ in range(2)]
        with torch.cuda.stream(cs):
            self.f_dev[t0 % 2].copy_(self.F[t0], non_blocking=True)
            up[t0 % 2].record(cs)
        for t in range(t0, t1):
            b = t % 2
            stream.wait_event(up[b])
            if t + 1 < t1:
                with torch.cuda.stream(cs):
                    self.f_dev[(t + 1) % 2].copy_(self.F[t + 1], non_blocking=True)
                    up[(t + 1) % 2].record(cs)
            self.solve(self.f_dev[b], self.x_dev[b])
            done = torch.cuda.Event()
            done.record(stream)
            cs.wait_event(done)
            with torch.cuda.stream(cs):
                self.x_host[b].copy_(self.x_dev[b], non_blocking=True)
        stream.wait_stream(cs)


def run_e2e(torch, solver, F_host, warmup, steps, k, strategy, rtol, dist=None):
    """Same metric through the public API (Solver.solve) from pinned host buffers: every step
    copies its right-hand side up and its solution back inside the timed region
    (CopyPipeline)."""
    rec = solver.recycler(k, strategy)
    n = solver.n_free
    pipe = CopyPipeline(torch, F_host, lambda f, x: solver.solve(f, rec, rtol, out=x))
    pipe.run(0, warmup)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    pipe.run(warmup, warmup + steps, e0)
    e1.record(stream)
    torch.cuda.synchronize()
    rec.close()
    sec = max_over_ranks(torch, e0.elapsed_time(e1) / 1e3, dist, torch.device("cuda", torch.cuda.current_device()))
    return sec, n * 8, n * 8


class OracleSample:
    """The oracle (nested-dissection multifrontal sparse Cholesky, FP64) on a member of the
    workload's graded-mesh family with sample_n^3 elements; sample_n equal to the workload's
    n solves the workload itself. The factorization is setup (excluded from rates, as the
    GPU arm's setup is); one step solves one right-hand side of the workload's sequence (two
    triangular solves that stream the factor once)."""

    def __init__(self, workload: str, wl, sample_n: int = 48, n: int | None = None):
        from oracle import cholesky, q1
        full = workload_mesh(workload, n=n)  # the mesh the GPU arm solves (--n overrides the size)
        self.n_full = full.nx
        self.sample_n = min(sample_n, full.nx)
        self.is_full = self.sample_n == full.nx
        self.mesh = full if self.is_full else workload_mesh(workload, n=self.sample_n)
        t0 = time.perf_counter()
        self.ch = cholesky.factor_mesh(self.mesh, q1.assemble(self.mesh))
        self.t_fac = time.perf_counter() - t0
        x0, x1, y0, y1, z0, z1 = full.free_box
        self.nnz_full, self.madd_full = cholesky.symbolic_counts((x1 - x0, y1 - y0, z1 - z0))
        self.nnz_s = self.ch.nnz_L()
        self.scale = self.nnz_full / self.nnz_s
        self.seed = wl["seed"]

    def run(self, nsolve: int, start: int = 0, warmup: int = 0):
        """(seconds per solve step, {step: solution}) for steps start .. start + nsolve - 1 of the
        sequence on the sample, after `warmup` untimed steps before them."""
        F = load_sequence(self.mesh, self.seed, warmup + nsolve, max(0, start - warmup))
        for t in range(warmup):
            self.ch.solve(F[t])
        xs = {}
        t0 = time.perf_counter()
        for i in range(nsolve):
            xs[start + i] = self.ch.solve(F[warmup + i])
        return (time.perf_counter() - t0) / nsolve, xs

    def describe(self, nsolve: int, t_sol: float) -> str:
        what = (f"the {self.n_full}^3 workload itself" if self.is_full else
                f"the {self.sample_n}^3 member of the workload's graded-mesh family")
        return (f"sparse Cholesky of {what} on {oracle_threads()} host threads (factor {self.t_fac:.1f} s, "
                f"setup excluded as for the GPU arm; {nsolve} solve steps at {t_sol:.3f} s each)")

    def measured(self, nsolve: int, t_sol: float) -> dict:
        return {"n": self.sample_n, "solves_per_s": 1.0 / t_sol, "solve_s": t_sol, "solve_steps": nsolve,
                "factor_s": self.t_fac, "nnz_L": self.nnz_s}

    def extrapolation(self, t_sol: float):
        if self.is_full:
            return None
        return {"solves_per_s": 1.0 / (t_sol * self.scale), "kind": "estimate, not measured",
                "basis": (f"solve time scaled by the ratio of factor nonzeros of the two nested-dissection "
                          f"orderings, {self.nnz_full:.3e} / {self.nnz_s:.3e} = {self.scale:.1f} (symbolic counts)")}


def oracle_threads() -> int:
    """Host threads the oracle's BLAS may use (OMP/OpenBLAS limits, else every core)."""
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS"):
        v = os.environ.get(var)
        if v and v.isdigit():
            return int(v)
    return os.cpu_count() or 1


def cpu_baseline(args, wl, nsolve=3, gpu_x=None, steps_from=0):
    """Timed CPU baseline: the oracle on a bounded sample of the workload (OracleSample).

    value is in the metric's unit: measured when the sample is the workload itself, else the
    measured sample rate scaled to the workload (marked as an estimate). When the sample is
    the workload, the same time steps' GPU solutions (gpu_x) are compared with the oracle's:
    relative 2-norm error of the full free-node solution per step."""
    smp = OracleSample(args.workload, wl, args.cpu_baseline_n, args.n)
    t_sol, xs = smp.run(nsolve, start=steps_from)
    ext = smp.extrapolation(t_sol)
    out = {"value": ext["solves_per_s"] if ext else 1.0 / t_sol, "unit": "solves/s", "cores": oracle_threads(),
           "kind": "oracle", "sample": smp.describe(nsolve, t_sol), "measured": smp.measured(nsolve, t_sol),
           "value_is": "scaled estimate (see extrapolation)" if ext else "measured on the workload",
           "extrapolation": ext}
    if smp.is_full and gpu_x:
        errs = {}
        for t, xo in xs.items():
            if t in gpu_x:
                errs[t] = float(np.linalg.norm(gpu_x[t] - xo) / np.linalg.norm(xo))
        out["gpu_rel_err_vs_oracle"] = {"steps": sorted(errs), "rel_err": [errs[t] for t in sorted(errs)],
                                        "max": max(errs.values()) if errs else None, "rtol": wl["rtol"]}
    return out


def reference_arm(args, wl, world, rank):
    """The oracle as the reference arm: W + K sparse-Cholesky solve steps on the host cores,
    on the bounded sample of the workload (OracleSample). Every number is the measured one of
    what ran; the workload-size rate from the factor-size ratio is reported separately as an
    estimate."""
    if rank != 0:
        return None
    smp = OracleSample(args.workload, wl, args.cpu_baseline_n, args.n)
    t_sol, _ = smp.run(args.steps, warmup=args.warmup)
    sec = t_sol * args.steps
    value = args.steps / sec
    ext = smp.extrapolation(t_sol)
    wname = args.workload if smp.is_full else f"{args.workload} (oracle on its {smp.sample_n}^3 member)"
    line = {"metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t_sol, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": wname, "n": smp.sample_n, "subdomains": (wl["n"] // wl["sub"]) ** 3,
                       "rtol": wl["rtol"], "method": "sparse Cholesky (oracle), exact solve per step"},
            "cpu_baseline": {"value": value, "unit": "solves/s", "cores": oracle_threads(), "kind": "oracle",
                             "sample": smp.describe(args.steps, t_sol)},
            "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "extrapolated_to_workload": ext, "setup_s": smp.t_fac}
    print(json.dumps(line), flush=True)
    return line


def max_over_ranks(torch, sec: float, dist, device) -> float:
    """Slowest rank's timed-region length (the whole-job time of weak-scaled replicas)."""
    if not dist:
        return sec
    t_ = torch.tensor([sec], dtype=torch.float64, device=device)
    dist.all_reduce(t_, op=dist.ReduceOp.MAX)
    return float(t_.item())


def rank_seed(wl, rank: int) -> int:
    """Each rank solves its own independent sequence (replicas, no data exchange)."""
    return wl["seed"] + 1000 * rank


# FP32 instruction issue of GB300: 152 SMs x 128 FP32 lanes x 2070 MHz (maximum SM clock);
# a df64 multiply-add (error-free two-product plus two-sum accumulation) takes 12 FP32
# instructions, so the df64 arithmetic of the Schur operator peaks at 40.3e12 / 12 df64
# multiply-adds per second, i.e. 6.71 TFLOP/s counted as FP64-equivalent flops
FP32_INSTR_PEAK = 152 * 128 * 2070e6
DF64_MADD_INSTR = 12
DF64_TFLOPS_PEAK = 2 * FP32_INSTR_PEAK / DF64_MADD_INSTR / 1e12


def tensor_peak(kind: str):
    """Dense tensor peak of the ensemble N_i kernel's operand type: the measured bf16 cuBLAS
    rate (burst), times the nominal tf32 : bf16 ratio (1.1 : 2.25 PFLOP/s) for tf32."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    bf16 = float(json.load(open(p))["bf16_tflops"]) if os.path.exists(p) else 1900.0
    return bf16 * (1.1 / 2.25) if kind == "tf32" else bf16


def kernel_table(prof, hbm, tensor_kind=None):
    """Per profiled class: device time, and against its roofline the achieved rate on
    algorithmic bytes (HBM) or algorithmic flops (df64 arithmetic on the FP32 pipes; for the
    ensemble N_i products the tensor-core work as issued, against the tensor peak of its
    operand type)."""
    out = {}
    for name, v in prof.items():
        ms, n, ab, af = v
        avg = ms / n if n else None
        e = {"ms_total": ms, "launches": n, "avg_ms": avg}
        if n and ab:
            gbs = ab / (avg / 1e3) / 1e9
            e.update(alg_bytes=ab, achieved_gbs=gbs, hbm_frac=gbs / hbm)
        if n and af:
            tf = af / (avg / 1e3) / 1e12
            if name == "ens_N" and tensor_kind:
                pk = tensor_peak(tensor_kind)
                e.update(tensor_flops_issued=af, tensor_tflops=tf, tensor_peak_tflops=pk,
                         tensor_kind=tensor_kind, tensor_frac=tf / pk)
            else:
                e.update(alg_flops=af, achieved_tflops=tf, alu_peak_tflops=DF64_TFLOPS_PEAK,
                         alu_frac=tf / DF64_TFLOPS_PEAK)
        out[name] = e
    return out


PROF_TIMING = ("CUDA events around every launch of the kernel on its stream, in a replay of the same warm-up and "
               "timed steps (fresh recycle state, identical iterates) with the PCG loop issued from the host; "
               "the timed steps themselves run each loop as one CUDA-graph launch")

ENS_METRIC = "member solves/s to rtol 1e-8, 32 graded-mesh sequences as one block (ensemble path); %HBM peak"


def ensemble_main(args, wl, torch, pkg, dist, world, rank, local, dev, mesh, seed, rtol):
    """Ensemble workload: R sequences (seeds seed .. seed+R-1) advanced as one block by
    dd_solve_batch with one shared recycled basis; the single-sequence path solves some of
    the same sequences one at a time on the same GPU for the batching ratio."""
    R = wl["nrhs"]
    k = wl["k"]
    nsteps = args.warmup + args.steps
    t0 = time.perf_counter()
    seqs = [load_sequence(mesh, seed + j, nsteps) for j in range(R)]
    F_host = torch.from_numpy(np.ascontiguousarray(np.stack(seqs, axis=1)))  # [steps][R][n]
    del seqs
    t_rhs = time.perf_counter() - t0
    F_dev = F_host.to(dev)
    t0 = time.perf_counter()
    S = pkg.Solver(mesh, **solver_options(wl, True), ens_nmm=args.ens_nmm)
    setup_s = time.perf_counter() - t0
    hbm, peak_kind = peaks()
    X = torch.empty_like(F_dev[0])
    stream = torch.cuda.current_stream()

    def ens_run(prof):
        rec = S.ensemble_recycler(k, "B4")
        for t in range(args.warmup):
            S.solve_batch(F_dev[t], rec, rtol, out=X)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        S.profile(prof, read=True)  # resets the counters; prof: event timing (host-issued loop)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        stats = []
        torch.cuda.synchronize()
        e0.record(stream)
        for t in range(args.warmup, nsteps):
            _, st = S.solve_batch(F_dev[t], rec, rtol, out=X)
            stats.append(st)
        e1.record(stream)
        torch.cuda.synchronize()
        sec = max_over_ranks(torch, e0.elapsed_time(e1) / 1e3, dist, dev)
        pr = S.profile(False, read=True)
        rec.close()
        return sec, stats, pr

    with ClockSampler(local) as clk:
        sec, stats, (_, launches) = ens_run(False)
    clocks = clk.summary()
    prof_sec, prof_stats, (prof, _) = ens_run(True)
    assert [[m["iters"] for m in st] for st in prof_stats] == [[m["iters"] for m in st] for st in stats]
    value = args.steps * R * world / sec
    its = [m["iters"] for st in stats for m in st]

    # single-sequence path on the same GPU: the first few members, each with its own state
    n_single = min(4, R)
    tot = 0.0
    for j in range(n_single):
        r1 = S.recycler(k, "B4")
        x1 = torch.empty_like(F_dev[0, 0])
        for t in range(args.warmup):
            S.solve(F_dev[t, j].contiguous(), r1, rtol, out=x1)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        fs = [F_dev[t, j].contiguous() for t in range(args.warmup, nsteps)]
        a.record(stream)
        for f in fs:
            S.solve(f, r1, rtol, out=x1)
        b.record(stream)
        torch.cuda.synchronize()
        tot += a.elapsed_time(b) / 1e3
        r1.close()
    single = {"value": n_single * args.steps / tot, "unit": "solves/s", "members_timed": n_single,
              "options": "same solver and options, dd_solve per sequence with its own recycle state"}

    e2e = None
    if not args.no_e2e:
        Fp = F_host.pin_memory()
        rec2 = S.ensemble_recycler(k, "B4")
        pipe = CopyPipeline(torch, Fp, lambda f, x: S.solve_batch(f, rec2, rtol, out=x))
        pipe.run(0, args.warmup)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        pipe.run(args.warmup, nsteps, a)
        b.record(stream)
        torch.cuda.synchronize()
        esec = max_over_ranks(torch, a.elapsed_time(b) / 1e3, dist, dev)
        nb = int(F_host[0].numel()) * 8
        e2e = {"value": args.steps * R * world / esec, "unit": "solves/s", "h2d_bytes_per_step": nb,
               "d2h_bytes_per_step": nb}
        rec2.close()

    nn = prof["ens_N"]
    nn_ms = nn[0] / max(nn[1], 1)
    achieved = nn[2] / (nn_ms / 1e3) / 1e9 if nn[1] else None
    nmm_kernel = {1: "k_symm_b<float> (CUDA cores)", 2: "k_nmm_tc<TF32X3> (persistent, tcgen05 kind::tf32)",
                  3: "k_nmm_tc<BF16X3> (persistent, tcgen05 kind::f16, bf16 slices)"}.get(S.info["ens_nmm"], "none")
    roof = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
            "frac": (achieved / hbm) if achieved else None, "traffic": None,
            "kernel": f"{nmm_kernel}: ensemble constrained-Neumann products N_i R_i, eq. 9",
            "peak_kind": f"{peak_kind} hbm_gbs (burst copy)", "alg_bytes_per_launch": nn[2],
            "avg_launch_ms": nn_ms, "launches": nn[1], "timing": PROF_TIMING,
            "replay_ms_per_step": 1e3 * prof_sec / args.steps}
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = cpu_baseline(args, wl, args.cpu_baseline_steps)
    if rank == 0:
        per_kernel = kernel_table(prof, hbm, {2: "tf32", 3: "bf16"}.get(S.info["ens_nmm"]))
        line = {"metric": ENS_METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": 1e3 * sec / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64 (df64 Schur, f32 BDDC)", "data": "synthetic",
                "config": {"workload": args.workload, "n": wl["n"], "subdomains": (wl["n"] // wl["sub"]) ** 3,
                           "members": R, "levels": wl["levels"], "k": k, "strategy": "B4 (shared W from member 0)",
                           "rtol": rtol, "n_free": S.n_free, "n_gamma": S.n_gamma,
                           "l2": "members' vectors and operators exceed L2 (inputs larger than L2)",
                           "rhs_seeds": [seed, seed + R - 1]},
                "iters_min_max_avg": [min(its), max(its), sum(its) / len(its)],
                "setup_s": setup_s, "rhs_gen_s": t_rhs, "single_sequence": single,
                "ens_nmm": {"kernel": {1: "simt", 2: "tcgen05 3xTF32", 3: "tcgen05 BF16x3"}.get(S.info["ens_nmm"],
                                                                                                "none"),
                            "tuning_ms": S.info["ens_nmm_ms"]},
                "ens_shapes": {"element_members_per_pass": S.info["ens_elem_rc"],
                               "fdm_members_per_block": S.info["ens_fdm_rc"]},
                "batching_speedup": value / single["value"],
                "e2e": e2e, "roofline": roof, "cpu_baseline": cpu, "clocks": clocks,
                "gpu_launches": launches, "kernels": per_kernel}
        print(json.dumps(line), flush=True)
    S.close()
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def ablation(args, wl, torch, pkg, dev, mesh, seed, rtol):
    """What adaptivity (Sect. 3.3) and B4 recycling (Sect. 4.2) buy on this workload at equal
    precision (the mixed-precision path): {adaptive off, on} x {k = 0, k = wl k}, each with
    its own setup, W untimed and K timed steps of the same sequence. Reports iterations
    min-max(avg), ms per step, the largest retained harmonic Ritz value (an estimate of
    lambda_max(M^{-1} A); lambda_min >= 1 for BDDC) and the recycling updates timed."""
    nsteps = args.warmup + args.steps
    F_dev = torch.from_numpy(load_sequence(mesh, seed, nsteps)).to(dev)
    rows = []
    for adaptive in (0, 1):
        o = solver_options(dict(wl, adaptive=adaptive), True)
        t0 = time.perf_counter()
        S = pkg.Solver(mesh, **o)
        setup_s = time.perf_counter() - t0
        for k in (0, wl["k"]):
            keep = {}
            sec, stats, _ = run_arm(torch, S, F_dev, args.warmup, args.steps, k, "B4", rtol, 1, None,
                                    keep_state=keep)
            its = [st["iters"] for st in stats]
            th = keep["recycle"]["theta"]
            rows.append({"adaptive": bool(adaptive), "n_adaptive": S.info["n_adaptive"], "k": k,
                         "iters_min_max_avg": [min(its), max(its), sum(its) / len(its)],
                         "ms_per_step": 1e3 * sec / args.steps, "solves_per_s": args.steps / sec,
                         "theta_max": float(th.max()) if len(th) else None, "setup_s": setup_s})
        S.close()
    line = {"metric": "ablation: adaptive BDDC x B4 recycling at equal (mixed) precision", "workload": args.workload,
            "n": wl["n"], "steps": args.steps, "warmup": args.warmup, "rtol": rtol, "rows": rows}
    print(json.dumps(line), flush=True)


def tau_sweep(args, wl, torch, pkg, dev, mesh, seed, rtol):
    """The adaptivity study of Sect. 6 on this workload: the threshold tau of the face
    eigenproblems (eq. 10) in {2, 2.5, 3, 3.5} and the workload's own, with cardinality and
    diagonal-stiffness weights, each with B4 recycling (k of the workload) on the mixed-
    precision path; its own setup per row, W untimed and K timed steps of the same sequence.
    Reports the adaptive constraints, the coarse problem size, iterations min-max(avg), ms per
    step (time per iteration), setup seconds and the largest kept harmonic Ritz value."""
    nsteps = args.warmup + args.steps
    F_dev = torch.from_numpy(load_sequence(mesh, seed, nsteps)).to(dev)
    rows = []
    taus = sorted({2.0, 2.5, 3.0, 3.5, float(wl.get("tau", 10.0))})
    for weights in ("card", "diag"):
        for tau in taus:
            o = dict(solver_options(dict(wl, adaptive=1, tau=tau), True), weights=weights)
            t0 = time.perf_counter()
            S = pkg.Solver(mesh, **o)
            setup_s = time.perf_counter() - t0
            keep = {}
            sec, stats, _ = run_arm(torch, S, F_dev, args.warmup, args.steps, wl["k"], "B4", rtol, 1, None,
                                    keep_state=keep)
            its = [st["iters"] for st in stats]
            th = keep["recycle"]["theta"]
            rows.append({"weights": weights, "tau": tau, "n_adaptive": S.info["n_adaptive"],
                         "n_coarse": S.info["n_coarse"], "iters_min_max_avg": [min(its), max(its), sum(its) / len(its)],
                         "ms_per_step": 1e3 * sec / args.steps, "ms_per_iter": 1e3 * sec / sum(its),
                         "solves_per_s": args.steps / sec, "setup_s": setup_s,
                         "theta_max": float(th.max()) if len(th) else None})
            S.close()
    line = {"metric": "tau sweep: adaptive BDDC threshold x weights with B4 recycling (mixed precision)",
            "workload": args.workload, "n": wl["n"], "k": wl["k"], "steps": args.steps, "warmup": args.warmup,
            "rtol": rtol, "rows": rows}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    # 200 steps of the 500-step sequence: the recycling phase (until the Ritz values
    # freeze, a handful to a dozen steps) weighs as it does in a long sequence
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="graded128", choices=sorted(WORKLOADS))
    ap.add_argument("--no-plain", action="store_true", help="skip the plain FP64 arm")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-baseline-n", type=int, default=48,
                    help="elements per axis of the oracle's sample (the workload's n: the workload itself, "
                         "factored once, with the GPU solutions of the same steps compared)")
    ap.add_argument("--cpu-baseline-steps", type=int, default=3)
    ap.add_argument("--ablation", action="store_true",
                    help="print the adaptive x recycling table at equal precision instead of the bench line")
    ap.add_argument("--tau-sweep", action="store_true",
                    help="print the adaptivity threshold x weights table (Sect. 6) instead of the bench line")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--rtol", type=float, default=None)
    ap.add_argument("--ens-nmm", default="auto", choices=["auto", "simt", "tc", "bf16x3"],
                    help="ensemble N_i product kernel (default: timed on the first call)")
    ap.add_argument("--n", type=int, default=None,
                    help="elements per axis of a smaller member of the workload's mesh family (profiling runs)")
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
    mesh = workload_mesh(args.workload, n=args.n)
    if args.n is not None:
        wl = dict(wl, n=args.n)
    seed = rank_seed(wl, rank)
    if wl.get("nrhs"):
        return ensemble_main(args, wl, torch, pkg, dist, world, rank, local, dev, mesh, seed, rtol)
    if args.ablation:
        return ablation(args, wl, torch, pkg, dev, mesh, seed, rtol)
    if args.tau_sweep:
        return tau_sweep(args, wl, torch, pkg, dev, mesh, seed, rtol)
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
        sec, stats, (_, launches) = run_arm(torch, mixed, F_dev, args.warmup, args.steps, k, "B4", rtol, world, dist)
    clocks = clk.summary()
    # per-kernel device times: a replay of the same warm-up and timed steps with CUDA
    # events around every operator application (host-issued loop, identical iterates)
    keep = {}
    cap = set(range(args.warmup, args.warmup + min(args.cpu_baseline_steps, args.steps)))
    prof_sec, prof_stats, (prof, _) = run_arm(torch, mixed, F_dev, args.warmup, args.steps, k, "B4", rtol, world,
                                              dist, prof=True, capture=cap, keep_state=keep)
    assert [s["iters"] for s in prof_stats] == [s["iters"] for s in stats]
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
        esec, h2d, d2h = run_e2e(torch, mixed, Fp, args.warmup, args.steps, k, "B4", rtol, dist)
        e2e = {"value": args.steps * world / esec, "unit": "solves/s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h}

    # dominant kernel: the batched FP32 constrained-Neumann GEMV u_i = N_i r_i of BDDC
    # (HBM-bound: the packed N_i triangles stream once per application)
    nn = prof["symv_N"]
    nn_ms = nn[0] / max(nn[1], 1)
    achieved = nn[2] / (nn_ms / 1e3) / 1e9 if nn[1] else None
    # DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one launch of this kernel
    # on the default workload (128^3, 4096 subdomains), from an ncu capture of this bench:
    # 1131.25 MB read + 13.22 MB written against 1129.2 MB algorithmic; None elsewhere
    traffic = 1144475392.0 if args.workload == "graded128" and args.n is None else None
    roof = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
            "frac": (achieved / hbm) if achieved else None, "traffic": traffic,
            "kernel": "k_symv<FP32> (batched constrained-Neumann N_i GEMV, eq. 9)",
            "peak_kind": f"{peak_kind} hbm_gbs (burst copy)", "alg_bytes_per_launch": nn[2],
            "avg_launch_ms": nn_ms, "launches": nn[1], "timing": PROF_TIMING,
            "replay_ms_per_step": 1e3 * prof_sec / args.steps,
            "sharing": "in each BDDC application the coarse branch runs on a second stream beside this "
                       "kernel, so the launch time above includes that sharing of the SMs and of HBM"}
    # the same kernel alone: the setup's launch-shape tuning times back-to-back launches of it
    # on the context's own operators (1.13 GB per launch, larger than L2) for each ring depth
    tms = [t for t in mixed.info.get("tune_symv_ms", []) if t > 0]
    if tms and nn[2]:
        t_alone = min(tms)
        a_alone = nn[2] / (t_alone / 1e3) / 1e9
        roof["alone"] = {"avg_launch_ms": t_alone, "achieved": a_alone, "frac": a_alone / hbm,
                         "timing": "CUDA events around back-to-back launches at setup (the tuned ring depth)"}
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = cpu_baseline(args, wl, args.cpu_baseline_steps, keep.get("x"), args.warmup)

    if rank == 0:
        per_kernel = kernel_table(prof, hbm)
        rs = keep.get("recycle", {})
        recycle = {"k": rs.get("k"), "frozen": rs.get("frozen"),
                   "theta_max": float(max(rs["theta"])) if rs.get("theta") is not None and len(rs["theta"]) else None,
                   "theta_min": float(min(rs["theta"])) if rs.get("theta") is not None and len(rs["theta"]) else None,
                   "updates": per_kernel.get("recycle_update", {}).get("launches")}
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
                "frozen_at_end": bool(stats[-1]["frozen"]), "recycle": recycle,
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
