#!/usr/bin/env python3
"""Benchmark: PCG time-to-rtol with the Chebyshev polynomial preconditioner.

One step = one full solve A x = b to rtol 1e-8 (PCG, P = W p_k(W^T A W) W^T,
Algorithm 2 applied by fused SpMV+recurrence kernels) on a matrix already
set up and resident in HBM (seed scaling, SELL layout, Lanczos interval and
coefficients done once before timing).  Default workload: 3-D 7-point
variable-coefficient diffusion on a 192^3 grid, lognormal(0, 2)
conductivities (seed 1), harmonic faces, N(0,1) right-hand side, FP64,
SELL-C-sigma layout chosen by pp_autotune, k = 5 (the fastest degree of
the sweep k in {5, ..., 160}), 60 Lanczos steps, xi = clip(10 alpha/beta,
1e-6, 1e-2).

Prints one JSON line (rank 0).  `--impl reference` times the CPU oracle on a
bounded sample of the same workload instead.
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    # k = 5: the fastest degree of the FP64 sweep k in {5, 10, 20, 40, 80, 160}; the interval from 60
    # Lanczos steps (the fastest of the sweep 10, 30, 60, 100, 200 at k = 5)
    # (blocks of PCG iterations replayed as CUDA graphs: 2 % faster than launching them one by one)
    "diffusion192": dict(N=192, sigma=2.0, seed=1, rhs="normal", k=5, lanczos=60, fmt="sell", prec="f64", graphs=1),
    # the FP32 / BF16 applies make the degree steps cheap next to the FP64 outer iteration: k = 20 is the
    # fastest of the sweep
    "diffusion192_f32": dict(N=192, sigma=2.0, seed=1, rhs="normal", k=20, lanczos=60, fmt="sell", prec="f32",
                             flexible=1, graphs=1),
    "diffusion192_bf16": dict(N=192, sigma=2.0, seed=1, rhs="normal", k=20, lanczos=60, fmt="sell", prec="bf16",
                              flexible=1, graphs=1),
    "diffusion128": dict(N=128, sigma=2.0, seed=1, rhs="normal", k=5, lanczos=60, fmt="sell", prec="f64"),
    "diffusion128_f32": dict(N=128, sigma=2.0, seed=1, rhs="normal", k=5, lanczos=60, fmt="sell", prec="f32",
                             flexible=1),
    # 32^3 Poisson is L2-resident and launch-bound: 10-iteration blocks replayed as CUDA graphs
    "poisson32": dict(N=32, sigma=0.0, seed=0, rhs="ones_noise", k=20, lanczos=10, fmt="csr", prec="f64",
                      graphs=1, check_every=10),
    # fracture network: the time to rtol is flat over k = 1..7 (products dominate); k = 3 with a
    # 30-step Lanczos interval is the fastest measured setting.  Every fracture-network workload replays
    # its blocks of PCG iterations as CUDA graphs (4 % faster in FP64, 9 % with the FP32 preconditioner)
    "dfn200": dict(dfn=True, seed=2, k=3, lanczos=30, prec="f64"),
    # p_k(S_hat) with the FP32 copy of the trace blocks, outer FP64 FCG(1)
    "dfn200_f32": dict(dfn=True, seed=2, k=15, lanczos=30, prec="f32", flexible=1),
    # its first 40 fractures with the closed-form blocks: a small case of the S_u kernels for profiler captures
    "dfn40": dict(dfn=True, seed=2, n_f=40, k=3, lanczos=30, prec="f64"),
    "dfn40_f32": dict(dfn=True, seed=2, n_f=40, k=15, lanczos=30, prec="f32", flexible=1),
    # the same network with general fracture blocks (P1 stiffness on jittered triangulations,
    # lognormal coefficients): A^{-1} from banded Cholesky factors built on the GPU
    "dfn200_p1": dict(dfn=True, seed=2, k=3, lanczos=30, prec="f64", general="p1"),
    # its first 40 fractures (0.4M nodes): a small case of the same kernels for profiler captures
    "dfn40_p1": dict(dfn=True, seed=2, n_f=40, k=3, lanczos=30, prec="f64", general="p1"),
    # per-instance symmetric DIA in the batch (the instances are 7-point stencils)
    # layout chosen by pp_batch_autotune (per-instance DIA or the global SELL-32 slice list)
    "batched64": dict(batch=True, seed=4, count=64, k=20, lanczos=10, prec="f32", fmt="auto"),
}
METRIC = "PCG time-to-rtol-1e-8 (s) and polyprec_apply HBM GB/s vs plain FP64, 1 GB300"
VAL_BYTES = {"f64": 8, "f32": 4, "bf16": 2}
VEC_BYTES = {"f64": 8, "f32": 4, "bf16": 4}


def build_problem(w):
    from paper_2208_01339_gb300 import inputs as I

    if w.get("dfn"):
        net = I.fracture_network(n_f=w.get("n_f", 200), seed=w["seed"])
        if w.get("general") == "p1":
            net = I.general_fracture_network(net, shuffle=False)
        return net, None
    if w.get("batch"):
        specs = I.batch_specs(w["count"], seed=w["seed"], nmax=w.get("nmax", 160))
        return specs, None

    if w["sigma"] == 0.0:
        A = I.poisson3d(w["N"])
    else:
        A = I.diffusion3d(w["N"], w["sigma"], seed=w["seed"])
    if w["rhs"] == "normal":
        b = I.rhs_normal(A.n, w["seed"])
    else:
        b = I.rhs_ones_plus_noise(A, w["seed"])
    return A, b


def bytes_per_step_launch(nnz: int, n: int, k: int, prec: str, ndiag: int = 0) -> float:
    """Algorithmic bytes of one fused degree step, averaged over the k steps
    of one application: every step streams the matrix once -- value + int32
    column index per nonzero (CSR, SELL), or the ndiag stored diagonals of n
    values each (symmetric DIA: main and upper diagonals, no indices) -- and
    touches n-vectors: step 1 reads r and writes y (2), step 2 reads x, r
    and writes y (3; x_old = r/theta is not stored), steps 3..k read x,
    x_old, r and write y (4).  Gathered x entries and the lower-triangle
    rereads of DIA are counted once (L2 reuse); padding is excluded."""
    sa, sv = VAL_BYTES[prec], VEC_BYTES[prec]
    if k <= 0:
        return 0.0
    vec_passes = 2 if k == 1 else 2 + 3 + 4 * (k - 2)
    mat = ndiag * n * sa if ndiag else nnz * (sa + 4)
    return (k * mat + n * sv * vec_passes) / k


def flops_per_step_launch(nnz: int, n: int, k: int, ndiag: int = 0) -> float:
    """Algorithmic arithmetic of one fused degree step, averaged over the k
    steps: one multiply-add (2 flops) per nonzero of A x -- with the unit
    diagonal of the Jacobi-scaled DIA storage the diagonal term is the
    vector entry itself, so 2 (nnz - n) + n -- then per row 3 flops in the
    first step (y = ca r + cb A r) and 6 in the others (y = ca x + cb x_old
    + cc (r - A x)).  The count is the method's, independent of how a kernel
    folds the coefficients."""
    if k <= 0:
        return 0.0
    mat = 2.0 * nnz if not ndiag else 2.0 * (nnz - n) + n
    return mat + n * (3.0 + 6.0 * (k - 1)) / k


def fp64_peak_tflops() -> float:
    """152 SMs x 2 FP64 FMA per clock per SM (4 flop) x 2.07 GHz: the nominal
    1.25 TFLOP/s FP64 rate of GB300 expressed in unit counts and clocks."""
    return 152 * 4 * 2.07e9 / 1e12


# the sources of each captured kernel family (traffic is reported only while they are unchanged)
KERNEL_SOURCES = {
    "dia": ("common.cuh", "kernels.cuh", "step_impl.cuh", "step_dia.cuh", "step_dia.cu"),
    "dia_tma": ("common.cuh", "kernels.cuh", "step_impl.cuh", "step_dia.cuh", "step_dia_tma.cu"),
    "dia_z": ("common.cuh", "kernels.cuh", "step_impl.cuh", "step_dia.cuh", "step_dia_z.cu"),
    "sell": ("common.cuh", "kernels.cuh", "step_impl.cuh", "step_f64.cu", "step_lp.cu"),
}


def source_sha(files=KERNEL_SOURCES["dia"]) -> str:
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2208_01339_gb300", "csrc")
    for f in files:
        with open(os.path.join(d, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            j = json.load(fh)
        if j.get("hbm_gbs"):
            return float(j["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs, copy)"
    return 6800.0, "fallback (6.8 TB/s)"


def traffic_from_profile(workload: str, k: int, prec: str, layout: str):
    """DRAM bytes per step launch from an ncu capture of the same kernel
    sources, layout and degree (None when there is none)."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as fh:
        j = json.load(fh)
    e = j.get(f"{workload}/k{k}/{prec}")
    if not e or e.get("layout") != layout:
        return None
    if e.get("source_sha") != source_sha(KERNEL_SOURCES[e.get("family", "dia")]):
        return None
    return {"bytes": e.get("dram_bytes_per_launch"), "launch": e.get("kernel"),
            "algorithmic_bytes_same_launch": e.get("algorithmic_bytes_same_launch"), "from": e.get("captured_on")}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.proc = None
        self.path = os.path.join("/tmp", f"pp_clocks_{os.getpid()}.csv")
        self.gpu = gpu_index

    def __enter__(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-i", str(self.gpu), "-lms", "200"], stdout=self.fh,
                                         stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        with open(self.path) as fh:
            for ln in fh:
                parts = [p.strip() for p in ln.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def oracle_iterations(workload: str, k: int, lanczos_steps: int):
    p = os.path.join(ROOT, "tests", "golden", "oracle_iterations.json")
    if not os.path.exists(p):
        return None
    with open(p) as fh:
        table = json.load(fh)
    # the FP32/BF16 variants solve the same system; the oracle is FP64
    base = workload.replace("_f32", "").replace("_bf16", "")
    key = f"k{k}/L{lanczos_steps}"
    return table.get(f"{workload}/{key}", table.get(f"{base}/{key}"))


def cpu_solve(A, b, k, lanczos_steps, maxit=10000):
    """The oracle's solve on all host cores (the oracle's loops with OpenMP
    over rows, liboracle_omp.so): Jacobi seed, Lanczos interval from the
    shared start vector, xi = clip(10 alpha/beta, 1e-6, 1e-2), PCG from x = 0
    to rtol 1e-8 with p_k by Algorithm 2.  Returns (x, stats, setup s, PCG s,
    threads)."""
    import oracle as O

    from paper_2208_01339_gb300 import inputs as I

    x, st, t_setup, t_pcg = O.omp_solve(A, b, I.lanczos_start(A.n, 0), k, lanczos_steps, rtol=1e-8, maxit=maxit)
    return x, st, t_setup, t_pcg, O.omp_threads()


# reference arm: PCG iterations per timed step (a bounded sample of the solve)
REF_ITERS = 12


def run_reference(args, w, rank):
    """The oracle on the host cores, on the same workload and metric: each
    step runs the oracle's all-core solve for REF_ITERS PCG iterations (setup
    -- scaling, Lanczos, coefficients -- excluded like the GPU's), and the
    time to rtol is the median time per iteration times the oracle's own
    iteration count for this workload."""
    if rank != 0:
        return
    import oracle as O

    O.build()
    A, b = build_problem(w)
    k = args.k if args.k is not None else w["k"]
    iters = oracle_iterations(args.workload, k, w["lanczos"])
    src = "the oracle's own count, tests/golden/oracle_iterations.json"
    per_it = []
    threads = O.omp_threads()
    for i in range(args.warmup + args.steps):
        _, st, _, t_pcg, _ = cpu_solve(A, b, k, w["lanczos"], maxit=REF_ITERS)
        if i >= args.warmup:
            per_it.append(t_pcg / max(1, st["iterations"]))
    t_it = statistics.median(per_it)
    if iters is None:  # no stored count: run the full solve once for it
        _, st, _, _, _ = cpu_solve(A, b, k, w["lanczos"])
        iters, src = st["iterations"], "a full oracle solve in this run"
    value = t_it * iters
    sample = (f"{REF_ITERS} PCG iterations per step of the oracle's all-core solve (OpenMP over rows, "
              f"{threads} threads) on the full {A.n}-row workload, k = {k}; time to rtol = median seconds per "
              f"iteration x {iters} iterations ({src})")
    out = {"metric": METRIC, "value": value, "unit": "s", "n_gpus": args.gpus, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": t_it * REF_ITERS * 1e3, "higher_is_better": False,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
           "oracle_ms_per_iteration": t_it * 1e3,
           "config": {"workload": args.workload, "n": A.n, "nnz": A.nnz, "k": k, "lanczos_steps": w["lanczos"]},
           "cpu_baseline": {"value": value, "unit": "s", "cores": threads, "kind": "oracle", "sample": sample,
                            "extrapolation": f"x {iters / REF_ITERS:.1f} (iterations {iters} / {REF_ITERS} timed)"},
           "e2e": {"value": value, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def run_k_sweep(args, w, A, b, opts, dev):
    """Degree sweep: one line per k with the time to rtol and iterations."""
    import torch

    from paper_2208_01339_gb300 import polyprec as P

    bt = torch.as_tensor(b, device=dev)
    for k in [int(v) for v in args.k_sweep.split(",")]:
        o = dict(opts)
        o["k"] = k
        S = P.Solver.from_host(A, device=dev, **o)
        for _ in range(2):
            S.solve(bt)
        torch.cuda.synchronize(dev)
        ts = []
        for _ in range(max(1, args.steps)):
            x, st = S.solve(bt)
            ts.append(st["t_solve_ms"])
        apply_us = st["t_apply_ms"] / max(1, st["apply_launches"]) * 1e3
        info = S.info()
        print(json.dumps({"workload": args.workload, "prec": w["prec"], "poly": args.poly, "k": k,
                          "iterations": st["iterations"],
                          "time_s": statistics.median(ts) / 1e3, "mvp": st["mvp"], "dots": st["dots"],
                          "step_us": round(apply_us, 2), "status": st["status"], "lowrank": info["lowrank"],
                          "alpha_hat": info["alpha_hat"], "setup_ms": round(info["t_setup_ms"], 2),
                          "ritz_resid": info["ritz_resid"]}), flush=True)
        S.close()


def run_dfn_sweep(args, w, net, dopts, dev):
    """Degree sweep on the fracture network (the shape of Table 4): one line
    per k with iterations, products, inner products and time to rtol."""
    import torch

    from paper_2208_01339_gb300 import polyprec as P

    for k in [int(v) for v in args.k_sweep.split(",")]:
        S = P.SchurSolver(net, device=dev, k=k, **dopts)
        bt = S.rhs(torch.as_tensor(net.q, device=dev))
        S.solve(bt)
        torch.cuda.synchronize(dev)
        ts = []
        for _ in range(max(1, args.steps)):
            _, st = S.solve(bt)
            ts.append(st["t_solve_ms"])
        info = S.info()
        print(json.dumps({"workload": args.workload, "k": k, "poly": dopts["poly"], "lowrank": dopts["lowrank"],
                          "band_max": info["band_max"], "factor_ms": round(info["t_factor_ms"], 2),
                          "trace_blocks_ms": round(info["t_trace_ms"], 2),
                          "lanczos_steps": dopts["lanczos_steps"], "iterations": st["iterations"],
                          "time_s": statistics.median(ts) / 1e3, "mvp": st["mvp"], "dots": st["dots"],
                          "setup_ms": round(info["t_setup_ms"], 2), "alpha_hat": info["alpha_hat"],
                          "beta_hat": info["beta_hat"], "xi": info["xi"], "ritz_resid": info["ritz_resid"],
                          "status": st["status"]}), flush=True)
        S.close()


def batch_step_bytes(specs, fmt: str, prec: str) -> float:
    """Algorithmic bytes of one batched degree step over every column: each
    instance's matrix streamed once for all its right-hand sides (DIA: 3
    stored diagonals of n values; SELL: value + int32 index per nonzero),
    and per column the vectors x, x_old, r read and y written (the later
    steps' 4 passes)."""
    sv, sx = VAL_BYTES[prec], VEC_BYTES[prec]
    tot = 0.0
    for sp in specs:
        n = sp.N ** 3
        nnz = 7 * n - 6 * sp.N ** 2
        tot += (3 * n * sv if fmt == "dia" else nnz * (sv + 4)) + 4 * n * sp.nrhs * sx
    return tot


def batch_step_kernel(fmt: str, prec: str) -> str:
    if fmt != "dia":
        return "b_cheb_kernel"
    return "b_cheb_z_kernel (plane marching)" if prec == "f32" else "b_cheb_dia3_kernel"


def run_batch(args, w, specs, k, dev, world, rank, emit=True):
    """Config-5 shape: many uneven instances with several RHS each, solved by
    the batched solver (FP32 p_k, FP64 flexible CG, CUDA graphs) in the
    layout pp_batch_autotune picks and, for comparison, one column at a
    time by the plain FP64 single-instance solver.  With N ranks the
    instances are dealt to ranks by work (heaviest first, least-loaded
    rank) and each rank solves its share; no data crosses ranks."""
    import torch

    from paper_2208_01339_gb300 import inputs as I
    from paper_2208_01339_gb300 import learn as Lrn
    from paper_2208_01339_gb300 import polyprec as P
    from paper_2208_01339_gb300 import replicas

    all_specs = specs
    mine = replicas.shard_balanced([s.N ** 3 * s.nrhs for s in all_specs], rank, world)
    specs = [all_specs[i] for i in mine]
    mats = [I.batch_instance(s) for s in specs]
    rhs = [I.batch_rhs(s) for s in specs]
    nrhs = [s.nrhs for s in specs]
    common = dict(k=k, lanczos_steps=w["lanczos"], rtol=1e-8, apply_prec=w["prec"], flexible=1, use_graphs=1,
                  check_every=10, maxit=5000)
    fmt, tune = w.get("fmt", "auto"), None
    if fmt == "auto":
        fmt, table = P.batch_autotune(mats, nrhs, device=dev, **common)
        tune = [[t["format"], round(t["us_per_step"], 2)] for t in table if t["status"] == 0]
    S = P.BatchSolver(mats, nrhs, device=dev, format=fmt, **common)
    bt = S.pack(rhs)
    abx0 = S.intervals()
    cols = np.cumsum([0] + nrhs)
    base = np.array([abx0[cols[i], :2] for i in range(len(specs))])
    mlp_used = 0
    if os.path.exists(Lrn.WEIGHTS):
        model = Lrn.Model.load()
        ab, used = Lrn.predicted_intervals(model, S.features(), base, device=dev)
        abx_mlp = np.concatenate([np.repeat(ab[i:i + 1], nrhs[i], axis=0) for i in range(len(specs))])
        S.intervals(abx_mlp)
        mlp_used = int(used.sum())
    for _ in range(max(3, args.warmup)):
        S.solve(bt)
    replicas.barrier(dev)
    stream = torch.cuda.current_stream(dev)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    stats = []
    for _ in range(args.steps):
        x, it, stv, st = S.solve(bt)
        stats.append(st)
    ev1.record(stream)
    replicas.barrier(dev)
    ms = replicas.max_over_ranks(ev0.elapsed_time(ev1) / args.steps, dev)
    xs = S.unpack(x)
    it_mlp = it.copy()
    # the same batch with the Lanczos interval and the 10/kappa rule, and with
    # the most frequent sweep label as one constant setting (iterations only)
    arms = {}
    for name, abx in (("fallback", abx0),
                      ("fixed", np.column_stack([abx0[:, 0] * Lrn.FIXED_BEST[0], abx0[:, 1] * Lrn.FIXED_BEST[1],
                                                 np.full(len(abx0), Lrn.FIXED_BEST[2])]))):
        S.intervals(abx)
        _, ita, sta, _ = S.solve(bt)
        arms[name] = {"iterations_mean": float(ita.mean()), "iterations_max": int(ita.max()),
                      "converged": int((sta == 0).sum())}
    arms["mlp" if mlp_used else "mlp (not trained)"] = {"iterations_mean": float(it_mlp.mean()),
                                                       "iterations_max": int(it_mlp.max())}
    step_us = S.time_step(reps=5)
    bytes_step = batch_step_bytes(specs, fmt, w["prec"])
    peak, peak_src = measured_peak()
    S.close()
    del S
    # plain FP64 one column at a time (same k, Lanczos interval per instance)
    t_seq = 0.0
    err = 0.0
    its64 = []
    for i, (A, Bm) in enumerate(zip(mats, rhs)):
        S64 = P.Solver.from_host(A, device=dev, k=k, lanczos_steps=w["lanczos"], rtol=1e-8, seed=i, format="dia")
        for r in range(Bm.shape[1]):
            b = torch.as_tensor(np.ascontiguousarray(Bm[:, r]), device=dev)
            S64.solve(b)  # warm
            torch.cuda.synchronize(dev)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            x64, st64 = S64.solve(b)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            t_seq += e0.elapsed_time(e1) / 1e3
            its64.append(st64["iterations"])
            xr = x64.cpu().numpy()
            err = max(err, float(np.linalg.norm(xs[i][:, r] - xr) / np.linalg.norm(xr)))
        S64.close()
        del S64
    t_seq = replicas.max_over_ranks(t_seq, dev)
    err = replicas.max_over_ranks(err, dev)
    rows = sum(s.N ** 3 for s in all_specs)
    if rank == 0:
        ach = bytes_step / (step_us * 1e-6) / 1e9
        out = {"metric": METRIC, "value": ms / 1e3, "unit": "s", "n_gpus": world, "steps": args.steps,
               "warmup": max(3, args.warmup), "ms_per_step": ms, "higher_is_better": False, "scaling": "strong",
               "vs_baseline": None, "dtype": w["prec"], "data": "synthetic",
               "config": {"workload": args.workload, "instances": len(all_specs), "rows": rows,
                          "columns": int(sum(s.nrhs for s in all_specs)), "k": k, "apply": w["prec"],
                          "outer": "f64 flexible CG", "graphs": 1, "interval": f"mlp ({mlp_used} instances)"
                          if mlp_used else "lanczos", "layout": fmt,
                          "autotune": ("pp_batch_autotune [format(2 SELL-32, 3 DIA), us/step] " + json.dumps(tune))
                          if tune else "off",
                          "ranks": f"{world} (instances dealt by work, heaviest first)",
                          "sequential_baseline": "each column alone, plain FP64 PCG, DIA, Lanczos interval"},
               "iterations_max": int(max(stats[-1]["iterations"], 0)),
               "sequential_f64_s": t_seq, "speedup_vs_sequential_f64": t_seq / (ms / 1e3),
               "max_rel_diff_vs_f64": err, "iterations_f64_max": int(max(its64)),
               "interval_arms": arms,
               "roofline": {"bound": "hbm", "kernel": f"{batch_step_kernel(fmt, w['prec'])} ({w['prec']}, {fmt}), one degree step "
                                                      f"over every column (rank 0's share)",
                            "achieved": round(ach, 1), "peak": peak, "unit": "GB/s", "frac": round(ach / peak, 4),
                            "traffic": None, "peak_source": peak_src, "avg_launch_us": round(step_us, 2),
                            "algorithmic_bytes_per_launch": int(bytes_step)},
               "gpu_launches": int(sum(s["kernel_launches"] for s in stats))}
        if emit:
            print(json.dumps(out), flush=True)
        return out
    return None


def batch_summary(args, dev):
    """The batched workload (64 uneven instances, FP32 p_k, MLP intervals,
    one graph-replayed solve) measured inside the default line: its time to
    rtol 1e-8 against the plain FP64 solver run on every column alone, the
    interval arms and the step roofline.  One timed solve after 3 warm-ups."""
    w = dict(WORKLOADS["batched64"])
    specs, _ = build_problem(w)
    sub = argparse.Namespace(**{**vars(args), "steps": 1, "warmup": 3})
    out = run_batch(sub, w, specs, w["k"], dev, 1, 0, emit=False)
    keys = ("value", "sequential_f64_s", "speedup_vs_sequential_f64", "max_rel_diff_vs_f64", "iterations_max",
            "iterations_f64_max", "interval_arms", "roofline")
    res = {k2: out[k2] for k2 in keys}
    res["time_s"] = res.pop("value")
    res["config"] = {k2: out["config"][k2] for k2 in ("instances", "rows", "columns", "k", "apply", "outer",
                                                       "interval", "layout", "autotune", "sequential_baseline")}
    res["steps_timed"] = 1
    return res


def run_dfn(args, w, net, S, bt, k, dev, world, rank, dist):
    """Fracture-network Schur complement: PCG on S_hat to rtol 1e-8."""
    import torch

    from paper_2208_01339_gb300 import polyprec as P_

    info = S.info()
    for _ in range(max(3, args.warmup)):
        S.solve(bt)
    torch.cuda.synchronize(dev)
    stream = torch.cuda.current_stream(dev)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stats = []
    ev0.record(stream)
    for _ in range(args.steps):
        _, st = S.solve(bt)
        stats.append(st)
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    ms = ev0.elapsed_time(ev1) / args.steps
    it = int(statistics.median(s["iterations"] for s in stats))
    # the right-hand side (one full A^{-1} solve) and the recovery of h and p
    # (two), timed separately: they sit outside the iteration
    qd = torch.as_tensor(net.q, device=dev)
    u, _ = S.solve(bt)
    reps = 3
    torch.cuda.synchronize(dev)
    ev0.record(stream)
    for _ in range(reps):
        S.rhs(qd)
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    rhs_ms = ev0.elapsed_time(ev1) / reps
    ev0.record(stream)
    for _ in range(reps):
        S.recover(qd, u)
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    recover_ms = ev0.elapsed_time(ev1) / reps
    # one S_u product timed alone: the trace blocks M are streamed twice (t = M v,
    # then M (G^h t - alpha z)), one FMA per entry each time
    m_bytes = info["nnz"] * 8
    xr = torch.as_tensor(np.random.default_rng(0).standard_normal(net.n_u), device=dev)
    yr = torch.empty_like(xr)
    for _ in range(3):
        S.schur_apply(xr, yr)
    reps = 20
    torch.cuda.synchronize(dev)
    ev0.record(stream)
    for _ in range(reps):
        S.schur_apply(xr, yr)
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    prod_s = ev0.elapsed_time(ev1) / reps / 1e3
    fp64_peak = P_.fp64_fma_rate(reps=3)
    peak_bw, peak_src = measured_peak()
    prod_bytes = 2.0 * m_bytes
    prod_flops = 4.0 * info["nnz"]
    apply_ms = sum(s["t_apply_ms"] for s in stats) / max(1, sum(s["apply_launches"] for s in stats))
    if w["prec"] == "f32":
        # the preconditioner's products use the FP32 copy of M: bound by HBM
        b32 = 2.0 * info["nnz"] * 4
        ach = b32 / (apply_ms * 1e-3) / 1e9
        roof32 = {"bound": "hbm", "kernel": "S_hat product inside p_k: 2 x m_apply_kernel (FP32 trace blocks) + 3 "
                                            "sparse trace kernels", "achieved": round(ach, 1), "peak": peak_bw,
                  "unit": "GB/s", "frac": round(ach / peak_bw, 4), "peak_source": peak_src, "traffic": None,
                  "algorithmic_bytes_per_product": int(b32), "avg_product_us": round(apply_ms * 1e3, 2)}
    roof = {"bound": "alu", "kernel": "S_u product: 2 x m_apply_kernel (FP64 trace blocks) + 3 sparse trace kernels",
            "achieved": round(prod_flops / prod_s / 1e12, 4), "unit": "TFLOP/s",
            "peak": round(fp64_peak, 4) if fp64_peak else None,
            "frac": round(prod_flops / prod_s / 1e12 / fp64_peak, 4) if fp64_peak else None,
            "peak_source": "measured in this run: pp_fp64_fma_rate", "traffic": None,
            "algorithmic_flops_per_product": int(prod_flops), "avg_product_us": round(prod_s * 1e6, 2),
            "hbm": {"achieved": round(prod_bytes / prod_s / 1e9, 1), "peak": peak_bw, "unit": "GB/s",
                    "frac": round(prod_bytes / prod_s / 1e9 / peak_bw, 4), "peak_source": peak_src,
                    "algorithmic_bytes_per_product": int(prod_bytes)}}
    if rank == 0:
        out = {"metric": METRIC, "value": ms / 1e3, "unit": "s", "n_gpus": world, "steps": args.steps,
               "warmup": max(3, args.warmup), "ms_per_step": ms, "higher_is_better": False, "scaling": "weak",
               "vs_baseline": None, "dtype": w["prec"], "data": "synthetic",
               "config": {"workload": args.workload, "n_f": net.n_f, "n_h": net.n_h, "n_u": net.n_u, "k": k,
                          "trace_block_entries": info["nnz"], "alpha_reg": net.alpha,
                          "lanczos_steps": w["lanczos"], "lowrank": args.lowrank,
                          "a_inverse": ("banded Cholesky per fracture" if info["band_max"] else
                                        "closed form (uniform rectangles)"),
                          "band_max": info["band_max"], "band_doubles": info["band_elems"]},
               "factor_ms": round(info["t_factor_ms"], 2), "trace_blocks_ms": round(info["t_trace_ms"], 2),
               "rhs_ms": round(rhs_ms, 3), "recover_ms": round(recover_ms, 3),
               "iterations": it, "setup_ms": round(info["t_setup_ms"], 2), "alpha_hat": info["alpha_hat"],
               "beta_hat": info["beta_hat"], "xi": info["xi"],
               "apply_ms": apply_ms,
               "trace_block_bytes": m_bytes, "roofline": roof32 if w["prec"] == "f32" else roof,
               "operator_roofline": roof if w["prec"] == "f32" else None,
               "gpu_launches": int(sum(s["kernel_launches"] for s in stats))}
        print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="diffusion192", choices=list(WORKLOADS))
    ap.add_argument("--k", type=int, default=None)
    ap.add_argument("--graphs", type=int, default=-1, help="CUDA graphs for PCG blocks (default: per workload)")
    ap.add_argument("--sell-variant", type=int, default=0,
                    help="0 auto, 1 direct loads, 2 TMA-staged, 3 plane marching (FP32/BF16 DIA)")
    ap.add_argument("--sell-C", type=int, default=0)
    ap.add_argument("--sell-sigma", type=int, default=0)
    ap.add_argument("--check-every", type=int, default=0, help="PCG iterations per host check (default: per workload)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-batch", action="store_true",
                    help="leave the batched workload's summary out of the default line")
    ap.add_argument("--no-variants", action="store_true",
                    help="skip the FP32/BF16 and k = 80 comparison solves of the default workload")
    ap.add_argument("--k-sweep", default="", help="comma-separated degrees: time one solve per degree instead")
    ap.add_argument("--batch-count", type=int, default=0, help="override the batched workload's instance count")
    ap.add_argument("--batch-nmax", type=int, default=0, help="override the batched workload's largest grid")
    ap.add_argument("--lowrank", type=int, default=0,
                    help="Section 3.1 low-rank correction with this many Ritz vectors (0: none)")
    ap.add_argument("--lanczos-steps", type=int, default=0, help="override the workload's Lanczos steps")
    ap.add_argument("--poly", default="cheb", choices=["cheb", "newton"],
                    help="Algorithm 2 (three-term recurrence) or Algorithm 1 (Newton form, k = 2^nlev - 1)")
    ap.add_argument("--flexible", type=int, default=-1,
                    help="outer iteration: 0 PCG, 1 FCG(1), m >= 2 FCG(m) (default: per workload)")
    ap.add_argument("--format", default="", choices=["", "csr", "sell", "dia"],
                    help="force the step storage (skips pp_autotune)")
    ap.add_argument("--grid", type=int, default=0, help="override the grid size N of a diffusion workload "
                                                        "(smaller cases for profiler captures)")
    ap.add_argument("--general", action="store_true",
                    help="fracture networks: pass A and use the banded Cholesky factors even for rectangles")
    ap.add_argument("--no-autotune", action="store_true",
                    help="skip pp_autotune (layout from --sell-C/--sell-sigma/--sell-variant or the defaults)")
    args = ap.parse_args()
    w = dict(WORKLOADS[args.workload])
    if args.batch_count:
        w["count"] = args.batch_count
    if args.batch_nmax:
        w["nmax"] = args.batch_nmax
    if args.lanczos_steps:
        w["lanczos"] = args.lanczos_steps
    if args.flexible >= 0:
        w["flexible"] = args.flexible
    if args.grid and "N" in w:
        w["N"] = args.grid
    if args.format:
        w["fmt"] = args.format

    from paper_2208_01339_gb300 import replicas

    rank, world, local = replicas.rank_env()
    if args.impl == "reference":
        run_reference(args, w, rank)
        return

    import torch

    dist = None
    if world > 1:
        import torch.distributed as dist  # noqa: PLC0415

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device(f"cuda:{local}")
    torch.cuda.set_device(dev)
    from paper_2208_01339_gb300 import build as B
    from paper_2208_01339_gb300 import polyprec as P

    B.build()
    A, b = build_problem(w)
    k = args.k if args.k is not None else w["k"]
    if w.get("batch"):
        return run_batch(args, w, A, k, dev, world, rank)
    if w.get("dfn"):
        net = A
        dopts = dict(lanczos_steps=w["lanczos"], rtol=1e-8, check_every=args.check_every or 8,
                     use_graphs=args.graphs if args.graphs >= 0 else w.get("graphs", 1), apply_prec=w["prec"],
                     flexible=w.get("flexible", 0),
                     maxit=5000, lowrank=args.lowrank, poly=args.poly, sell_variant=args.sell_variant)
        dopts["general"] = True if args.general else None
        if args.k_sweep:
            return run_dfn_sweep(args, w, net, dopts, dev)
        S = P.SchurSolver(net, device=dev, k=k, **dopts)
        bt = S.rhs(torch.as_tensor(net.q, device=dev))
        return run_dfn(args, w, net, S, bt, k, dev, world, rank, dist)
    graphs = args.graphs if args.graphs >= 0 else w.get("graphs", 0)
    check_every = args.check_every if args.check_every > 0 else w.get("check_every", 8)
    opts = dict(k=k, lanczos_steps=w["lanczos"], format=w["fmt"], apply_prec=w["prec"], rtol=1e-8,
                check_every=check_every, use_graphs=graphs, flexible=w.get("flexible", 0),
                sell_variant=args.sell_variant, sell_C=args.sell_C, sell_sigma=args.sell_sigma, lowrank=args.lowrank,
                poly=args.poly)
    rp, ci, va = P.to_device_csr(A, dev)
    tune = None
    if not args.no_autotune and not args.format and w["fmt"] == "sell":
        # untimed setup: choose the step storage by timing every layout
        chosen, table = P.autotune(rp, ci, va, A.n, **opts)
        opts.update({key: chosen[key] for key in ("format", "sell_C", "sell_sigma", "sell_variant")})
        tune = [[t["format"], t["sell_C"], t["sell_sigma"], t["sell_variant"], round(t["us_per_step"], 2)]
                for t in table if t["status"] == 0]
    if args.k_sweep:
        return run_k_sweep(args, w, A, b, opts, dev)
    S = P.Solver(rp, ci, va, A.n, **opts)
    variant = opts.get("sell_variant", 0)
    info = S.info()
    bt = torch.as_tensor(b, device=dev)
    x = torch.zeros_like(bt)
    stream = torch.cuda.current_stream(dev)

    def barrier():
        replicas.barrier(dev)

    for _ in range(max(3, args.warmup)):
        S.solve(bt, x)
    barrier()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    stats = []
    with ClockSampler(int(os.environ.get("CUDA_VISIBLE_DEVICES", str(local)).split(",")[0] or 0)) as clk:
        barrier()
        ev0.record(stream)
        for _ in range(args.steps):
            _, st = S.solve(bt, x)
            stats.append(st)
        ev1.record(stream)
        barrier()
    clocks = clk.summary()
    ms = replicas.max_over_ranks(ev0.elapsed_time(ev1) / args.steps, dev)

    # end to end: pinned host b -> device, solve, device -> pinned host x
    e2e = None
    if not args.no_e2e:
        hb = torch.empty(A.n, dtype=torch.float64, pin_memory=True)
        hb.copy_(torch.as_tensor(b))
        hx = torch.empty(A.n, dtype=torch.float64, pin_memory=True)
        db = torch.empty_like(bt)
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            db.copy_(hb, non_blocking=True)
            xs, _ = S.solve(db)
            hx.copy_(xs, non_blocking=True)
        e1.record(stream)
        barrier()
        e_ms = replicas.max_over_ranks(e0.elapsed_time(e1) / args.steps, dev)
        e2e = {"value": e_ms / 1e3, "unit": "s", "h2d_bytes_per_step": A.n * 8, "d2h_bytes_per_step": A.n * 8}

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return

    it = [s["iterations"] for s in stats]
    fmt_name = {1: "CSR", 2: "SELL", 3: "DIA"}[info["format"]]
    layout = layout_name(info, variant, w["prec"])
    fp64_peak = None
    if w["prec"] == "f64" or not args.no_variants:
        fp64_peak = P.fp64_fma_rate(reps=5)
    roof = step_roofline(info, stats, A, k, w["prec"], args.workload, variant, fp64_peak)

    # one-shot time to solution: setup (layout, seed scaling, Lanczos,
    # coefficients) plus one solve, wall clock, on a fresh context
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    S1 = P.Solver(rp, ci, va, A.n, **opts)
    x1, _ = S1.solve(bt)
    torch.cuda.synchronize(dev)
    one_shot = time.perf_counter() - t0
    S1.close()
    del S1, x1

    cpu, err, x_oracle = None, None, None
    xg = x.cpu().numpy()
    if not args.no_cpu_baseline and world == 1:
        import oracle as O

        O.build()
        x_oracle, st_o, t_setup_o, t_pcg_o, threads = cpu_solve(A, b, k, w["lanczos"])
        cpu = {"value": t_pcg_o, "unit": "s", "cores": threads, "kind": "oracle",
               "sample": f"the whole workload: one full solve to rtol 1e-8 ({st_o['iterations']} iterations) by the "
                         f"oracle's loops with OpenMP over rows on {threads} host threads; setup (scaling, "
                         f"{w['lanczos']} Lanczos steps, coefficients: {t_setup_o:.2f} s) excluded like the GPU's; "
                         f"no extrapolation",
               "iterations": st_o["iterations"], "setup_s": round(t_setup_o, 3)}
        err = solution_error(xg, x_oracle, int(statistics.median(it)), st_o["iterations"])

    variants = None
    if not args.no_variants and args.workload == "diffusion192":
        variants = run_variants(args, A, rp, ci, va, bt, opts, x_oracle, fp64_peak, ms / 1e3, dev)
    batched = None
    if not args.no_batch and args.workload == "diffusion192" and world == 1:
        S.close()
        del S
        batched = batch_summary(args, dev)

    out = {
        "metric": METRIC, "value": ms / 1e3, "unit": "s", "n_gpus": world, "steps": args.steps,
        "warmup": max(3, args.warmup), "ms_per_step": ms, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": w["prec"], "data": "synthetic",
        "config": {"workload": args.workload, "grid": f"{w['N']}^3", "n": A.n, "nnz": A.nnz, "k": k,
                   "sigma_ln": w["sigma"], "format": fmt_name,
                   "lanczos_steps": w["lanczos"], "rtol": 1e-8,
                   "l2": "inputs larger than L2 (matrix >> 129 MB)" if A.nnz * 12 > 129e6 else "L2-resident inputs",
                   "graphs": graphs, "check_every": check_every, "layout": layout,
                   "outer": {0: "PCG", 1: "FCG(1)"}.get(w.get("flexible", 0), f"FCG({w.get('flexible', 0)})"),
                   "autotune": ("pp_autotune: [format(1 CSR, 2 SELL, 3 DIA), C, sigma, variant(1 direct, 2 TMA), "
                                "us/step] " + json.dumps(tune)) if tune else "off",
                   "lowrank": args.lowrank,
                   "parallelism": f"replicas x{world}"},
        "iterations": int(statistics.median(it)), "setup_ms": round(info["t_setup_ms"], 2),
        "one_shot_s": round(one_shot, 4),
        "alpha_hat": info["alpha_hat"], "beta_hat": info["beta_hat"], "xi": info["xi"],
        "err_vs_oracle": err, "roofline": roof, "cpu_baseline": cpu, "e2e": e2e,
        "north_star": variants, "batched": batched,
        "gpu_launches": int(sum(s["kernel_launches"] for s in stats)), "clocks": clocks,
    }
    print(json.dumps(out), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def layout_name(info, variant, prec="f64") -> str:
    if info["format"] == 2:
        return f"SELL C={info['sell_C']} sigma={info['sell_sigma']} {'direct' if variant == 1 else 'tma'}"
    if info["format"] == 3:
        return f"DIA ndiag={info['ndiag']}" + ({2: " tma", 3: " z-march"}.get(variant, "") if prec != "f64" else "")
    return "CSR"


def solution_error(xg, xo, it_gpu, it_oracle):
    """Relative 2-norm and per-element (scaled by max |x|) difference of the
    GPU solution from the oracle's, both solved to rtol 1e-8."""
    d = np.asarray(xg) - np.asarray(xo)
    return {"rel_2norm": float(np.linalg.norm(d) / np.linalg.norm(xo)),
            "rel_max_elem": float(np.max(np.abs(d)) / np.max(np.abs(xo))),
            "iterations_gpu": int(it_gpu), "iterations_oracle": int(it_oracle),
            "oracle": "the oracle's all-core FP64 solve of the same system to the same rtol"}


def step_roofline(info, stats, A, k, prec, workload, variant, fp64_peak):
    """Roofline of the dominant kernel, the fused degree step: algorithmic
    bytes (or flops) per launch over its average launch time, both from the
    solves' own CUDA-event records of the step launches."""
    t_apply = sum(s["t_apply_ms"] for s in stats)
    n_launch = sum(s["apply_launches"] for s in stats)
    if n_launch <= 0 or t_apply <= 0:
        return None
    bpl = bytes_per_step_launch(A.nnz, A.n, k, prec, info["ndiag"] if info["format"] == 3 else 0)
    avg_s = t_apply / 1e3 / n_launch
    peak, peak_src = measured_peak()
    ach = bpl / avg_s / 1e9
    layout = layout_name(info, variant, prec)
    dia_kind = {2: "tma_", 3: "z_"}.get(variant, "") if prec != "f64" else ""
    kname = {2: f"sell_step_{'tma_' if variant != 1 else ''}kernel ({prec}, C={info['sell_C']})",
             3: f"dia_step_{dia_kind}kernel ({prec}, {info['ndiag']} stored diagonals)",
             1: f"csr_step_kernel ({prec})"}[info["format"]]
    tr = traffic_from_profile(workload, k, prec, layout)
    hbm = {"bound": "hbm", "achieved": round(ach, 1), "peak": peak, "unit": "GB/s", "frac": round(ach / peak, 4),
           "traffic": tr["bytes"] if tr else None, "traffic_of": tr, "peak_source": peak_src,
           "kernel": kname, "algorithmic_bytes_per_launch": int(bpl), "avg_launch_us": round(avg_s * 1e6, 2)}
    if prec != "f64":
        return hbm
    # FP64 arithmetic is scarce on GB300: the FP64 step is bound by the FP64
    # pipe before HBM (ncu: FP64 pipe ~90% busy, DRAM ~45%)
    fl = flops_per_step_launch(A.nnz, A.n, k, info["ndiag"] if info["format"] == 3 else 0)
    tf = fl / avg_s / 1e12
    pk = fp64_peak if fp64_peak else fp64_peak_tflops()
    return {"bound": "alu", "achieved": round(tf, 4), "peak": round(pk, 4), "unit": "TFLOP/s",
            "frac": round(tf / pk, 4), "traffic": hbm["traffic"], "traffic_of": hbm["traffic_of"],
            "peak_source": ("measured in this run: pp_fp64_fma_rate (independent DFMA chains on every SM, CUDA "
                            "events)" if fp64_peak else "derived: 152 SMs x 4 FP64 flop/clk x 2.07 GHz"),
            "peak_derived": round(fp64_peak_tflops(), 4), "frac_of_derived": round(tf / fp64_peak_tflops(), 4),
            "kernel": kname, "algorithmic_flops_per_launch": int(fl), "avg_launch_us": hbm["avg_launch_us"],
            "hbm": {k2: hbm[k2] for k2 in ("achieved", "peak", "unit", "frac", "peak_source",
                                          "algorithmic_bytes_per_launch")}}


# The precision variant and the paper's degree range on the same system:
# (name, apply precision, degree, outer iteration: 0 PCG, 1 FCG(1))
VARIANTS = [("f32_k20", "f32", 20, 1), ("bf16_k20", "bf16", 20, 1), ("f64_k80", "f64", 80, 0),
            ("f32_k80", "f32", 80, 1), ("bf16_k80", "bf16", 80, 1)]


def run_variants(args, A, rp, ci, va, bt, opts, x_oracle, fp64_peak, fp64_s, dev):
    """Time to rtol 1e-8 of the FP32/BF16 applications of p_k inside FP64
    flexible CG, and of FP64 at k = 80, on the same matrix, right-hand side
    and layout as the FP64 line: the comparison the method's precision
    variant is judged by (faster than plain FP64 on the same GPU)."""
    import torch

    from paper_2208_01339_gb300 import polyprec as P

    stream = torch.cuda.current_stream(dev)
    out = []
    reps = max(3, min(args.steps, 10))
    # the step storage of each apply precision, chosen by pp_autotune in that precision
    layouts = {"f64": {key: opts[key] for key in ("format", "sell_C", "sell_sigma", "sell_variant")}}
    for prec in sorted({v[1] for v in VARIANTS} - {"f64"}):
        chosen, _ = P.autotune(rp, ci, va, A.n, **dict(opts, apply_prec=prec, k=20))
        layouts[prec] = {key: chosen[key] for key in ("format", "sell_C", "sell_sigma", "sell_variant")}
    for name, prec, kk, flex in VARIANTS:
        o = dict(opts, apply_prec=prec, k=kk, flexible=flex, **layouts[prec])
        S = P.Solver(rp, ci, va, A.n, **o)
        info = S.info()
        x = torch.zeros_like(bt)
        for _ in range(3):
            S.solve(bt, x)
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        stats = []
        e0.record(stream)
        for _ in range(reps):
            _, st = S.solve(bt, x)
            stats.append(st)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        t = e0.elapsed_time(e1) / reps / 1e3
        roof = step_roofline(info, stats, A, kk, prec, f"diffusion192{'' if prec == 'f64' else '_' + prec}",
                             o.get("sell_variant", 0), fp64_peak)
        ent = {"name": name, "apply": prec, "k": kk, "outer": "FCG(1)" if flex else "PCG",
               "layout": layout_name(info, o.get("sell_variant", 0), prec), "time_s": round(t, 5),
               "iterations": int(stats[-1]["iterations"]), "rel_res": stats[-1]["rel_res"],
               "speedup_vs_fp64_k5": round(fp64_s / t, 3), "steps_timed": reps,
               "step_roofline": {kk2: roof[kk2] for kk2 in ("bound", "achieved", "peak", "unit", "frac",
                                                           "avg_launch_us", "traffic")} if roof else None}
        if x_oracle is not None:
            xv = x.cpu().numpy()
            d = xv - x_oracle
            ent["err_vs_oracle"] = {"rel_2norm": float(np.linalg.norm(d) / np.linalg.norm(x_oracle)),
                                    "rel_max_elem": float(np.max(np.abs(d)) / np.max(np.abs(x_oracle)))}
        out.append(ent)
        S.close()
        del S
    t64_80 = next(e["time_s"] for e in out if e["name"] == "f64_k80")
    for e in out:
        if e["k"] == 80 and e["apply"] != "f64":
            e["speedup_vs_fp64_k80"] = round(t64_80 / e["time_s"], 3)
    best = min(out, key=lambda e: e["time_s"])
    return {"fp64_k5_s": round(fp64_s, 5), "variants": out, "fastest": best["name"],
            "fastest_speedup_vs_fp64": round(fp64_s / best["time_s"], 3),
            "note": "same matrix, right-hand side, Lanczos interval length and layout; FP64 outer iteration, "
                    "dots and residuals in every variant; err_vs_oracle against the oracle's FP64 solution"}


if __name__ == "__main__":
    main()
