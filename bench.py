"""Benchmark: SIS solves/s of the batched plates workload on GB300 (one JSON line).

Workload (default "plates32x8"): eight steady problems of Sec. 2.4 solved together --
delta in {0.1, 1, 10, 100} x {Poiseuille, thermal transpiration}, 32^3 velocity grid on
[-6, 6]^3, 100 sections on the clustered node map, M = 32 directions, SIS with
N = nu_bar/delta, stopped when the flow rates change by less than eps per iteration.
One step = one batched solve of all eight problems to convergence (every hot-path step,
A1-A8, runs on every iteration).  Inputs are synthetic (the problem parameters; h starts
at 0).  Working set: 808 cells x 32^3 x 4 B per array (106 MB) over several arrays, plus
the 134 MB of tensor-core operator blocks, well above L2 (129 MB).

  value     solves/s of one batched solve per step (BF16-refined: lbe_solve_batch; FP32 / FP64:
            the resident batch, lbe_batch_run), CUDA events on the calling stream
  e2e       solves/s through the one-shot public call lbe_solve_batch (host problems in,
            host results out; setup, uploads and convergence-flag reads inside)
  roofline  the tensor-core GEMM of the collision operator (A1-A3), timed alone by the library
            with CUDA events on its own stream at the same size: the method's algorithmic
            flops (FFT-equivalent) over its duration, executed flops beside them
  roofline_sweep  the transport sweep (A5) of an FP32 solve of the workload, every launch
            timed by the library: algorithmic bytes over duration against HBM
  fp64_gpu  the plain FP64 GPU path at the same eps (the comparison the mixed precision beats)
  duct64x32 the 64 x 32 duct (2048 cells, 32^3) solved in the same precision
  serving   the 256-request serving stream: saturated solves/s and p50 / p99 latency with
            Poisson arrivals (the line's latency_ms)
  autotuner the launch choices measured at first use
  cpu_baseline  the FP64 oracle on a bounded sample of the same workload (extrapolated), on
            one core and on all host cores

--workload mix_ne_ar24: the binary-mixture line (Ne-Ar plates, Table 4's setting: FP64, double-float
and BF16-refined solves, the square duct and the porous cell).  --workload mix_porous100: the
mixture in the periodic unit cell of a square array of cylinders (100 x 100 cells, porosity 0.6,
delta in {1, 10}, BF16-refined), with the tensor-core GEMM of its operator against the bf16 peak.

--impl reference times the oracle instead (the reference arm of this repository).
Multi-GPU: replicas only (independent solves per rank), launched by torchrun.
"""
import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

PEAKS_FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                  "sm_max_mhz": 2070.0}


PRECISIONS = {"fp32": lambda L: L.FP32, "fp64": lambda L: L.FP64, "bf16": lambda L: L.BF16_REFINED,
              "fp32r": lambda L: L.FP32_REFINED, "df32": lambda L: L.DF32}
DTYPES = {"fp32": "f32", "fp64": "f64", "bf16": "bf16/f32 inner + f64 residual",
          "fp32r": "f32 inner + f64 residual", "df32": "f32 pairs (operator only)"}


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        d["_source"] = "measured"
        return d
    d = dict(PEAKS_FALLBACK)
    d["_source"] = "fallback"
    return d


def workload_problems(lbe, name, precision, eps):
    from paper_1612_04488_gb300 import workloads as W
    if name == "plates32x8":
        kw = W.PLATES_32
        return [lbe.problem(**kw, delta=d, forcing=f, scheme=lbe.SIS, precision=precision, eps=eps,
                            max_iter=400)
                for d in W.PLATES_32_DELTAS for f in (0, 1)]
    if name == "plates16":
        return [lbe.problem(**W.PLATES_16, scheme=lbe.SIS, precision=precision, eps=eps, max_iter=400)]
    if name == "duct64x32":
        return [lbe.problem(**W.DUCT_64x32, scheme=lbe.SIS, precision=precision, eps=eps, max_iter=400)]
    raise ValueError(name)


def dense_exec_flops(nv, parity):
    """Executed tensor flops of one cell through the dense operator: three BF16 products
    (A_hi x_hi, A_lo x_hi, A_hi x_lo) of each sub-block, 2 flops per multiply-add.  The
    sub-blocks: the reflection blocks ((nv/2)^3 square) that the v1 <-> v2 transposition maps
    to others, and the even and odd halves (H^2 (H +- 1) / 2 square, H = nv/2) of those it maps
    to themselves -- plates {even, odd, whole}, ducts {even, odd, whole, whole, even, odd}."""
    H = nv // 2
    nf, ns, na = H ** 3, H * H * (H + 1) // 2, H * H * (H - 1) // 2
    sizes = [ns, na, nf] if parity == 2 else [ns, na, nf, nf, ns, na]
    return 3 * 2.0 * sum(n * n for n in sizes)


def fft_flops_per_cell(nv, M):
    """Algorithmic flops of one cell-L-eval: (M + 2) complex 3D FFTs (5 N log2 N each,
    N = nv^3) plus the multiplier products (6 per point per transform) and the angular
    accumulation (4 per point per direction)."""
    n3 = nv ** 3
    return 5.0 * n3 * np.log2(n3) * (M + 2) + 6.0 * n3 * (M + 1) + 4.0 * n3 * M


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, index):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + q,
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None
        return self

    def __exit__(self, *a):
        if self.p:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except Exception:
                self.p.kill()

    def summary(self):
        self.f.flush()
        self.f.seek(0)
        mhz, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                mhz.append(float(parts[1]))
                mx = max(mx, float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        os.unlink(self.f.name)
        if not mhz:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": float(np.median(mhz)), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(mhz)}


def oracle_sample(name, target_s=12.0):
    """Time the FP64 oracle on a bounded sample of the workload and extrapolate solves/s.

    Sample: the collision operator on k cells (k grown until ~target_s/2 of work), one
    kinetic sweep and one SIS update of the 101-node plate; per-iteration time of a case =
    101 x (per-cell L-eval) + sweep + update; solve time = iterations x that, with the
    iteration counts the oracle's own SIS needs at 16^3 scaled... the counts are taken
    from the GPU run when given (same discrete scheme), else 40 per case."""
    from oracle import fsm, solver, transport
    from paper_1612_04488_gb300 import workloads as W
    if name == "plates32x8":
        nv, M, ns, ncase = 32, 32, 100, 8
    elif name == "plates16":
        nv, M, ns, ncase = 16, 16, 20, 1
    else:
        nv, M, ns, ncase = 32, 32, 2048 - 1, 1
    t0 = time.perf_counter()
    F = fsm.FSM(nv, 6.0, M, 4.5)
    t_setup = time.perf_counter() - t0
    h = W.random_h(4, nv, 6.0, seed=3)
    k = 0
    t_apply = 0.0
    while t_apply < target_s / 2 and k < 256:
        t0 = time.perf_counter()
        F.apply(h[k % 4], 1.0)
        t_apply += time.perf_counter() - t0
        k += 1
    per_cell = t_apply / k
    n = ns + 1
    x = transport.nodes_clustered(ns) if name == "plates32x8" else transport.nodes_uniform(ns)
    rhs = W.random_h(n, nv, 6.0, seed=4) if n <= 201 else W.random_h(8, nv, 6.0, seed=4)
    t0 = time.perf_counter()
    if n <= 201:
        hh = transport.sweep_1d(rhs, F.nu, F.V1, x)
        Uh, qh, W1, W2, X12 = solver.cell_moments(F, hh)
        G1, G2 = solver.l_moments(F, hh, hh, 1.25)
        solver.diffusion_1d(Uh, W1, G1, x, 1.25, 1.0)
    t_rest = time.perf_counter() - t0
    t_iter = n * per_cell + t_rest
    return dict(per_cell_s=per_cell, cells_sampled=k, t_iter_s=t_iter, setup_s=t_setup,
                sample_s=t_apply + t_rest, ncase=ncase, n=n)


def _oracle_worker(a):
    """One host process: build the oracle operator, then time L-evals for ~target_s."""
    nv, M, R, seed, target_s = a
    from oracle import fsm
    from paper_1612_04488_gb300 import workloads as W
    F = fsm.FSM(nv, 6.0, M, R)
    h = W.random_h(2, nv, 6.0, seed=seed)
    k, t = 0, 0.0
    while t < target_s and k < 512:
        t0 = time.perf_counter()
        F.apply(h[k % 2], 1.0)
        t += time.perf_counter() - t0
        k += 1
    return k, t


def oracle_parallel_rate(nv, M, R, target_s, procs=None):
    """Cell-L-evals/s of the oracle with one process per host core (spawned, so it is safe
    after CUDA has been initialised).  Returns (rate, processes)."""
    import multiprocessing as mp
    procs = procs or os.cpu_count() or 1
    ctx = mp.get_context("spawn")
    with ctx.Pool(procs) as pool:
        out = pool.map(_oracle_worker, [(nv, M, R, 100 + i, target_s) for i in range(procs)])
    return sum(k / t for k, t in out if t > 0), procs


def run_reference(args):
    """Reference arm: the FP64 oracle, timed on bounded samples on the host cores."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    if args.workload.startswith("mix_"):
        print(json.dumps({"impl": "reference", "unavailable": "the mixture oracle forms dense spectral matrices at "
                                                              "N^6 M cost and runs at nv <= 12 only: no bounded "
                                                              "sample of the 24^3 workload"}), flush=True)
        return 0
    iters = args.ref_iters
    vals = []
    for _ in range(args.warmup):
        oracle_sample(args.workload, target_s=2.0)
    t_wall = 0.0
    for _ in range(args.steps):
        s = oracle_sample(args.workload, target_s=args.ref_sample_s)
        t_solve = s["t_iter_s"] * iters
        vals.append(1.0 / t_solve)
        t_wall += s["sample_s"]
    value = float(np.median(vals))
    line = {
        "impl": "reference", "metric": "SIS solves/s at 1e-6 flow-rate error", "value": value,
        "unit": "solves/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000.0 * t_wall / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "iterations_per_solve": iters,
                   "sample": "oracle L-eval on sampled cells + one sweep/update, extrapolated"},
        "cpu_baseline": {"value": value, "unit": "solves/s", "cores": 1, "kind": "oracle",
                         "sample": "per-cell L-eval x cells + sweep per iteration x %d iterations "
                                   "(the mean FP64 SIS iteration count of the workload)" % iters},
        "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


MIX_NE_AR = (39.95 / 20.18, 1.0 / 0.711)   # m_Ar / m_Ne; d_Ar / d_Ne (Sec. 4: d_Ne / d_Ar = 0.711)
FP64_NOMINAL_TFLOPS = 1.25                   # GB300 FP64, nominal


def table4_chi05():
    rows = {}
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tests", "golden",
                        "table4_ne_ar_poiseuille_chi05.txt")
    for line in open(path):
        if line.strip() and not line.startswith("#"):
            x = [float(t) for t in line.split()]
            rows[x[0]] = x[2:]
    return rows


def mixture_measure(lbe, torch, device, steps, warmup, nv=24, M=32, deltas=(1.0, 10.0)):
    """Binary-mixture SIS (Sec. 4) on Table 4's setting: Ne-Ar, chi_Ne = 0.5, plates with 100
    clustered sections, FP64, eps 1e-8; a step solves one problem per delta.  Returns the
    throughput, the FP64 GEMM of the dense mixture operator against the nominal FP64 rate,
    and the flow rates against Table 4."""
    stream = torch.cuda.Stream(device)
    ctx = lbe.Context(device)
    ctx.set_stream(stream.cuda_stream)
    pbs = [lbe.mix_problem(MIX_NE_AR[0], MIX_NE_AR[1], 0.5, delta=d, ns=100, grid_kind=1, nv=nv, vmax=5.0, M=M,
                           R=3.75, eps=1e-8, max_iter=400) for d in deltas]
    t0 = time.perf_counter()
    ctx.mix_info(pbs[0].mix, nv, 5.0, M, 3.75)
    build_s = time.perf_counter() - t0
    # the operator's GEMM in double-float on the FP32 pipes (FP64-class), same stopping test
    fpbs = [lbe.mix_problem(MIX_NE_AR[0], MIX_NE_AR[1], 0.5, delta=d, ns=100, grid_kind=1, nv=nv, vmax=5.0, M=M,
                            R=3.75, eps=1e-8, max_iter=400, precision=lbe.DF32) for d in deltas]
    for pb in fpbs:
        ctx.mix_solve(pb, want_U=False)
    fa, fb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    fa.record(stream)
    fres = [ctx.mix_solve(pb, want_U=False)[0] for pb in fpbs]
    fb.record(stream)
    fb.synchronize()
    lbe.set_kernel_timing(True)
    q0 = lbe.stats()
    ctx.mix_solve(fpbs[-1], want_U=False)
    q1 = lbe.stats()
    lbe.set_kernel_timing(False)
    ms_df = (q1["dense_gemm_ms"] - q0["dense_gemm_ms"]) / max(q1["dense_gemm_timed"] - q0["dense_gemm_timed"], 1)
    # BF16 hi / lo operator on the tensor cores, then FP64-class iterations to the same stopping test
    rpbs = [lbe.mix_problem(MIX_NE_AR[0], MIX_NE_AR[1], 0.5, delta=d, ns=100, grid_kind=1, nv=nv, vmax=5.0, M=M,
                            R=3.75, eps=1e-8, max_iter=400, precision=lbe.BF16_REFINED) for d in deltas]
    for _ in range(warmup):
        for pb in pbs + rpbs:
            ctx.mix_solve(pb, want_U=False)
    torch.cuda.synchronize()
    ra, rb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ra.record(stream)
    for _ in range(steps):
        rres = [ctx.mix_solve(pb, want_U=False)[0] for pb in rpbs]
    rb.record(stream)
    rb.synchronize()
    ms_ref = ra.elapsed_time(rb)
    s0 = lbe.stats()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    w0 = time.perf_counter()
    a.record(stream)
    for _ in range(steps):
        res = [ctx.mix_solve(pb, want_U=False)[0] for pb in pbs]
    b.record(stream)
    b.synchronize()
    wall = time.perf_counter() - w0
    s1 = lbe.stats()
    ms = a.elapsed_time(b)
    # the FP64 GEMM alone, timed per launch by the library during one more solve
    lbe.set_kernel_timing(True)
    g0 = lbe.stats()
    ctx.mix_solve(pbs[-1], want_U=False)
    g1 = lbe.stats()
    lbe.set_kernel_timing(False)
    n_t = g1["dense_gemm_timed"] - g0["dense_gemm_timed"]
    ms_gemm = (g1["dense_gemm_ms"] - g0["dense_gemm_ms"]) / max(n_t, 1)
    rows = 2 * nv ** 3 // 4                      # both species, one value per plate orbit
    cells = 101
    flops = 2.0 * rows * rows * cells
    achieved = flops / (ms_gemm / 1000.0) / 1e12
    T = table4_chi05()
    t4 = {}
    for d, r in zip(deltas, res):
        got = [r.M_A, r.M_B, -r.Q_A / 0.5, -r.Q_B / 0.5]
        t4[str(d)] = {"got": got, "table4": T[d], "rel": [g / p - 1.0 for g, p in zip(got, T[d])],
                      "iters": r.iters, "status": r.status}
    # the square duct (Table 5's setting): 40 x 40 cells, delta = 10, BF16 refined
    dpb = lbe.mix_problem(MIX_NE_AR[0], MIX_NE_AR[1], 0.5, delta=10.0, nv=nv, vmax=5.0, M=M, R=3.75, eps=1e-7,
                          max_iter=400, precision=lbe.BF16_REFINED, dim=2, nx=40, ny=40, width=1.0)
    ctx.mix_solve(dpb, want_U=False)
    da, db = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    da.record(stream)
    dr = ctx.mix_solve(dpb, want_U=False)[0]
    db.record(stream)
    db.synchronize()
    t5 = [0.630, 0.610, 0.057, 0.038]   # Table 5, aspect ratio 1, delta = 10: M_Ne, M_Ar, -2Q_Ne, -2Q_Ar
    dgot = [dr.M_A, dr.M_B, -2.0 * dr.Q_A, -2.0 * dr.Q_B]
    duct = {"solves_per_s": 1000.0 / da.elapsed_time(db), "cells": 1600, "iters": dr.iters,
            "fp64_iters": dr.fp64_iters, "status": dr.status, "got": dgot, "table5": t5,
            "rel": [g / p - 1.0 for g, p in zip(dgot, t5)],
            "what": "square duct, 40 x 40 cells, delta = 10, BF16 refined, eps 1e-7"}
    # the porous workload: the periodic unit cell of a square array of cylinders (solid fraction 0.4),
    # 100 x 100 cells, d_B / d_A = 1 / 0.72, delta = 10; the low-precision solve and the refined one
    por = {}
    for tag, prec in (("bf16", lbe.BF16), ("refined", lbe.BF16_REFINED)):
        ppb = lbe.mix_problem(MIX_NE_AR[0], 1.0 / 0.72, 0.5, delta=10.0, nv=nv, vmax=5.0, M=M, R=3.75, eps=1e-6,
                              max_iter=400, precision=prec, dim=2, nx=100, ny=100, solid=0.4)
        if tag == "bf16":
            ctx.mix_solve(ppb, want_U=False)
        pa, pbv = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        pa.record(stream)
        pr = ctx.mix_solve(ppb, want_U=False)[0]
        pbv.record(stream)
        pbv.synchronize()
        por[tag] = {"solves_per_s": 1000.0 / pa.elapsed_time(pbv), "iters": pr.iters, "fp64_iters": pr.fp64_iters,
                    "status": pr.status, "rates": [pr.M_A, pr.M_B, pr.Q_A, pr.Q_B]}
    por["bf16_max_rel_vs_refined"] = max(abs(x / y - 1.0) for x, y in zip(por["bf16"]["rates"][:2],
                                                                           por["refined"]["rates"][:2]))
    por["what"] = ("periodic unit cell, centred cylinder of area 0.4 (staircase), 100 x 100 cells, Ne-Ar chi 0.5, "
                   "d_B / d_A = 1 / 0.72, delta = 10, eps 1e-6")
    nsolve = len(pbs) * steps
    rel = max(abs(x / y - 1.0) for r, q in zip(rres, res)
              for x, y in ((r.M_A, q.M_A), (r.M_B, q.M_B), (r.Q_A, q.Q_A), (r.Q_B, q.Q_B)))
    frel = max(abs(x / y - 1.0) for r, q in zip(fres, res)
               for x, y in ((r.M_A, q.M_A), (r.M_B, q.M_B), (r.Q_A, q.Q_A), (r.Q_B, q.Q_B)))
    df32 = {"solves_per_s": len(fpbs) / (fa.elapsed_time(fb) / 1000.0), "max_rel_err_vs_fp64": frel,
            "gemm_ms_per_launch": ms_df, "gemm_fp64_equivalent_tflops": flops / (ms_df / 1000.0) / 1e12,
            "gemm_speedup_vs_fp64": ms_gemm / ms_df,
            "what": "the operator's GEMM in double-float arithmetic on the FP32 pipes (TwoProduct by FMA, "
                    "TwoSum accumulation), everything else FP64"}
    refined = {"solves_per_s": nsolve / (ms_ref / 1000.0), "ms_per_step": ms_ref / steps,
               "iters": [r.iters for r in rres], "fp64_iters": [r.fp64_iters for r in rres],
               "max_rel_err_vs_fp64": rel,
               "what": "tcgen05 BF16 hi/lo operator (float accumulation) down to its floor, then defect "
                       "correction: FP64-class (double-float GEMM) iterations, the same 1e-8 stopping test, "
                       "whose errors are solved for by the source-free iteration on the tensor cores"}
    out = {"solves_per_s": nsolve / (ms / 1000.0), "ms_per_step": ms / steps, "build_s": build_s,
           "refined": refined, "df32": df32, "duct": duct, "porous": por, "fp64_iters": [r.iters for r in res],
           "e2e": {"value": nsolve / wall, "unit": "solves/s",
                   "h2d_bytes_per_step": int((s1["h2d_bytes"] - s0["h2d_bytes"]) / steps),
                   "d2h_bytes_per_step": int((s1["d2h_bytes"] - s0["d2h_bytes"]) / steps)},
           "gpu_launches": int(s1["kernel_launches"] - s0["kernel_launches"]),
           "roofline": {"bound": "alu", "kernel": "k_mix_gemm (FP64 dense mixture operator, plate orbit layout, "
                                                  "%d x %d x %d cells)" % (rows, rows, cells),
                        "achieved": achieved, "peak": FP64_NOMINAL_TFLOPS, "unit": "TFLOP/s",
                        "frac": achieved / FP64_NOMINAL_TFLOPS, "peak_source": "nominal GB300 FP64 rate",
                        "traffic": None, "timed_launches": int(n_t), "ms_per_launch": ms_gemm,
                        "flops_per_launch": flops,
                        "algorithmic_unit": "2 (2 nv^3/4)^2 flops per cell: the dense operator is the method's "
                                            "form here (the unequal-mass gain does not factor into transforms)"},
           "table4": t4,
           "config": {"workload": "mix_ne_ar%d" % nv, "mixture": "Ne-Ar hard spheres, chi_Ne = 0.5",
                      "deltas": list(deltas), "nv": nv, "M": M, "vmax": 5.0, "R": 3.75, "ns": 100,
                      "grid": "clustered", "eps": 1e-8, "precision": "FP64"}}
    ctx.close()
    return out


def porous_measure(lbe, torch, device, steps, warmup, nv=24, M=32, deltas=(1.0, 10.0), eps=1e-6, n=100):
    """Binary mixture in the periodic unit cell of a square array of cylinders: n x n cells,
    solid fraction 0.4 (porosity 0.6), Ne-Ar chi = 0.5, d_B / d_A = 1 / 0.72, 24^3, M = 32.
    A step solves one problem per delta with LBE_BF16_REFINED to eps.  Also: the tensor-core
    GEMM of the mixture operator timed by the library during a BF16 solve (the kernel the
    low-precision iterations spend on), against the measured bf16 peak."""
    stream = torch.cuda.Stream(device)
    ctx = lbe.Context(device)
    ctx.set_stream(stream.cuda_stream)

    def mk(d, prec):
        return lbe.mix_problem(MIX_NE_AR[0], 1.0 / 0.72, 0.5, delta=d, nv=nv, vmax=5.0, M=M, R=3.75, eps=eps,
                               max_iter=400, precision=prec, dim=2, nx=n, ny=n, solid=0.4)

    pbs = [mk(d, lbe.BF16_REFINED) for d in deltas]
    # the first solve builds the operator in the duct orbit layout and its tensor-core form
    t0 = time.perf_counter()
    ctx.mix_solve(pbs[0], want_U=False)
    first_s = time.perf_counter() - t0
    for _ in range(warmup):
        for pb in pbs:
            ctx.mix_solve(pb, want_U=False)
    torch.cuda.synchronize()
    s0 = lbe.stats()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    w0 = time.perf_counter()
    a.record(stream)
    for _ in range(steps):
        res = [ctx.mix_solve(pb, want_U=False)[0] for pb in pbs]
    b.record(stream)
    b.synchronize()
    wall = time.perf_counter() - w0
    s1 = lbe.stats()
    ms = a.elapsed_time(b)
    # the low-precision solve alone, with the tensor-core GEMM timed launch by launch
    bpb = mk(deltas[-1], lbe.BF16)
    lbe.set_kernel_timing(True)
    g0 = lbe.stats()
    br = ctx.mix_solve(bpb, want_U=False)[0]
    g1 = lbe.stats()
    lbe.set_kernel_timing(False)
    n_t = g1["dense_gemm_timed"] - g0["dense_gemm_timed"]
    ms_gemm = (g1["dense_gemm_ms"] - g0["dense_gemm_ms"]) / max(n_t, 1)
    # the GEMM's columns: the fluid cells, those whose centre lies outside the circle of area 0.4
    c = (np.arange(n) + 0.5) * (1.0 / n) - 0.5
    fluid = int((c[:, None] ** 2 + c[None, :] ** 2 >= 0.4 / np.pi).sum())
    rows = 2 * nv ** 3 // 2                      # both species, one value per duct orbit
    flops = 2.0 * rows * rows * fluid           # the dense operator is the method's form
    peaks = load_peaks()
    peak = peaks.get("bf16_tflops", 1900.0)
    achieved = flops / (ms_gemm / 1000.0) / 1e12
    ref = res[-1]
    rel = max(abs(x / y - 1.0) for x, y in ((br.M_A, ref.M_A), (br.M_B, ref.M_B)))
    nsolve = len(pbs) * steps
    out = {"solves_per_s": nsolve / (ms / 1000.0), "ms_per_step": ms / steps, "first_solve_s": first_s,
           "solves": [{"delta": d, "iters": r.iters, "fp64_iters": r.fp64_iters, "status": r.status,
                       "rates": [r.M_A, r.M_B, r.Q_A, r.Q_B]} for d, r in zip(deltas, res)],
           "bf16": {"delta": deltas[-1], "iters": br.iters, "status": br.status, "max_rel_vs_refined": rel},
           "e2e": {"value": nsolve / wall, "unit": "solves/s",
                   "h2d_bytes_per_step": int((s1["h2d_bytes"] - s0["h2d_bytes"]) / steps),
                   "d2h_bytes_per_step": int((s1["d2h_bytes"] - s0["d2h_bytes"]) / steps)},
           "gpu_launches": int(s1["kernel_launches"] - s0["kernel_launches"]),
           "roofline": {"bound": "tensor", "kernel": "k_dense_gemm (mixture operator, BF16 hi/lo, %d x %d x %d fluid "
                                                     "cells)" % (rows, rows, fluid),
                        "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                        "peak_source": "bf16_tflops (burst, %s)" % peaks["_source"], "traffic": None,
                        "timed_launches": int(n_t), "ms_per_launch": ms_gemm, "flops_per_launch": flops,
                        "executed_flops_per_launch": 3.0 * flops,
                        "algorithmic_unit": "2 (2 nv^3/2)^2 flops per fluid cell (one product of the dense "
                                            "operator; the hi/lo split executes three)"},
           "config": {"workload": "mix_porous%d" % n, "mixture": "Ne-Ar hard spheres, chi_Ne = 0.5, "
                                                               "d_B / d_A = 1 / 0.72",
                      "geometry": "periodic unit cell, centred cylinder of area 0.4 (staircase), %d x %d cells, "
                                  "%d fluid" % (n, n, fluid),
                      "deltas": list(deltas), "nv": nv, "M": M, "vmax": 5.0, "R": 3.75, "eps": eps,
                      "precision": "BF16_REFINED",
                      "l2": "inputs larger than L2 (h: %d MB in FP64)" % (n * n * nv ** 3 * 8 // 2 ** 20)}}
    ctx.close()
    return out


def run_porous(args):
    import torch
    from paper_1612_04488_gb300 import lbe
    torch.cuda.set_device(0)
    with Clocks(0) as clk:
        m = porous_measure(lbe, torch, 0, args.steps, args.warmup)
    line = {"metric": "binary-mixture SIS solves/s at 1e-6 flow-rate change (porous unit cell)",
            "value": m["solves_per_s"], "unit": "solves/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": m["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": DTYPES["bf16"], "data": "synthetic", "config": m["config"],
            "roofline": m["roofline"], "solves": m["solves"], "bf16": m["bf16"], "first_solve_s": m["first_solve_s"],
            "e2e": m["e2e"], "clocks": clk.summary(), "gpu_launches": m["gpu_launches"]}
    print(json.dumps(line), flush=True)
    return 0


def run_mixture(args):
    import torch
    from paper_1612_04488_gb300 import lbe
    torch.cuda.set_device(0)
    with Clocks(0) as clk:
        m = mixture_measure(lbe, torch, 0, args.steps, args.warmup)
    line = {"metric": "binary-mixture SIS solves/s (Ne-Ar plates, Table 4 setting)", "value": m["solves_per_s"],
            "unit": "solves/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": m["ms_per_step"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic", "config": m["config"], "roofline": m["roofline"],
            "table4": m["table4"], "build_s": m["build_s"], "refined": m["refined"], "df32": m["df32"],
            "duct": m["duct"], "porous": m["porous"],
            "e2e": m["e2e"],
            "clocks": clk.summary(),
            "gpu_launches": m["gpu_launches"]}
    print(json.dumps(line), flush=True)
    return 0


def run_op_only(args):
    """Collision operator alone on the workload's cells (for profiling); prints timings.
    bf16: the tensor-core parity-subspace operator; fp32 / fp64: the fast-spectral one, over
    all directions or, with --sym, over one direction per reflection orbit (as the solves run
    it)."""
    import torch

    from paper_1612_04488_gb300 import lbe
    from paper_1612_04488_gb300 import workloads as W

    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    ctx = lbe.Context(0)
    prec = PRECISIONS[args.precision](lbe)
    prec = lbe.FP32 if prec == lbe.FP32_REFINED else prec
    pbs = workload_problems(lbe, args.workload, prec, args.eps)
    nv, M = pbs[0].nv, pbs[0].M
    cells = sum(lbe.cells_of(p) for p in pbs)
    dt = torch.float64 if prec in (lbe.FP64, lbe.DF32) else torch.float32
    h = W.random_h(cells, nv, 6.0, seed=11)
    h = 0.5 * (h + h[:, :, ::-1, :])
    hd = torch.tensor(h, device="cuda", dtype=dt)
    dd = torch.full((cells,), 1.0, device="cuda", dtype=torch.float64)
    lp = torch.empty_like(hd)
    lo = torch.empty_like(hd)
    parity = 2 if pbs[0].geom.dim == 1 else 1
    times = []
    for i in range(args.warmup + args.steps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        if prec == lbe.BF16_REFINED or args.sym:
            ctx.apply_L_sym(nv, 6.0, M, pbs[0].R, prec, parity, cells, dd.data_ptr(), hd.data_ptr(), lp.data_ptr(),
                            lo.data_ptr(), stream=stream.cuda_stream)
        else:
            ctx.apply_L(nv, 6.0, M, pbs[0].R, prec, cells, dd.data_ptr(), hd.data_ptr(), lp.data_ptr(), None,
                        stream=stream.cuda_stream)
        b.record(stream)
        b.synchronize()
        if i >= args.warmup:
            times.append(a.elapsed_time(b))
    print(json.dumps({"op_only": True, "workload": args.workload, "precision": args.precision, "cells": cells,
                      "ms": times, "l_evals_per_s": cells / (np.median(times) / 1000.0)}), flush=True)
    ctx.close()
    return 0


def serve_stream(ctx, lbe, prec, eps, requests):
    """The serving stream (workload "serve256"): mixed plates / ducts, nv in {24, 32}, delta
    log-uniform on [0.01, 100], submitted to the continuous-batching service.  Phase 1 submits
    everything at t = 0 (saturated throughput); phase 2 replays the stream with Poisson
    arrivals at 0.8x that rate and measures per-request latency (submit to result)."""
    from paper_1612_04488_gb300 import workloads as W

    def to_pb(r):
        geo = {k: r[k] for k in ("dim", "ns", "grid_kind", "nx", "ny", "width") if k in r}
        return lbe.problem(**geo, delta=r["delta"], nv=r["nv"], vmax=r["vmax"], M=r["M"], forcing=r["forcing"],
                           scheme=lbe.SIS, precision=prec, eps=eps, max_iter=400)

    reqs = W.serving_requests(n=requests, seed=20261203)
    pbs = [to_pb(r) for r in reqs]

    def run_stream(arrivals):
        t0 = time.perf_counter()
        tickets, sub_t = [], []
        done = {}
        i = 0
        while len(done) < len(pbs):
            now = time.perf_counter() - t0
            while i < len(pbs) and arrivals[i] <= now:
                tickets.append(ctx.submit(pbs[i]))
                sub_t.append(time.perf_counter() - t0)
                i += 1
            for k, tk in enumerate(tickets):
                if k not in done:
                    ok, r = ctx.poll(tk)
                    if ok:
                        done[k] = (time.perf_counter() - t0, r)
            time.sleep(0.0005)
        wall = time.perf_counter() - t0
        lat = [done[k][0] - sub_t[k] for k in range(len(pbs))]
        res = [done[k][1] for k in range(len(pbs))]
        return wall, lat, res

    # warm-up: build the tables of both grids and the buckets
    warm = pbs[:4]
    tk = [ctx.submit(p) for p in warm]
    while not all(ctx.poll(t)[0] for t in tk):
        time.sleep(0.001)
    wall_sat, lat_sat, res_sat = run_stream([0.0] * len(pbs))
    rate_sat = len(pbs) / wall_sat
    rng = np.random.default_rng(7)
    rate = 0.8 * rate_sat
    arr = np.cumsum(rng.exponential(1.0 / rate, size=len(pbs)))
    wall, lat, res = run_stream(list(arr))
    bad = sum(1 for r in res + res_sat if r.status != lbe.OK)
    return {"workload": "serve%d" % requests, "requests": len(pbs), "failed": bad,
            "solves_per_s": len(pbs) / wall, "saturated_solves_per_s": rate_sat, "arrival_rate": rate,
            "latency_ms": {"p50": 1000 * float(np.percentile(lat, 50)), "p99": 1000 * float(np.percentile(lat, 99)),
                           "what": "Poisson arrivals at 0.8x the saturated rate, submit to result"},
            "latency_saturated_ms": {"p50": 1000 * float(np.percentile(lat_sat, 50)),
                                     "p99": 1000 * float(np.percentile(lat_sat, 99))},
            "mix": "plates 50-200 sections / ducts 20x20-80x40, nv 24/32, delta log-uniform [0.01, 100], M = 32",
            "eps": eps}


def run_serve(args):
    """The serving stream alone (--serve), one JSON line."""
    import torch

    from paper_1612_04488_gb300 import lbe

    torch.cuda.set_device(0)
    ctx = lbe.Context(0)
    prec = PRECISIONS[args.precision](lbe)
    sv = serve_stream(ctx, lbe, prec, args.eps, args.requests)
    line = {"metric": "serving: solves/s and per-request latency (Poisson arrivals)",
            "value": sv["solves_per_s"], "unit": "solves/s", "n_gpus": 1, "higher_is_better": True,
            "dtype": DTYPES[args.precision], "data": "synthetic", "config": {"workload": sv["workload"]},
            "serving": sv}
    print(json.dumps(line), flush=True)
    ctx.close()
    return 0


# DRAM bytes (read + write) of one launch of the GEMM kernel the tuner picks (the persistent
# k_dense_gemm_ws), from an ncu capture of `bench.py --op-only` (plates32x8, 808 cells), valid
# only while the kernel's source is the one captured: the digest covers the kernels and their
# stage configuration.
GEMM_TRAFFIC = {"plates32x8": {"cells": 808, "bytes": 131834624 + 9925632, "digest": "0a6efc136065442e"}}


def gemm_source_digest():
    import hashlib
    src = open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "paper_1612_04488_gb300", "csrc",
                            "fsm_dense.cu")).read()
    a = src.index("struct GemmCfg")
    b = src.index("// ---- reflection blocks and their transposition halves")
    return hashlib.sha256(src[a:b].encode()).hexdigest()[:16]


def gemm_traffic(workload, cells):
    t = GEMM_TRAFFIC.get(workload)
    if not t or t["cells"] != cells or t["digest"] != gemm_source_digest():
        return None
    return t["bytes"]


def replica_throughput(local_ms, units_per_rank, dist=None, device="cpu"):
    """Whole-job throughput of independent replicas: every rank processed units_per_rank units;
    the job took as long as its slowest rank (max over ranks).  Returns (units/s, slowest ms)."""
    import torch

    t = torch.tensor([float(local_ms)], dtype=torch.float64, device=device)
    world = 1
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        world = dist.get_world_size()
    slowest = float(t.item())
    return units_per_rank * world / (slowest / 1000.0), slowest


def run_ours(args):
    import torch

    from paper_1612_04488_gb300 import lbe

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist_
        dist = dist_
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    ctx = lbe.Context(local)
    ctx.set_stream(stream.cuda_stream)
    prec = PRECISIONS[args.precision](lbe)
    pbs = workload_problems(lbe, args.workload, prec, args.eps)
    nsolve = len(pbs)
    batch = ctx.batch(pbs) if prec in (lbe.FP32, lbe.FP64) else None

    def one_step():
        return batch.run() if batch is not None else ctx.solve_batch(pbs)

    for _ in range(args.warmup):
        res = one_step()
    # ---- timed region: K batched solves, device resident --------------------------------
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    st0 = lbe.stats()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    step_ms, solve_ms = [], []
    with Clocks(local) as clk:
        torch.cuda.nvtx.range_push("timed")  # lets a profiler select exactly these launches
        e0.record(stream)
        for _ in range(args.steps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            res = one_step()
            b.record(stream)
            b.synchronize()
            step_ms.append(a.elapsed_time(b))
            solve_ms += [1000.0 * r.seconds for r in res]
        e1.record(stream)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
    st1 = lbe.stats()
    if dist:
        dist.barrier()
    value, total_ms = replica_throughput(e0.elapsed_time(e1), nsolve * args.steps, dist, "cuda")
    launches = int(st1["kernel_launches"] - st0["kernel_launches"])
    iters = [r.iters for r in res]
    refinements = [r.refinements for r in res]
    status = [r.status for r in res]
    clocks = clk.summary()

    # ---- accuracy against the FP64 GPU path (parity-tested against the oracle) ----------
    ref = None
    fp64 = None
    if args.check_fp64 and prec != lbe.FP64:
        rpbs = workload_problems(lbe, args.workload, lbe.FP64, min(args.eps, 1e-10))
        ref = ctx.solve_batch(rpbs)
        err = max(max(abs(r.mass_flow - q.mass_flow) / abs(q.mass_flow),
                      abs(r.heat_flow - q.heat_flow) / abs(q.heat_flow)) for r, q in zip(res, ref))
        # the plain FP64 GPU path at the same eps: the comparison the mixed precision must beat
        b64 = ctx.batch(workload_problems(lbe, args.workload, lbe.FP64, args.eps))
        b64.run()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        r64 = b64.run()
        b.record(stream)
        b.synchronize()
        b64.close()
        fp64 = {"solves_per_s": nsolve / (a.elapsed_time(b) / 1000.0), "eps": args.eps,
                "iterations": [r.iters for r in r64],
                "max_rel_err_vs_fp64_1e-10": max(max(abs(r.mass_flow - q.mass_flow) / abs(q.mass_flow),
                                                     abs(r.heat_flow - q.heat_flow) / abs(q.heat_flow))
                                                 for r, q in zip(r64, ref))}
    else:
        err = None

    # ---- end to end: the one-shot public call ----------------------------------------
    torch.cuda.synchronize()
    s0 = lbe.stats()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        ctx.solve_batch(pbs)
    t_e2e = time.perf_counter() - t0
    s1 = lbe.stats()
    e2e = {"value": nsolve * args.steps * world / t_e2e, "unit": "solves/s",
           "h2d_bytes_per_step": int((s1["h2d_bytes"] - s0["h2d_bytes"]) / args.steps),
           "d2h_bytes_per_step": int((s1["d2h_bytes"] - s0["d2h_bytes"]) / args.steps)}

    # ---- collision operator alone (dominant kernel) ------------------------------------
    nv, M = pbs[0].nv, pbs[0].M
    cells = sum(lbe.cells_of(p) for p in pbs)
    from paper_1612_04488_gb300 import workloads as W
    hnp = W.random_h(cells, nv, 6.0, seed=11)
    hnp = 0.5 * (hnp + hnp[:, :, ::-1, :])  # plate parity: odd in v3, even in v2
    deltas = torch.tensor(np.repeat([p.delta for p in pbs], [lbe.cells_of(p) for p in pbs]),
                          device="cuda", dtype=torch.float64)
    parity = 2 if pbs[0].geom.dim == 1 else 1

    def time_apply(precision, reps, sym):
        dt = torch.float64 if precision in (lbe.FP64, lbe.DF32) else torch.float32
        hd = torch.tensor(hnp, device="cuda", dtype=dt)
        lp = torch.empty_like(hd)
        lo = torch.empty_like(hd)

        def call():
            if sym:
                ctx.apply_L_sym(nv, 6.0, M, pbs[0].R, precision, parity, cells, deltas.data_ptr(), hd.data_ptr(),
                                lp.data_ptr(), lo.data_ptr(), stream=stream.cuda_stream)
            else:
                ctx.apply_L(nv, 6.0, M, pbs[0].R, precision, cells, deltas.data_ptr(), hd.data_ptr(),
                            lp.data_ptr(), None, stream=stream.cuda_stream)
        call()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            call()
        b.record(stream)
        b.synchronize()
        return a.elapsed_time(b) / reps

    peaks = load_peaks()
    ms_fp64 = time_apply(lbe.FP64, 2, False)
    ms_fp64_sym = time_apply(lbe.FP64, 2, True)
    ms_fp32_sym = time_apply(lbe.FP32, 5, True)
    alg_flops = fft_flops_per_cell(nv, M) * cells
    ms_df_sym = time_apply(lbe.DF32, 2, True)
    if prec == lbe.BF16_REFINED:
        # the GEMM alone: the library brackets each launch with CUDA events on its stream
        lbe.set_kernel_timing(True)
        g0 = lbe.stats()
        ms_op = time_apply(lbe.BF16_REFINED, 10, True)
        g1 = lbe.stats()
        lbe.set_kernel_timing(False)
        n_t = g1["dense_gemm_timed"] - g0["dense_gemm_timed"]
        ms_gemm = (g1["dense_gemm_ms"] - g0["dense_gemm_ms"]) / max(n_t, 1)
        exec_flops = dense_exec_flops(nv, parity) * cells  # useful products only (no padding columns)
        peak = peaks.get("bf16_tflops", 1900.0)
        # achieved: the method's algorithmic work (the FFT-equivalent flops of one full
        # cell-L-eval x the cells of one launch) over the launch's duration
        achieved = alg_flops / (ms_gemm / 1000.0) / 1e12
        executed = exec_flops / (ms_gemm / 1000.0) / 1e12
        roofline = {"bound": "tensor", "kernel": "k_dense_gemm (tcgen05 kind::f16, BF16 hi/lo x3, FP32 TMEM "
                                                 "accumulate), %d cells" % cells,
                    "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                    "peak_source": "bf16_tflops (burst, %s)" % peaks["_source"],
                    "traffic": gemm_traffic(args.workload, cells),
                    "timed_launches": n_t, "ms_per_launch": ms_gemm,
                    "algorithmic_flops_per_launch": alg_flops,
                    "algorithmic_unit": "%.1f MFLOP per cell-L-eval (FFT-equivalent, all %d directions) x %d cells"
                                        % (fft_flops_per_cell(nv, M) / 1e6, M, cells),
                    "executed_flops_per_launch": exec_flops, "executed_tflops": executed,
                    "executed_frac": executed / peak,
                    "whole_call_ms": ms_op, "whole_call": "gather + GEMM + expand (lbe_apply_L_sym)"}
    else:
        ms_op = ms_fp32_sym if prec != lbe.FP64 else ms_fp64_sym
        clk_mhz = peaks.get("sm_max_mhz", 2070.0)
        lanes = 128 if prec != lbe.FP64 else 2
        peak = 152 * lanes * 2 * clk_mhz * 1e6 / 1e12
        sym_flops = (5.0 * nv ** 3 * np.log2(nv ** 3) * (M // (4 if parity == 2 else 2) + 2)) * cells
        achieved = sym_flops / (ms_op / 1000.0) / 1e12
        roofline = {"bound": "alu", "kernel": "fast spectral transforms (fsm_cc chain, symmetry-reduced)",
                    "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                    "peak_source": "152 SMs x %d lanes x 2 x %.0f MHz" % (lanes, clk_mhz), "traffic": None,
                    "algorithmic_flops_per_launch": sym_flops, "ms_per_launch": ms_op}
    # ---- the transport sweep (HBM-bound), timed by the library inside an FP32 solve of the workload
    sweep = None
    if prec != lbe.FP64:
        bf = ctx.batch(workload_problems(lbe, args.workload, lbe.FP32, args.eps))
        bf.run()
        lbe.set_kernel_timing(True)
        w0 = lbe.stats()
        bf.run()
        w1 = lbe.stats()
        lbe.set_kernel_timing(False)
        bf.close()
        n_sw = w1["sweep_timed"] - w0["sweep_timed"]
        if n_sw:
            sw_ms = w1["sweep_ms"] - w0["sweep_ms"]
            sw_bytes = w1["sweep_bytes"] - w0["sweep_bytes"]
            gbs = sw_bytes / (sw_ms / 1000.0) / 1e9
            hbm = peaks.get("hbm_gbs", 6800.0)
            sweep = {"bound": "hbm", "kernel": "k_sweep1d<float>" if pbs[0].geom.dim == 1 else "k_sweep2d<float>",
                     "achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm,
                     "peak_source": "hbm_gbs (%s)" % peaks["_source"], "timed_launches": n_sw,
                     "ms_per_launch": sw_ms / n_sw, "bytes_per_launch": sw_bytes / n_sw,
                     "algorithmic_unit": "8 B per cell-velocity (FP32 rhs read + h written)",
                     "what": "every sweep launch of one FP32 SIS solve of the workload (problems drop out as "
                             "they converge)"}
    l_evals = {"op": cells / (ms_op / 1000.0), "fp32_fft_sym": cells / (ms_fp32_sym / 1000.0),
               "df32_fft_sym": cells / (ms_df_sym / 1000.0),
               "fp64_fft_sym": cells / (ms_fp64_sym / 1000.0), "fp64_fft_full": cells / (ms_fp64 / 1000.0)}

    line = {
        "metric": "SIS solves/s at 1e-6 flow-rate error", "value": value, "unit": "solves/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": DTYPES[args.precision],
        "data": "synthetic",
        "config": {"workload": args.workload, "solves_per_step": nsolve, "cells": cells, "nv": nv, "M": M,
                   "eps": args.eps,
                   "l2": "inputs larger than L2 (h, L+h, h half-step: %d MB in FP32)" % (3 * cells * nv ** 3 * 4 // 2 ** 20),
                   "parallelism": "replicas" if world > 1 else "single"},
        "batch_latency_ms": {"p50": float(np.percentile(solve_ms, 50)), "p99": float(np.percentile(solve_ms, 99)),
                             "what": "per solve, batch start to that solve's convergence"},
        "iterations": iters, "refinements": refinements, "status": status,
        "max_rel_err_vs_fp64": err,
        "l_evals_per_s": l_evals["op"], "l_evals_per_s_fp64": l_evals["fp64_fft_sym"], "l_evals_detail": l_evals,
        "roofline": roofline, "roofline_sweep": sweep, "fp64_gpu": fp64, "autotuner": ctx.tuning_report(),
        "e2e": e2e, "clocks": clocks, "gpu_launches": launches,
    }
    # ---- the other workloads on the same line: the 64 x 32 duct (2048 cells, one solve) and
    # the serving stream (per-request p50 / p99 latency) ------------------------------------
    if args.workload == "plates32x8" and not args.no_extra:
        dpbs = workload_problems(lbe, "duct64x32", prec, args.eps)
        ctx.solve_batch(dpbs)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        dres = [ctx.solve_batch(dpbs)[0] for _ in range(2)]
        b.record(stream)
        b.synchronize()
        line["duct64x32"] = {"solves_per_s": 2.0 / (a.elapsed_time(b) / 1000.0), "cells": 2048,
                             "iterations": dres[-1].iters, "refinements": dres[-1].refinements,
                             "status": dres[-1].status}
        mx = mixture_measure(lbe, torch, local, 1, 1)
        line["mixture"] = {k: mx[k] for k in ("solves_per_s", "config", "roofline", "table4", "build_s", "refined",
                                              "df32", "duct", "porous")}
        sctx = lbe.Context(local)
        line["serving"] = serve_stream(sctx, lbe, prec, args.eps, args.requests)
        line["latency_ms"] = dict(line["serving"]["latency_ms"], workload=line["serving"]["workload"])
        sctx.close()
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # one extrapolation for both arms: per-iteration oracle time x the SIS iterations per
        # solve (--ref-iters, the workload's FP64 count), single core and all cores
        s = oracle_sample(args.workload, target_s=args.ref_sample_s)
        it = args.ref_iters
        one = 1.0 / (s["t_iter_s"] * it)
        rate, procs = oracle_parallel_rate(nv, M, pbs[0].R if pbs[0].R > 0 else 4.5, args.ref_sample_s / 2)
        t_iter_all = s["n"] * (1.0 / rate) + (s["t_iter_s"] - s["n"] * s["per_cell_s"])
        allc = 1.0 / (t_iter_all * it)
        line["cpu_baseline"] = {"value": allc, "unit": "solves/s", "cores": procs, "kind": "oracle",
                                "single_core": one,
                                "sample": "FP64 oracle L-evals for %.0f s on each of %d processes (%.1f cell-L-evals/s) "
                                          "+ one sweep/update of a %d-node plate; per-iteration time x %d iterations "
                                          "per solve" % (args.ref_sample_s / 2, procs, rate, s["n"], it)}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if batch is not None:
        batch.close()
    ctx.close()
    if dist:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="plates32x8", choices=["plates32x8", "plates16", "duct64x32",
                                                                  "mix_ne_ar24", "mix_porous100"])
    ap.add_argument("--precision", default="bf16", choices=sorted(PRECISIONS))
    ap.add_argument("--eps", type=float, default=1e-7)
    ap.add_argument("--ref-iters", type=int, default=35,
                    help="SIS iterations per solve for the oracle extrapolation (the workload's mean "
                         "FP64 count at eps = 1e-7)")
    ap.add_argument("--ref-sample-s", type=float, default=12.0)
    ap.add_argument("--no-check-fp64", dest="check_fp64", action="store_false")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--op-only", action="store_true", help="time the collision operator alone")
    ap.add_argument("--sym", action="store_true", help="--op-only: parity-reduced fast-spectral operator")
    ap.add_argument("--serve", action="store_true", help="serving stream with Poisson arrivals")
    ap.add_argument("--requests", type=int, default=256)
    ap.add_argument("--no-extra", action="store_true", help="skip the duct and serving entries of the line")
    args = ap.parse_args()
    if args.serve:
        return run_serve(args)
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "mix_ne_ar24":
        return run_mixture(args)
    if args.workload == "mix_porous100":
        return run_porous(args)
    if args.op_only:
        return run_op_only(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
