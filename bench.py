#!/usr/bin/env python
"""BoxMG V(2,1) throughput on one GB300 (or N replicas), one JSON line.

Workload (default): the largest single-GPU problem, 2D -div(k grad u) on an
8191 x 8191 interior grid (67.1 M unknowns), 9-point Q1 finite-element
stencil, k = exp(g) with g a Gaussian random field (std 2, correlation length
32 cells, seed 4), RHS uniform[-1, 1) (seed 7), four-colour Gauss-Seidel
V(2,1), twelve levels down to 3 x 3, synthetic seeded inputs.

A step is one iteration of the solve loop: one V(2,1) cycle (FP64) followed by
the residual norm and the device-side convergence test.  `value` is the FP64
path's unknowns per second per V(2,1) (grid unknowns x steps / device time),
over all ranks.  The FP32- and BF16-stencil refinement variants and the time to
a 1e-10 relative residual of every variant are reported beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--impl reference]

`--impl reference` times the CPU oracle (numpy, FP64, its colour passes and
residuals over row bands on every host core) on the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads as w  # noqa: E402

METRIC = "unknowns/s per V(2,1) & time to 1e-10 residual: FP64 vs mixed/learned, 1 GB300"
UNIT = "unknowns/s"

WORKLOADS = {
    "fe2047-binary1e4": dict(
        text="2047x2047 interior, 9-point Q1 FE of -div(k grad u), k in {1,1e4} on 16x16 blocks "
             "(Bernoulli 0.5, seed 2), RHS U[-1,1) seed 3, four-colour GS V(2,1), 10 levels",
        make=lambda: w.binary_contrast_problem(2047, 16, 1.0, 1e4, seed_k=2, seed_f=3)),
    "poisson127": dict(
        text="127x127 interior, 5-point Poisson, RHS U[-1,1) seed 1, red-black GS V(2,1), 6 levels",
        make=lambda: w.poisson_problem(127, 1)),
    "lognormal8191": dict(
        text="8191x8191 interior, 9-point Q1 FE, k = exp(g), g Gaussian field std 2, correlation 32 cells, "
             "seed 4; RHS U[-1,1) seed 7; 12 levels",
        make=lambda: w.lognormal_problem(8191, 2.0, 32.0, seed_k=4, seed_f=7)),
    "lognormal4095": dict(
        text="4095x4095 interior, 9-point Q1 FE, k = exp(g), g Gaussian field std 2, correlation 32 cells, "
             "seed 4; RHS U[-1,1) seed 7; 11 levels (the 8191^2 workload's recipe at a size ncu captures)",
        make=lambda: w.lognormal_problem(4095, 2.0, 32.0, seed_k=4, seed_f=7)),
}
WORKLOADS["learned4095"] = dict(
    text="4095x4095 interior, 9-point Q1 FE, k in {1,1e6} on 8x8 cell tiles (Bernoulli 0.5, seed 6), RHS U[-1,1) "
         "seed 100006; the learned-interpolation family: the network is trained on the GPU on 31^2 crops of 255^2 "
         "problems of the family (seeds 1000..) with the two-grid loss, then bmg_setup measures learned vs Dendy",
    make=lambda: w.high_contrast_problem(4095, seed=6))
DEFAULT_WORKLOAD = "lognormal8191"

# DRAM bytes (read + write) per fine point of one launch of a level-0 kernel,
# from one ncu capture of the current kernel (dram__bytes_read.sum +
# dram__bytes_write.sum over the launch / the level's unknowns) on the named
# workload, keyed by kernel (and shape).  A launch's traffic is this figure x
# the unknowns of the bench's level 0: the kernels stream their arrays, so
# traffic grows in proportion to the grid.  A kernel missing here, or changed
# since its capture, reports traffic null.
NCU_DRAM_BYTES_PER_POINT = {
    # captured with the 4-row ring; the ring depth does not change which rows and columns a strip reads
    **{f"k_gs_strip64 56xW cp.async/{r} fused": (1089.14e6 / 4095 ** 2, "lognormal4095") for r in (4, 6)},
    **{f"k_gs_strip<float> 56xW bulk/{r}": (540.66e6 / 4095 ** 2, "lognormal4095") for r in (4, 6)},
    **{f"k_gs_strip<bf16> 56xW bulk/{r}": (398.64e6 / 4095 ** 2, "lognormal4095") for r in (4, 6)},
    **{f"k_gs_strip2_ring<float> 48xW bulk/{r}": (549.46e6 / 4095 ** 2, "lognormal4095") for r in (4, 6)},
    **{f"k_gs_strip2_ring<bf16> 48xW bulk/{r}": (404.43e6 / 4095 ** 2, "lognormal4095") for r in (4, 6)},
}
TILE_SHAPES = ("56xW bulk/4", "56xW bulk/6", "56xW bulk/8", "56x32 bulk/4", "56x32 regs", "56x16 regs")
TILE64_SHAPES = ("56xW cp.async/4", "56x16 cp.async/4", "56xW cp.async/6", "56x8 cp.async/4")   # W: one wave
PAIR_SHAPES = ("48xW bulk/4", "48xW bulk/6", "48xW bulk/8", "48x26 bulk/4")   # W: one wave


BATCHED = dict(text="256 independent 9-point Q1 problems, sides uniform from {63,127,255,511,1023} (seed 5), "
                    "k = exp(g), g Gaussian field std 1, correlation 32 cells (seeds 10000+2b), RHS U[-1,1) "
                    "(seeds 10001+2b); batched V(2,1) to 1e-8 per problem")


def run_batched(args, rank, local_rank, world):
    """The batched extension: one step = one iteration of every problem of the
    rank's batch (V(2,1) + norm, or one refinement step), all in one CUDA
    graph.  Weak scaling over ranks: each rank solves its own 256 problems."""
    import torch
    import paper_2502_05279_gb300 as bmg
    torch.cuda.set_device(local_rank)
    ranks = Ranks("nccl")
    first, count = batched_shard(rank)
    probs = w.batched_problems(count, 5, 1.0, 32.0, first=first)
    N = sum((p[1].shape[-1] - 2) ** 2 for p in probs)
    coefs = [torch.from_numpy(p[1]).cuda() for p in probs]
    rhs = [torch.from_numpy(p[2]).cuda() for p in probs]
    out = {"metric": METRIC, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "data": "synthetic (seeded generators, no datasets)",
           "config": {"workload": "batched256", "description": BATCHED["text"], "unknowns_per_rank_0": N,
                      "problems_per_rank": count, "parallelism": "problems sharded over ranks" if world > 1
                      else "single GPU", "l2": "working set > L2 (FP64 level-0 stencils + vectors = %.0f MB)"
                      % (N * 64 / 1e6)}, "variants": {}}
    clock_s = None
    for prec in ("fp64", "fp32", "bf16"):
        ranks.barrier()
        t0 = time.perf_counter()
        B = bmg.Batch(9, coefs, precision=prec, arith=args.arith)
        torch.cuda.synchronize()
        setup_ms = (time.perf_counter() - t0) * 1e3
        xs = [torch.zeros_like(r) for r in rhs]
        B.time_cycles(rhs, xs, max(args.warmup, 3))
        ranks.barrier()
        before = B.launch_count
        if prec == "fp64":
            with ClockSampler(local_rank) as cs:
                with cs.timed():
                    ms = B.time_cycles(rhs, xs, args.steps)
            clock_s = cs.summary()
        else:
            ms = B.time_cycles(rhs, xs, args.steps)
        launches = B.launch_count - before
        ranks.barrier()
        rate = whole_job_rate(N * args.steps, ms * 1e-3, ranks)
        for x in xs:
            x.zero_()
        ranks.barrier()
        t0 = time.perf_counter()
        _, its, rrs, ok = B.solve(rhs, xs, tol=1e-8, maxit=100)
        torch.cuda.synchronize()
        tts = ranks.max((time.perf_counter() - t0) * 1e3)
        rec = {"value": rate, "ms_per_step": ranks.max(ms) / args.steps,
               "setup_ms_incl_autotune": round(setup_ms, 1), "time_to_1e-8_ms": round(tts, 2),
               "iterations_max": max(its), "iterations_min": min(its), "all_converged": ok,
               "launches_per_step": launches / args.steps,
               "tuned_cluster_by_stage": [B.tuned_cluster(b) for b in range(9)]}
        if prec == "fp64":
            rec["gpu_launches"] = launches
            # end to end through the public API with host buffers: every step copies all
            # right-hand sides in from pinned memory, solves to 1e-8, copies all x back
            rhs_host = [torch.from_numpy(p[2]).pin_memory() for p in probs]
            x_host = [torch.empty_like(r) .pin_memory() for r in rhs_host]
            e2e_steps, e2e_its = 2, 0
            ranks.barrier()
            t0 = time.perf_counter()
            for _ in range(e2e_steps):
                for d, h_ in zip(rhs, rhs_host):
                    d.copy_(h_, non_blocking=True)
                for x in xs:
                    x.zero_()
                _, its, _, _ = B.solve(rhs, xs, tol=1e-8, maxit=100)
                for h_, x in zip(x_host, xs):
                    h_.copy_(x, non_blocking=True)
                torch.cuda.synchronize()
                e2e_its += max(its)
            e2e_s = time.perf_counter() - t0
            nbytes = sum(int(r.numel()) * 8 for r in rhs_host)
            rec["e2e"] = {"value": whole_job_rate(N * e2e_its, e2e_s, ranks), "unit": UNIT,
                          "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes,
                          "note": "Batch.solve (FP64, every problem to 1e-8) from a zero guess per step; unknowns x "
                                  "batch iterations / wall time; right-hand sides H2D from pinned memory, x D2H"}
        out["variants"][prec] = rec
        B.close()
    v = out["variants"].pop("fp64")
    out["value"] = v["value"]
    out["ms_per_step"] = v["ms_per_step"]
    out["e2e"] = v.pop("e2e")
    out["gpu_launches"] = int(v.pop("gpu_launches"))
    out["fp64"] = v
    out["dtype"] = "f64"
    out["clocks"] = clock_s
    if rank == 0:
        if world == 1 and not args.no_cpu:
            out["cpu_baseline"] = batched_cpu_baseline(probs)
        print(json.dumps(out))
    ranks.close()


RHS_BATCHES = {
    "rhs64-1023": dict(text="64 right-hand sides U[-1,1) (seeds 500..563) of one 1023x1023 9-point Q1 problem, "
                            "k = exp(g), g Gaussian field std 2, correlation 32 cells (seed 4); bmg_batch_rhs vs 64 "
                            "solo solves, V(2,1)", n=1023, k=64),
    "rhs8-4095": dict(text="8 right-hand sides U[-1,1) (seeds 500..507) of one 4095x4095 9-point Q1 problem (its FP32 "
                           "stencil exceeds L2), k = exp(g), g Gaussian field std 2, correlation 32 cells (seed 4); "
                           "bmg_batch_rhs with one-pass sweeps taking 2 or 4 right-hand sides per warp (autotuned) "
                           "and with one per warp, vs 8 solo solves, V(2,1)", n=4095, k=8),
}


PERIODIC = {
    "periodic4095": dict(text="4096x4095 interior points, periodic in x (4096 = 2^12 columns, point 4097 is point 1), "
                              "zero Dirichlet in y; 9-point Q1 FE of -div(k grad u), k = exp(g), g the periodic "
                              "Gaussian field std 2, correlation 32 cells (seed 50) on the 4096^2 cells; RHS U[-1,1) "
                              "seed 51; FP64 V(2,1), four-colour GS, 11 levels down to 4 x 3", n=4095, axes="x"),
}


def run_periodic(args, rank, local_rank, world):
    """Periodic sides: the FP64 V(2,1) of the periodic hierarchy (each 9-point
    level swept by the one-pass strip kernel with wrapped indices or the
    row-parity pair, whichever setup timed as faster), its
    throughput, its time to 1e-10 and the level-0 sweep against the copy
    bandwidth and the FP64 instruction rate."""
    import torch
    import paper_2502_05279_gb300 as bmg
    torch.cuda.set_device(local_rank)
    ranks = Ranks("nccl")
    spec = PERIODIC[args.workload]
    kind, planes, f, px, py = w.periodic_problem(spec["n"], spec["axes"], seed_k=50, seed_f=51)
    nx, ny = planes.shape[-1] - 2, planes.shape[-2] - 2
    N = nx * ny
    coef = torch.from_numpy(planes).cuda()
    rhs = torch.from_numpy(f).cuda()
    t0 = time.perf_counter()
    h = bmg.Hierarchy(kind, coef, arith=args.arith, periodic=spec["axes"])
    torch.cuda.synchronize()
    setup_ms = (time.perf_counter() - t0) * 1e3
    x = torch.zeros_like(rhs)
    if args.only:
        # warm-up and timed cycles only: the small run profiled by ncu
        h.time_cycles(rhs, x, args.warmup)
        ms = h.time_cycles(rhs, x, args.steps)
        if rank == 0:
            print(json.dumps({"only": "fp64", "arith": args.arith, "workload": args.workload,
                              "ms_per_step": ms / args.steps, "launches": h.launch_count}))
        h.close()
        ranks.close()
        return
    fp64_rate = bmg.measure_fp64_rate() * 1e9        # DP instructions per second, measured here
    h.time_cycles(rhs, x, max(args.warmup, 3))
    ranks.barrier()
    before = h.launch_count
    with ClockSampler(local_rank) as cs:
        with cs.timed():
            ms = h.time_cycles(rhs, x, args.steps)
        launches = h.launch_count - before
        ms = ranks.max(ms)
        prof = h.profile(rhs, torch.zeros_like(rhs), 3)
        x.zero_()
        h.solve(rhs, x, tol=1e-10, maxit=2)                 # graph capture, untimed
        x.zero_()
        ranks.barrier()
        with cs.timed():
            t0 = time.perf_counter()
            _, iters, relres, ok = h.solve(rhs, x, tol=1e-10, maxit=args.maxit_vcycle)
            torch.cuda.synchronize()
            t_solve = ranks.max(time.perf_counter() - t0)
        # flexible CG preconditioned by the same cycle
        t0 = time.perf_counter()
        hf = bmg.Hierarchy(kind, coef, arith=args.arith, periodic=spec["axes"], krylov="fcg")
        torch.cuda.synchronize()
        setup_fcg_ms = (time.perf_counter() - t0) * 1e3
        x.zero_()
        hf.solve(rhs, x, tol=1e-10, maxit=2)                # graph capture, untimed
        x.zero_()
        ranks.barrier()
        with cs.timed():
            t0 = time.perf_counter()
            _, iters_f, relres_f, ok_f = hf.solve(rhs, x, tol=1e-10, maxit=args.maxit_vcycle)
            torch.cuda.synchronize()
            t_fcg = ranks.max(time.perf_counter() - t0)
    clocks = cs.summary()
    # end to end through the public API with host buffers (FCG, as the Dirichlet bench line)
    rhs_host = torch.from_numpy(f).pin_memory()
    x_host = torch.empty_like(rhs_host).pin_memory()
    rhs_dev, x_dev = torch.empty_like(rhs), torch.empty_like(rhs)
    e2e_cycles = 0
    rhs_dev.copy_(rhs_host, non_blocking=True)          # one untimed step: the graph for these buffers
    x_dev.zero_()
    hf.solve(rhs_dev, x_dev, tol=1e-10, maxit=args.maxit_vcycle)
    torch.cuda.synchronize()
    ranks.barrier()
    t0 = time.perf_counter()
    for _ in range(2):
        rhs_dev.copy_(rhs_host, non_blocking=True)
        x_dev.zero_()
        _, it, _, _ = hf.solve(rhs_dev, x_dev, tol=1e-10, maxit=args.maxit_vcycle)
        x_host.copy_(x_dev, non_blocking=True)
        torch.cuda.synchronize()
        e2e_cycles += it
    e2e_s = ranks.max(time.perf_counter() - t0)
    hf.close()
    levels = h.num_levels
    sweep_kind = {bmg.TILE_SWEEP: "strip", 1: "rows", 0: "direct"}
    sweep_by_level = [sweep_kind[h.tuned_cluster(l)] for l in range(levels)]
    h.close()
    if rank != 0:
        ranks.close()
        return
    hbm_peak = measured_peak("hbm_gbs", 6800.0)
    relax0 = [r for r in prof if r["kernel"] == "relax" and r["level"] == 0][0]
    sweeps = 3 * 3                                            # V(2,1), three profiled cycles
    per_sweep_s = relax0["ms"] / sweeps * 1e-3
    byt = SWEEP_BYTES[("fp64", kind)] * N
    gbs = byt / per_sweep_s / 1e9
    instr_pt = ALG_FP64_INSTR_PER_POINT[(kind, args.arith)]
    out = {"metric": METRIC, "value": whole_job_rate(N * args.steps, ms * 1e-3, ranks), "unit": UNIT,
           "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic (seeded generators, no datasets)",
           "config": {"workload": args.workload, "description": spec["text"], "unknowns": N, "arith": args.arith,
                      "levels": levels, "parallelism": "replicas" if world > 1 else "single GPU",
                      "l2": "working set > L2 (FP64 level-0 stencil + vectors = %.0f MB)" % (N * 64 / 1e6)},
           "roofline": {"bound": "hbm", "kernel": "k_p_gs_strip level 0 (one-pass strip walk, one launch per sweep)",
                        "achieved": round(gbs, 1), "peak": hbm_peak[0], "unit": "GB/s",
                        "frac": round(gbs / hbm_peak[0], 4), "peak_source": hbm_peak[1], "traffic": None,
                        "traffic_source": None, "alg_bytes_per_sweep": byt,
                        "alg_bytes_per_point": SWEEP_BYTES[("fp64", kind)],
                        "fp64_pipe": {"achieved": round(instr_pt * N / per_sweep_s / 1e12, 4),
                                      "peak": round(fp64_rate / 1e12, 4), "unit": "T FP64 instr/s",
                                      "frac": round(instr_pt * N / per_sweep_s / fp64_rate, 4),
                                      "instr_per_point": instr_pt,
                                      "peak_source": "FP64 instruction rate measured in this run "
                                                     "(bmg_measure_fp64_rate)"},
                        "time_share": round(relax0["ms"] / sum(q["ms"] for q in prof), 3),
                        "avg_sweep_us": round(per_sweep_s * 1e6, 2)},
           "e2e": {"value": world * N * e2e_cycles / e2e_s, "unit": UNIT, "h2d_bytes_per_step": int(f.nbytes),
                   "d2h_bytes_per_step": int(f.nbytes),
                   "note": "bmg_solve (FP64, flexible CG, one V(2,1) per iteration) to 1e-10 from a zero guess "
                           "per step; rhs H2D from pinned memory, x D2H"},
           "gpu_launches": int(launches), "clocks": clocks, "sweep_by_level": sweep_by_level,
           "time_to_tol": {"fp64": {"setup_ms": round(setup_ms, 1),
                                    "vcycle": dict(solve_ms=round(t_solve * 1e3, 3), iterations=iters, relres=relres,
                                                   converged=ok),
                                    "fcg": dict(solve_ms=round(t_fcg * 1e3, 3), iterations=iters_f, relres=relres_f,
                                                converged=ok_f, setup_ms=round(setup_fcg_ms, 1))}},
           "profile_per_cycle_us": sorted(([r["level"], r["kernel"], round(r["launches"] / 3),
                                            round(r["ms"] / 3 * 1e3, 1)] for r in prof), key=lambda e: -e[3])}
    out["cpu_baseline"] = periodic_cpu_baseline(args, kind, planes, f, px, py) if not args.no_cpu and world == 1 \
        else None
    print(json.dumps(out))
    ranks.close()


def periodic_cpu_baseline(args, kind, planes, f, px, py):
    """The periodic oracle on one host thread: setup, then one V(2,1) cycle +
    residual norm on the full problem (a bounded sample)."""
    _, times, _ = periodic_oracle_cycles(kind, planes, f, px, py, 1)
    return {"value": f[1:-1, 1:-1].size / times[0], "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"periodic oracle (numpy FP64, one thread): setup + 1 V(2,1) cycle with residual norm on the "
                      f"full {args.workload} problem; cycle {times[0] * 1e3:.0f} ms"}


def periodic_oracle_cycles(kind, planes, f, px, py, cycles):
    from oracle import boxmg as bx
    from oracle import periodic as pr
    t0 = time.perf_counter()
    levels = pr.setup(kind, planes, px, py)
    setup_s = time.perf_counter() - t0
    x = np.zeros_like(f)
    times = []
    for _ in range(cycles):
        t0 = time.perf_counter()
        pr.vcycle(levels, 0, x, f)
        bx.norm(pr.residual(levels[0].planes, x, f, px, py))
        times.append(time.perf_counter() - t0)
    return setup_s, times, levels


def run_rhs_batch(args, rank, local_rank, world):
    """Many right-hand sides of one operator: one batch sharing the hierarchy
    (bmg_batch_rhs) against the same hierarchy solving them one at a time."""
    import torch
    import paper_2502_05279_gb300 as bmg
    torch.cuda.set_device(local_rank)
    ranks = Ranks("nccl")
    RHS_BATCH = RHS_BATCHES[args.workload]
    n, k = RHS_BATCH["n"], RHS_BATCH["k"]
    kind, planes, _ = w.lognormal_problem(n, 2.0, 32.0, seed_k=4, seed_f=7)
    coef = torch.from_numpy(planes).cuda()
    rhs = [torch.from_numpy(w.rhs_uniform(n, 500 + q)).cuda() for q in range(k)]
    N = n * n * k
    out = {"metric": METRIC, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "data": "synthetic (seeded generators)",
           "config": {"workload": args.workload, "description": RHS_BATCH["text"], "unknowns": N,
                      "parallelism": "replicas" if world > 1 else "single GPU"}, "variants": {}}
    clock_s = None
    for prec in ("fp64", "fp32"):
        h = bmg.Hierarchy(kind, coef, precision=prec, arith=args.arith)
        B = bmg.Batch.from_hierarchy(h, k)
        xs = [torch.zeros_like(r) for r in rhs]
        B.time_cycles(rhs, xs, max(args.warmup, 3))
        ranks.barrier()
        before = B.launch_count
        if prec == "fp64":
            with ClockSampler(local_rank) as cs:
                with cs.timed():
                    ms = B.time_cycles(rhs, xs, args.steps)
            clock_s = cs.summary()
        else:
            ms = B.time_cycles(rhs, xs, args.steps)
        launches = B.launch_count - before
        x1 = torch.zeros_like(rhs[0])
        h.time_cycles(rhs[0], x1, max(args.warmup, 3))
        ms_solo = h.time_cycles(rhs[0], x1, args.steps)       # one right-hand side
        for x in xs:
            x.zero_()
        ranks.barrier()
        t0 = time.perf_counter()
        _, its, _, ok = B.solve(rhs, xs, tol=1e-10, maxit=300)
        torch.cuda.synchronize()
        tb = time.perf_counter() - t0
        t0 = time.perf_counter()
        its_solo = []
        for r in rhs:
            _, it, _, _ = h.solve(r, torch.zeros_like(r), tol=1e-10, maxit=300)
            its_solo.append(it)
        torch.cuda.synchronize()
        ts = time.perf_counter() - t0
        # the same batch with one right-hand side per warp in the one-pass sweeps
        Boff = bmg.Batch.from_hierarchy(h, k, rhs_block="off")
        xs_off = [torch.zeros_like(r) for r in rhs]
        Boff.time_cycles(rhs, xs_off, max(args.warmup, 3))
        ms_off = Boff.time_cycles(rhs, xs_off, args.steps)
        Boff.close()
        out["variants"][prec] = {
            "value": whole_job_rate(N * args.steps, ms * 1e-3, ranks), "ms_per_step": ms / args.steps,
            "ms_per_step_one_rhs_per_warp": ms_off / args.steps,
            "solo_value": n * n * args.steps / (ms_solo * 1e-3), "solo_ms_per_step_one_rhs": ms_solo / args.steps,
            "gpu_launches": launches, "time_to_1e-10_all_ms": round(tb * 1e3, 1),
            "time_to_1e-10_one_by_one_ms": round(ts * 1e3, 1), "iterations_max": max(its),
            "same_iterations_as_solo": list(its) == its_solo, "all_converged": ok}
        B.close()
        h.close()
    v = out["variants"].pop("fp64")
    out.update(value=v["value"], ms_per_step=v["ms_per_step"], gpu_launches=int(v.pop("gpu_launches")), dtype="f64",
               clocks=clock_s, fp64=v)
    if rank == 0:
        print(json.dumps(out))
    ranks.close()


def dist_info():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)), int(os.environ.get("WORLD_SIZE", 1))


class Ranks:
    """Rank bookkeeping of an N-process run (one process per GPU, launched by
    torchrun): a barrier around every timed region and max/sum over ranks.
    The process group (NCCL on GPUs, gloo in the CPU tests) carries only these
    scalars; no solver data crosses ranks."""

    def __init__(self, backend: str = "nccl"):
        import torch
        self.torch = torch
        self.rank, self.local_rank, self.world = dist_info()
        self.cuda = backend == "nccl"
        self.dist = None
        if self.world > 1:
            import torch.distributed as dist
            if not dist.is_initialized():
                dist.init_process_group(backend)
            self.dist = dist

    def barrier(self):
        if self.cuda:
            self.torch.cuda.synchronize()
        if self.dist:
            self.dist.barrier()

    def _reduce(self, v: float, op) -> float:
        if not self.dist:
            return float(v)
        t = self.torch.tensor([float(v)], dtype=self.torch.float64, device="cuda" if self.cuda else "cpu")
        self.dist.all_reduce(t, op=op)
        return float(t.item())

    def max(self, v: float) -> float:
        return self._reduce(v, self.dist.ReduceOp.MAX if self.dist else None)

    def sum(self, v: float) -> float:
        return self._reduce(v, self.dist.ReduceOp.SUM if self.dist else None)

    def close(self):
        if self.dist:
            self.dist.destroy_process_group()
            self.dist = None


def batched_shard(rank: int, per_rank: int = 256):
    """Weak scaling of the batched workload: rank r solves problems
    [r * per_rank, (r + 1) * per_rank) of one seeded sequence, so rank 0 of
    any run solves the single-GPU batch."""
    return rank * per_rank, per_rank


def whole_job_rate(units_this_rank: float, seconds_this_rank: float, ranks: "Ranks") -> float:
    """Units processed by all ranks / the slowest rank's time."""
    return ranks.sum(units_this_rank) / ranks.max(seconds_this_rank)


# ----------------------------------------------------------------------------------
# clocks
# ----------------------------------------------------------------------------------

class ClockSampler:
    """nvidia-smi clocks and throttle reasons every 50 ms in the background;
    only samples that arrive while a timed region is open (timed() context)
    enter the summary."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.windows = []
        self.reader = None

    def __enter__(self):
        import threading
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
            return self

        def read():
            for line in self.proc.stdout:
                self.lines.append((time.perf_counter(), line))
        self.reader = threading.Thread(target=read, daemon=True)
        self.reader.start()
        return self

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            if self.reader:
                self.reader.join(timeout=5)
        return False

    class _Window:
        def __init__(self, owner):
            self.owner = owner

        def __enter__(self):
            self.t0 = time.perf_counter()

        def __exit__(self, *exc):
            self.owner.windows.append((self.t0, time.perf_counter()))
            return False

    def timed(self):
        return ClockSampler._Window(self)

    def summary(self):
        if not self.proc:
            return None
        sms, mx, reasons = [], None, set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for t, line in list(self.lines):
            if not any(a <= t <= b for a, b in self.windows):
                continue
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sms.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sms:
            return None
        return {"sm_mhz": statistics.median(sms), "sm_max_mhz": mx, "samples": len(sms), "reasons": sorted(reasons),
                "timed_regions_s": round(sum(b - a for a, b in self.windows), 3)}


# ----------------------------------------------------------------------------------
# the CUDA path
# ----------------------------------------------------------------------------------

# FP64 instructions of one Gauss-Seidel update: rounded, (k-1) mul + (k-1) sub + 1 mul;
# fused, (k-1) fma + 1 mul
ALG_FP64_INSTR_PER_POINT = {(5, "rounded"): 9, (9, "rounded"): 17, (5, "fused"): 5, (9, "fused"): 9}
SWEEP_BYTES = {("fp64", 9): 64, ("fp64", 5): 48, ("fp32", 9): 32, ("fp32", 5): 24, ("bf16", 9): 24, ("bf16", 5): 20}
# Two sweeps + residual + restriction in one pass, per fine point: the stencil with both a_O and 1/a_O
# (FP32: 6 x 4 B; BF16: 2 x 4 + 4 x 2 B), f, x read and written, the eight weights of a coarse point
# (8 x 4 B per 4 fine points) and the coarse right-hand side and iterate written (2 x 4 B per 4).
PAIR_RESTRICT_BYTES = {"fp32": 24 + 4 + 8 + 8 + 2, "bf16": 16 + 4 + 8 + 8 + 2}


def run_ours(args, rank, local_rank, world):
    import torch
    import paper_2502_05279_gb300 as bmg
    torch.cuda.set_device(local_rank)
    ranks = Ranks("nccl")
    spec = WORKLOADS[args.workload]
    kind, planes, f = spec["make"]()
    n = planes.shape[-1] - 2
    N = n * n
    coef = torch.from_numpy(planes if kind == 9 else planes[:3].copy()).cuda()
    rhs = torch.from_numpy(f).cuda()
    barrier = ranks.barrier
    max_over_ranks = ranks.max

    if args.only:
        # one hierarchy, warm-up and timed cycles only: the small run profiled by ncu
        h = bmg.Hierarchy(kind, coef, precision=args.only, krylov=args.krylov, smoother=args.smoother,
                          arith=args.arith, fuse_restrict=args.fuse_restrict)
        x = torch.zeros_like(rhs)
        h.time_cycles(rhs, x, args.warmup)
        ms = h.time_cycles(rhs, x, args.steps)
        if rank == 0:
            print(json.dumps({"only": args.only, "krylov": args.krylov, "arith": args.arith,
                              "workload": args.workload, "ms_per_step": ms / args.steps,
                              "launches": h.launch_count}))
        h.close()
        return

    variants = {}
    timed_launches = 0
    fp64_rate = bmg.measure_fp64_rate() * 1e9        # DP instructions per second, measured here
    sampler = ClockSampler(local_rank).__enter__()
    for prec in ("fp64", "fp32", "bf16"):
        barrier()
        t0 = time.perf_counter()
        h = bmg.Hierarchy(kind, coef, precision=prec, arith=args.arith)
        torch.cuda.synchronize()
        setup_ms = (time.perf_counter() - t0) * 1e3
        x = torch.zeros_like(rhs)
        h.time_cycles(rhs, x, max(args.warmup, 3))
        barrier()
        before = h.launch_count
        with sampler.timed():
            ms = h.time_cycles(rhs, x, args.steps)
        if prec == "fp64":
            timed_launches = h.launch_count - before
        barrier()
        ms = max_over_ranks(ms)
        prof = h.profile(rhs, torch.zeros_like(rhs), 3)
        # time to tolerance from a zero guess (host-timed: includes the host polls),
        # stationary cycles and flexible CG with the same cycle as preconditioner
        tts = {}
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        hk = bmg.Hierarchy(kind, coef, precision=prec, krylov="fcg", arith=args.arith)
        torch.cuda.synchronize()
        setup_tuned_ms = (time.perf_counter() - t0) * 1e3      # the tuners' decisions already made

        modes = [("vcycle", h, args.maxit_vcycle), ("fcg", hk, 500)]
        hk2 = None
        if prec != "fp64":   # two FP32 cycles per FP64 outer step amortise the FP64-bound outer work
            hk2 = bmg.Hierarchy(kind, coef, precision=prec, krylov="fcg", inner_cycles=2, arith=args.arith)
            modes.append(("fcg_2cycles", hk2, 500))
        for mode, hh, cap in modes:
            x.zero_()
            hh.solve(rhs, x, tol=1e-10, maxit=2)                 # graph capture and first launches, untimed
            x.zero_()
            barrier()
            with sampler.timed():
                t0 = time.perf_counter()
                _, iters, relres, ok = hh.solve(rhs, x, tol=1e-10, maxit=cap)
                torch.cuda.synchronize()
                t1 = time.perf_counter()
            tts[mode] = dict(solve_ms=round(max_over_ranks((t1 - t0) * 1e3), 3), iterations=iters,
                             relres=relres, converged=ok)
        if hk2 is not None:
            hk2.close()
        variants[prec] = dict(ms=ms, setup_ms=setup_ms, setup_tuned_ms=setup_tuned_ms, tts=tts, prof=prof, h=h, hk=hk,
                              tuned=[h.tuned_cluster(l) for l in range(h.num_levels)],
                              pairs=[h.tuned_pair(l) for l in range(h.num_levels)])
    sampler.__exit__(None, None, None)
    clock_s = sampler.summary()

    # the FP64 cycle in the other arithmetic mode, for comparison (cycle time and profile only)
    other = "rounded" if args.arith == "fused" else "fused"
    ho = bmg.Hierarchy(kind, coef, precision="fp64", arith=other)
    xo = torch.zeros_like(rhs)
    ho.time_cycles(rhs, xo, max(args.warmup, 3))
    barrier()
    ms_other = max_over_ranks(ho.time_cycles(rhs, xo, args.steps))
    prof_other = ho.profile(rhs, torch.zeros_like(rhs), 3)
    tuned_other = [ho.tuned_cluster(l) for l in range(ho.num_levels)]
    ho.close()

    # end to end through the public API with host buffers (FP64 path, flexible CG to 1e-10)
    h = variants["fp64"]["hk"]
    rhs_host = torch.from_numpy(f).pin_memory()
    x_host = torch.empty_like(rhs_host).pin_memory()
    rhs_dev = torch.empty_like(rhs)
    x_dev = torch.empty_like(rhs)
    e2e_steps = 2
    e2e_cycles = 0
    # one untimed step: the solve's graph is captured for these buffers (a warm-up, as for the
    # device-timed steps); every timed step still copies its inputs in and its result out
    rhs_dev.copy_(rhs_host, non_blocking=True)
    x_dev.zero_()
    h.solve(rhs_dev, x_dev, tol=1e-10, maxit=500)
    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        rhs_dev.copy_(rhs_host, non_blocking=True)
        x_dev.zero_()
        _, it, _, _ = h.solve(rhs_dev, x_dev, tol=1e-10, maxit=500)
        x_host.copy_(x_dev, non_blocking=True)
        torch.cuda.synchronize()
        e2e_cycles += it
    e2e_s = max_over_ranks(time.perf_counter() - t0)

    if rank != 0:
        ranks.close()
        return

    def dominant(prof, fp32):
        rows = [r for r in prof if r["kernel"] == "relax" and r["level"] == 0 and r["fp32"] == fp32]
        return rows[0] if rows else max(prof, key=lambda r: r["ms"])

    sweeps_per_cycle = 3                                        # V(2,1)
    hbm_peak = measured_peak("hbm_gbs", 6800.0)

    def per_launch(prec, fp32, prof=None):
        """Dominant kernel's average device time per launch and the Gauss-Seidel
        sweeps one launch performs (1/2 for the row kernel, 1 for the tile kernel)."""
        r = dominant(variants[prec]["prof"] if prof is None else prof, fp32)
        cycles = 3
        return r, r["ms"] / r["launches"] * 1e-3, sweeps_per_cycle * cycles / r["launches"]

    def traffic(name, sweeps):
        """DRAM bytes of one launch: the captured bytes per fine point (of a
        launch of the same kernel and shape) x the level's unknowns."""
        got = NCU_DRAM_BYTES_PER_POINT.get(name)
        if got is None:
            return None, None
        return round(got[0] * N), f"ncu capture on {got[1]}, {got[0]:.2f} B per fine point, x {N} points"

    def roofline_fp64(arith, prof, tuned):
        """The FP64 sweep against both roofs: its algorithmic bytes against the
        measured HBM copy bandwidth (the headline fraction) and its useful
        FP64 instructions against the measured FP64 instruction rate (the roof
        that binds it on this GPU)."""
        r, per_launch_s, sweeps = per_launch("fp64", False, prof)
        instr = ALG_FP64_INSTR_PER_POINT[(kind, arith)] * N * sweeps
        byt = SWEEP_BYTES[("fp64", kind)] * N * sweeps
        share = r["ms"] / sum(q["ms"] for q in prof)
        name = (f"k_gs_strip64 {TILE64_SHAPES[tuned[0] - 16]}" if tuned[0] >= 16 else "k_gs_rows<double>") + \
            (" fused" if arith == "fused" else "")
        gbs = byt / per_launch_s / 1e9
        tr, tr_src = traffic(name, sweeps)
        return {"bound": "hbm", "kernel": f"{name} level 0 ({'half ' if sweeps < 1 else ''}sweep per launch)",
                "achieved": round(gbs, 1), "peak": hbm_peak[0], "unit": "GB/s", "frac": round(gbs / hbm_peak[0], 4),
                "peak_source": hbm_peak[1], "traffic": tr, "traffic_source": tr_src,
                "alg_bytes_per_launch": byt, "alg_bytes_per_point": SWEEP_BYTES[("fp64", kind)],
                "fp64_pipe": {"achieved": round(instr / per_launch_s / 1e12, 4), "peak": round(fp64_rate / 1e12, 4),
                              "unit": "T FP64 instr/s", "frac": round(instr / per_launch_s / fp64_rate, 4),
                              "instr_per_point": ALG_FP64_INSTR_PER_POINT[(kind, arith)],
                              "peak_source": "FP64 instruction rate measured in this run (bmg_measure_fp64_rate)"},
                "time_share": round(share, 3), "avg_launch_us": round(per_launch_s * 1e6, 2)}

    def roofline_32(prec):
        """Dominant FP32 sweep kernel of level 0: the two-sweep pass when the
        autotuner chose it (its algorithmic bytes are one read of the level's
        arrays and one write of x for two sweeps), else the one-pass or row
        kernel (one sweep's bytes per sweep it performs)."""
        prof = variants[prec]["prof"]
        st = "bf16" if prec == "bf16" else "float"
        pair = [q for q in prof if q["kernel"] == "relax_pair" and q["level"] == 0 and q["fp32"]]
        fused = [q for q in prof if q["kernel"] == "pair_restrict" and q["level"] == 0 and q["fp32"]]
        if fused:
            r = fused[0]
            sweeps = 2.0
            byt = PAIR_RESTRICT_BYTES[prec] * N
            name = f"k_gs_strip2r_ring<{st}> 44xW bulk/{4 if variants[prec]['pairs'][0] != 1 else 6}"
        elif pair:
            r = pair[0]
            sweeps = 2.0
            byt = SWEEP_BYTES[(prec, kind)] * N
            name = f"k_gs_strip2_ring<{st}> {PAIR_SHAPES[variants[prec]['pairs'][0]]}"
        else:
            r, _, sweeps = per_launch(prec, True)
            byt = SWEEP_BYTES[(prec, kind)] * N * sweeps
            tuned = variants[prec]["tuned"][0]
            name = (f"k_gs_strip<{st}> {TILE_SHAPES[tuned - 16]}" if tuned >= 16 else f"k_gs_rows<float,{st}>")
        per_launch_s = r["ms"] / r["launches"] * 1e-3
        achieved = byt / per_launch_s / 1e9
        share = r["ms"] / sum(q["ms"] for q in prof)
        what = ("two sweeps + residual + restriction" if fused else "two sweeps") if sweeps == 2.0 else \
            ("half sweep" if sweeps < 1 else "sweep")
        tr, tr_src = traffic(name, sweeps)
        return {"bound": "hbm", "kernel": f"{name} level 0 ({what} per launch)",
                "achieved": round(achieved, 1), "peak": hbm_peak[0], "unit": "GB/s",
                "frac": round(achieved / hbm_peak[0], 4), "peak_source": hbm_peak[1], "traffic": tr,
                "traffic_source": tr_src, "alg_bytes_per_launch": byt, "sweeps_per_launch": sweeps,
                "per_sweep_equiv_gbs": round(SWEEP_BYTES[(prec, kind)] * N * sweeps / per_launch_s / 1e9, 1),
                "time_share": round(share, 3), "avg_launch_us": round(per_launch_s * 1e6, 2)}

    v64 = variants["fp64"]
    value = world * N * args.steps / (v64["ms"] * 1e-3)
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": v64["ms"] / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic (seeded generators, no datasets)",
        "config": {"workload": args.workload, "description": spec["text"], "unknowns": N, "arith": args.arith,
                   "levels": v64["h"].num_levels, "parallelism": "replicas" if world > 1 else "single GPU",
                   "l2": "working set > L2 (FP64 level-0 stencil + vectors = %.0f MB)" % (N * 64 / 1e6)},
        "roofline": roofline_fp64(args.arith, v64["prof"], v64["tuned"]),
        "e2e": {"value": world * N * e2e_cycles / e2e_s, "unit": UNIT,
                "h2d_bytes_per_step": int(f.nbytes), "d2h_bytes_per_step": int(f.nbytes),
                "note": "bmg_solve (FP64, flexible CG, one V(2,1) per iteration) to 1e-10 from a zero guess per "
                        "step; rhs H2D from pinned memory, x D2H"},
        "gpu_launches": int(timed_launches),
        "clocks": clock_s,
        "time_to_tol": {p: dict(setup_ms=round(v["setup_ms"], 1), setup_ms_tuned=round(v["setup_tuned_ms"], 1),
                                **v["tts"]) for p, v in variants.items()},
        "variants": {**{p: {"value": world * N * args.steps / (v["ms"] * 1e-3), "ms_per_step": v["ms"] / args.steps,
                            "roofline": roofline_32(p), "tuned_cluster_by_level": v["tuned"],
                            "two_sweep_pass_by_level": v["pairs"]}
                        for p, v in variants.items() if p != "fp64"},
                     "fp64_" + other: {"value": world * N * args.steps / (ms_other * 1e-3),
                                       "ms_per_step": ms_other / args.steps,
                                       "roofline": roofline_fp64(other, prof_other, tuned_other),
                                       "tuned_cluster_by_level": tuned_other}},
        "tuned_cluster_by_level": variants["fp64"]["tuned"],
    }
    # per-level, per-kernel device time of one cycle (the paper's Fig. 10 breakdown)
    out["profile_per_cycle_us"] = {
        p: sorted(([r["level"], r["kernel"] + ("32" if r["fp32"] else ""), round(r["launches"] / 3), round(r["ms"] / 3 * 1e3, 1)]
                   for r in v["prof"]), key=lambda e: -e[3])
        for p, v in variants.items()}
    if args.workload == "learned4095":
        out["variants"]["learned"] = learned_variant(args, kind, coef, rhs, n, N, world)
    for v in variants.values():
        v["h"].close()
        v["hk"].close()
    out["cpu_baseline"] = cpu_baseline(args, kind, planes, f) if not args.no_cpu and world == 1 else None
    print(json.dumps(out))
    ranks.close()


def learned_variant(args, kind, coef, rhs, n, N, world):
    """Train the network on the GPU (two-grid loss on 31^2 crops of the 255^2
    family), then set up the evaluation problem with it: bmg_setup measures the
    learned and the Dendy V(2,1) factors and keeps the better; report both,
    the training and setup times, flexible-CG time to 1e-10 (or the residual
    reached) and the cycle rate of the hierarchy the setup kept."""
    import torch
    import paper_2502_05279_gb300 as bmg
    from paper_2502_05279_gb300 import learned_training as lt
    t0 = time.perf_counter()
    mlp, hist, _, train_s = lt.train(n_problems=args.learned_problems, epochs=args.learned_epochs, batch=152,
                                     log=lambda *_: None)
    prep_train_s = time.perf_counter() - t0
    ev = lt.evaluate(mlp, n=n, seed=6, tol=1e-10, maxit=500)
    h = bmg.Hierarchy(kind, coef, mlp=mlp, arith=args.arith)
    x = torch.zeros_like(rhs)
    h.time_cycles(rhs, x, max(args.warmup, 3))
    ms = h.time_cycles(rhs, x, args.steps)
    used = h.interp_info()[0]
    h.close()
    mlp.close()
    return {"value": world * N * args.steps / (ms * 1e-3), "ms_per_step": ms / args.steps, "kept": used,
            "train": {"problems": args.learned_problems, "crops": args.learned_problems, "epochs": args.learned_epochs,
                      "two_grid_loss_by_epoch": hist, "train_s": round(train_s, 3),
                      "prepare_and_train_s": round(prep_train_s, 2)},
            "evaluation": ev}


def measured_peak(key, fallback):
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)[key]), "MEASURED_PEAKS.json (measured)"
    except (OSError, KeyError, ValueError):
        return fallback, "fallback"


# ----------------------------------------------------------------------------------
# the CPU oracle (baseline and reference arm)
# ----------------------------------------------------------------------------------

def host_cores() -> int:
    """Host cores this process may run on."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_cycles(kind, planes, f, cycles, threads=1, levels=None):
    """Oracle setup (unless given), then `cycles` V(2,1) cycles each followed
    by the residual norm, the colour passes and residuals over row bands on
    `threads` host threads (bit for bit the one-thread cycle); returns
    (setup_s, per-cycle seconds, levels)."""
    from oracle import boxmg as bx
    t0 = time.perf_counter()
    if levels is None:
        levels = bx.setup(kind, planes)
    setup_s = time.perf_counter() - t0
    bands = bx.RowBands(threads)
    x = np.zeros_like(f)
    times = []
    try:
        for _ in range(cycles):
            t0 = time.perf_counter()
            bx.vcycle(levels, 0, x, f, bands=bands)
            bx.norm(bx.residual(levels[0].planes, x, f, bands=bands))
            times.append(time.perf_counter() - t0)
    finally:
        bands.close()
    return setup_s, times, levels


def cpu_baseline(args, kind, planes, f):
    """The oracle on the host cores, all of them and one: one setup, then the
    same V(2,1) cycle + residual norm on the full problem (a bounded sample:
    one or a few cycles per leg)."""
    n = planes.shape[-1] - 2
    cores = host_cores()
    cycles = 1 if n >= 4095 else (3 if n >= 2047 else 20)
    setup_s, t_all, levels = oracle_cycles(kind, planes, f, cycles, threads=cores)
    _, t_one, _ = oracle_cycles(kind, planes, f, cycles, threads=1, levels=levels)
    per_all, per_one = statistics.median(t_all), statistics.median(t_one)
    return {"value": n * n / per_all, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"oracle (numpy FP64; colour passes and residuals over row bands on {cores} threads, the same "
                      f"bits as one) setup ({setup_s:.1f} s, one thread) + {cycles} V(2,1) cycle(s) with residual "
                      f"norm on the full {args.workload} problem per leg; median cycle {per_all * 1e3:.0f} ms on "
                      f"{cores} cores, {per_one * 1e3:.0f} ms on one",
            "one_thread": {"value": n * n / per_one, "unit": UNIT, "cores": 1}}


BATCH_SAMPLE_UNKNOWNS = 2_500_000


def batch_sample(probs, budget: int = BATCH_SAMPLE_UNKNOWNS):
    """The leading problems of a batch whose unknowns add up to at most
    `budget` (at least one problem): the bounded CPU sample of the batch."""
    out, tot = [], 0
    for p in probs:
        m = (p[1].shape[-1] - 2) ** 2
        if out and tot + m > budget:
            break
        out.append(p)
        tot += m
    return out, tot


def oracle_batch_cycles(probs, cycles, threads=1, hier=None):
    """Oracle setup of every problem (unless given), then `cycles` rounds of
    one V(2,1) cycle plus residual norm on each, the colour passes and
    residuals over row bands on `threads` host threads; returns (setup_s,
    per-round seconds, hierarchies)."""
    from oracle import boxmg as bx
    t0 = time.perf_counter()
    if hier is None:
        hier = [(bx.setup(k, pl), f) for k, pl, f in probs]
    setup_s = time.perf_counter() - t0
    bands = bx.RowBands(threads)
    xs = [np.zeros_like(f) for _, f in hier]
    times = []
    try:
        for _ in range(cycles):
            t0 = time.perf_counter()
            for (levels, f), x in zip(hier, xs):
                bx.vcycle(levels, 0, x, f, bands=bands)
                bx.norm(bx.residual(levels[0].planes, x, f, bands=bands))
            times.append(time.perf_counter() - t0)
    finally:
        bands.close()
    return setup_s, times, hier


def batched_cpu_baseline(probs):
    sample, m = batch_sample(probs)
    cores = host_cores()
    setup_s, t_all, hier = oracle_batch_cycles(sample, 3, threads=cores)
    _, t_one, _ = oracle_batch_cycles(sample, 3, threads=1, hier=hier)
    per_all, per_one = statistics.median(t_all), statistics.median(t_one)
    return {"value": m / per_all, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"oracle (numpy FP64; colour passes and residuals over row bands on {cores} threads): setup "
                      f"({setup_s:.1f} s) + 3 rounds of one V(2,1) cycle with residual norm on the first "
                      f"{len(sample)} problems of the batch ({m} unknowns) per leg; median round "
                      f"{per_all * 1e3:.0f} ms on {cores} cores, {per_one * 1e3:.0f} ms on one",
            "one_thread": {"value": m / per_one, "unit": UNIT, "cores": 1}}


def run_reference(args, rank, world):
    if rank != 0:
        return
    warm = min(args.warmup, 1)
    cores = host_cores()
    if args.workload == "batched256":
        sample, m = batch_sample(w.batched_problems(256, 5, 1.0, 32.0))
        steps = min(args.steps, 5)
        setup_s, times, _ = oracle_batch_cycles(sample, steps + warm, threads=cores)
        text, unknowns = BATCHED["text"], m
        what = f"the first {len(sample)} problems of the batch ({m} unknowns)"
    elif args.workload in PERIODIC:
        spec = PERIODIC[args.workload]
        kind, planes, f, px, py = w.periodic_problem(spec["n"], spec["axes"], seed_k=50, seed_f=51)
        steps = min(args.steps, 2)
        setup_s, times, _ = periodic_oracle_cycles(kind, planes, f, px, py, steps + warm)
        cores = 1
        text, unknowns = spec["text"], f[1:-1, 1:-1].size
        what = f"the full {args.workload} problem (one thread: the periodic oracle has no row-band runner)"
    elif args.workload in RHS_BATCHES:
        RHS_BATCH = RHS_BATCHES[args.workload]
        n = RHS_BATCH["n"]
        kind, planes, _ = w.lognormal_problem(n, 2.0, 32.0, seed_k=4, seed_f=7)
        sample = [(kind, planes, w.rhs_uniform(n, 500 + q)) for q in range(2)]
        steps = min(args.steps, 2 if n >= 4095 else 5)
        setup_s, times, _ = oracle_batch_cycles(sample, steps + warm, threads=cores)
        text, unknowns = RHS_BATCH["text"], 2 * n * n
        what = f"2 of the {RHS_BATCH['k']} right-hand sides (the operator set up once per right-hand side)"
    else:
        spec = WORKLOADS[args.workload]
        kind, planes, f = spec["make"]()
        n = planes.shape[-1] - 2
        steps = min(args.steps, 2 if n >= 4095 else (5 if n >= 2047 else 50))
        setup_s, times, _ = oracle_cycles(kind, planes, f, steps + warm, threads=cores)
        text, unknowns = spec["text"], n * n
        what = f"the full {args.workload} problem"
    times = times[warm:]
    tot = sum(times)
    value = unknowns * len(times) / tot
    spread = "one host thread" if cores == 1 else f"colour passes and residuals over row bands on {cores} host threads"
    sample = (f"{len(times)} timed V(2,1) cycles (+ {warm} warm-up) of the oracle on {what}, {spread} (steps capped "
              f"from {args.steps} to keep the CPU run to minutes); setup {setup_s:.1f} s")
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": len(times), "warmup": args.warmup,
           "ms_per_step": tot / len(times) * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f64", "data": "synthetic (seeded generators, no datasets)", "impl": "reference",
           "config": {"workload": args.workload, "description": text, "unknowns": unknowns},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD,
                    choices=sorted(WORKLOADS) + ["batched256"] + sorted(RHS_BATCHES) + sorted(PERIODIC))
    ap.add_argument("--impl", default="ours", choices=("ours", "reference"))
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-oracle baseline leg")
    ap.add_argument("--maxit-vcycle", type=int, default=200, help="cap of the stationary-cycle solve")
    ap.add_argument("--only", choices=("fp64", "fp32", "bf16"), default=None,
                    help="time one hierarchy's cycles only (short run for profilers)")
    ap.add_argument("--krylov", choices=("none", "fcg"), default="none", help="solve mode for --only")
    ap.add_argument("--smoother", default="auto", help="FP32 Gauss-Seidel kernel for --only (auto, rows, tile0..4)")
    ap.add_argument("--fuse-restrict", default="auto", choices=("auto", "off", "on"),
                    help="two sweeps + residual + restriction in one pass, for --only")
    ap.add_argument("--learned-problems", type=int, default=2000, help="training problems (one crop each)")
    ap.add_argument("--learned-epochs", type=int, default=8, help="training epochs of the learned variant")
    ap.add_argument("--arith", choices=("rounded", "fused"), default="fused",
                    help="cycle arithmetic: fused multiply-adds (default) or one rounding per operation")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    rank, local_rank, world = dist_info()
    if args.impl == "reference":
        run_reference(args, rank, world)
    elif args.workload == "batched256":
        run_batched(args, rank, local_rank, world)
    elif args.workload in RHS_BATCHES:
        run_rhs_batch(args, rank, local_rank, world)
    elif args.workload in PERIODIC:
        run_periodic(args, rank, local_rank, world)
    else:
        run_ours(args, rank, local_rank, world)


if __name__ == "__main__":
    main()
