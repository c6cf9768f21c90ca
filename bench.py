#!/usr/bin/env python
"""Benchmark of one Newton-step linear solve on a GB300.

A step is one pass of the whole hot path over the 128x128x64, b = 4 synthetic
thermal Jacobian (1,048,576 cells, 8 SAGD wells, 4,194,336 unknowns with the wells padded to b x b blocks):
transmissibility/Jacobian assembly on the GPU, full CPR-FPF setup (ABF
decoupling, pressure AMG, colouring, block ILU(0)), and FGMRES(30) to a true
FP64 relative residual of 1e-6 -- with the CPR stored and applied in FP32
(the default) or FP64 (--precision fp64).  value = device milliseconds per
step (lower is better), inputs resident in HBM.

Multi-GPU: the path is one system per GPU ("replicas"); every rank solves its
own copy and the step time is the maximum over ranks.

--impl reference times the CPU oracle (plain C, FP64, single thread) on a
bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {"16x16x4_b4": 0, "128x128x64_b4": 1, "256x256x128_b5": 2, "64x64x32_b4": 3,
             "512x256x64_b4": 4, "96x96x48_b4": None}


def make_workload(name):
    from paper_1812_03952_gb300 import synthetic as S
    if WORKLOADS[name] is None:      # mid-size case for profiler captures (matrix > L2, < 2 GB total)
        return S.small_system(96, 96, 48, 4, seed=77, sigma=1.5, n_pairs=4, kvkh=0.1, name=name)
    return S.config(WORKLOADS[name])
METRIC = "CPR-FGMRES solve ms (assembly + CPR setup + FGMRES to true rel. res. 1e-6)"
PEAKS_PATH = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM_GBS = 6800.0


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="trs", choices=["trs", "reference"])
    p.add_argument("--workload", default="128x128x64_b4", choices=sorted(WORKLOADS))
    p.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    p.add_argument("--rtol", type=float, default=1e-6)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-fp64-compare", action="store_true")
    p.add_argument("--sequence", type=int, default=0,
                   help="time a sequence of this many Newton-like systems (accumulation blocks rescaled by "
                        "seeded +-20%% factors, AMG hierarchy rebuilt every --reuse steps, forward and adjoint "
                        "solve per system) instead of single solves")
    p.add_argument("--reuse", type=int, default=5)
    p.add_argument("--decoupling", default="abf", choices=["abf", "none", "frs", "frs+abf"],
                   help="decoupling of the forward CPR")
    p.add_argument("--adjoint-decoupling", default="none", choices=["abf", "none", "frs", "frs+abf"],
                   help="decoupling of the CPR built on A^T for the adjoint solves")
    p.add_argument("--ilu-fill", type=int, default=0, choices=[0, 1],
                   help="level of fill of the block ILU stage (0: ILU(0), 1: ILU(1))")
    p.add_argument("--no-ilu-compare", action="store_true",
                   help="skip timing the other ILU level on the same system")
    p.add_argument("--restart", type=int, default=30, help="FGMRES restart length")
    p.add_argument("--cheb-degree", type=int, default=2, help="Chebyshev smoother degree")
    p.add_argument("--krylov", default="fgmres", choices=["fgmres", "bicgstab"],
                   help="outer Krylov method of the timed step")
    p.add_argument("--no-krylov-compare", action="store_true",
                   help="skip timing the other Krylov method on the same system")
    return p.parse_args()


# ----------------------------------------------------------------- helpers
class ClockSampler:
    """nvidia-smi clock / throttle samples while the timed region runs."""

    def __init__(self, index):
        self.index = index
        self.samples = []
        self.proc = None

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except FileNotFoundError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                self.samples.append(parts)

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        mx = [float(s[2]) for s in self.samples if s[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for s in self.samples for k in range(4) if s[5 + k] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.samples)}


def peaks():
    try:
        with open(PEAKS_PATH) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return FALLBACK_HBM_GBS, "fallback"


def dist_setup(n_gpus):
    import torch
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    return rank, world, local


def barrier_max(value, world):
    """Maximum of a per-rank value over all ranks (the step time of the
    slowest replica)."""
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


# ------------------------------------------------------------ oracle timing
def oracle_sample(sysm, n_iter, iters_full):
    """Times the CPU oracle on a bounded sample: assembly + CPR setup +
    n_iter FGMRES iterations, extrapolated to iters_full iterations."""
    from oracle import oracle as O
    O.build()
    t0 = time.perf_counter()
    Ao = O.assemble(sysm)
    t1 = time.perf_counter()
    cpr = O.CPR(Ao)
    t2 = time.perf_counter()
    res = O.fgmres(Ao, cpr, sysm.rhs, rtol=1e-30, maxit=n_iter)
    t3 = time.perf_counter()
    per_iter = (t3 - t2) / max(1, res.iters)
    est_ms = 1e3 * ((t1 - t0) + (t2 - t1) + per_iter * iters_full)
    return est_ms, {"assemble_s": t1 - t0, "setup_s": t2 - t1, "iter_s": per_iter, "iters_timed": res.iters,
                    "wall_s": t3 - t0}


# FGMRES iterations of the FP64 path on the 128x128x64 workload (the oracle
# runs the same algorithm; used to scale the oracle's bounded sample).
FULL_ITERS = {"128x128x64_b4": 12, "64x64x32_b4": 31, "16x16x4_b4": 18, "256x256x128_b5": 60,
              "512x256x64_b4": 60, "96x96x48_b4": 12}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from paper_1812_03952_gb300 import synthetic as S
    sysm = make_workload(args.workload)
    n_iter = 1
    times = []
    detail = None
    for step in range(args.warmup + args.steps):
        est, detail = oracle_sample(sysm, n_iter, FULL_ITERS[args.workload])
        if step >= args.warmup:
            times.append(est)
    value = statistics.median(times)
    sample = (f"oracle assembly + CPR setup + {n_iter} FGMRES iteration on the full {args.workload} system, "
              f"scaled to {FULL_ITERS[args.workload]} iterations")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "ms", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": value, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "precision": "fp64 (CPU oracle)", "rtol": args.rtol},
            "cpu_baseline": {"value": value, "unit": "ms", "cores": 1, "kind": "oracle", "sample": sample,
                             "detail": detail},
            "e2e": {"value": value, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------ Newton-like sequence
def run_sequence(args):
    """Total device time of a sequence of Newton-like systems: per system,
    accumulation blocks rescaled by seeded (1 + 0.2 u) factors, assembly, CPR refresh (full rebuild every
    args.reuse systems, AMG reused otherwise), forward solve, transpose,
    CPR on A^T (same reuse), adjoint solve and the dL/dtheta chain."""
    import torch
    from paper_1812_03952_gb300 import build as B
    from paper_1812_03952_gb300 import synthetic as S
    from paper_1812_03952_gb300 import trs
    B.build()
    trs.load()
    rank, world, local = dist_setup(args.gpus)
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream()
    sysm = make_workload(args.workload)
    ds = trs.DeviceSystem(sysm, dev)
    # per-system factors (1 + 0.2 u) on each cell's accumulation block: the
    # part of the diagonal block a Newton update of the state changes
    scales = torch.from_numpy(S.diagonal_scalings(sysm.n_cells, args.sequence, S.SEED_BASE + 99)).to(dev)
    acc0 = ds.acc.clone()
    bb = sysm.b * sysm.b
    g = torch.zeros(sysm.n_unknowns, dtype=torch.float64, device=dev)
    g[torch.from_numpy(np.unique(sysm.perf_cell).astype(np.int64) * sysm.b).to(dev)] = 1.0
    A = ds.assemble()
    M = trs.CPR(A, precision=args.precision, cheb_degree=args.cheb_degree, decoupling=args.decoupling,
                ilu_fill=args.ilu_fill)
    AT = A.transpose()
    MT = trs.CPR(AT, precision=args.precision, cheb_degree=args.cheb_degree, decoupling=args.adjoint_decoupling,
                 ilu_fill=args.ilu_fill)
    x = torch.zeros_like(ds.rhs)
    records = []

    def run_all(record):
        for k in range(args.sequence):
            torch.mul(acc0.view(-1, bb), scales[k].view(-1, 1), out=ds.acc.view(-1, bb))
            ds.assemble()
            reuse = (k % args.reuse) != 0
            M.update(A, reuse_amg=reuse)
            _, rf = trs.krylov_solve(args.krylov, A, M, ds.rhs, x, rtol=args.rtol, restart=args.restart)
            A.transpose(into=AT)
            MT.update(AT, reuse_amg=reuse)
            lam, _, ra = trs.solve_adjoint(A, AT, MT, g, x, rtol=args.rtol, restart=args.restart,
                                           method=args.krylov)
            trs.chain_theta(A, ds.k, ds.M, lam, x, sysm.kvkh, sysm.c_t)
            if record:
                records.append({"step": k, "amg": "reused" if reuse else "rebuilt",
                                "fwd_iters": rf.stats["iters"], "fwd_relres": rf.stats["true_relres"],
                                "adj_iters": ra.stats["iters"], "adj_relres": ra.stats["true_relres"],
                                "fwd_ms": rf.stats["ms_solve"], "adj_ms": ra.stats["ms_solve"]})

    for _ in range(max(1, args.warmup)):
        run_all(False)
    torch.cuda.synchronize()
    barrier(world)
    l0 = trs.kernel_launches()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        e0.record(stream)
        for _ in range(args.steps):
            records.clear()
            run_all(True)
        e1.record(stream)
        torch.cuda.synchronize()
    ms = barrier_max(e0.elapsed_time(e1) / args.steps, world)
    if rank == 0:
        line = {"metric": f"Newton-like sequence of {args.sequence} systems: forward + adjoint CPR-"
                          f"{args.krylov.upper()} total ms",
                "value": ms, "unit": "ms", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": ms, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
                "dtype": "f64+f32" if args.precision == "fp32" else "f64", "data": "synthetic",
                "config": {"workload": args.workload, "cells": sysm.n_cells, "b": sysm.b, "wells": sysm.n_wells,
                           "unknowns": sysm.n_unknowns, "systems": args.sequence, "amg_rebuild_every": args.reuse,
                           "rtol": args.rtol, "precision": args.precision,
                           "decoupling": args.decoupling, "adjoint_decoupling": args.adjoint_decoupling,
                           "restart": args.restart, "ilu_fill": args.ilu_fill,
                           "l2": "inputs larger than L2", "parallelism": "replicas" if world > 1 else "single GPU"},
                "per_system": records, "clocks": clk.summary(), "gpu_launches": trs.kernel_launches() - l0}
        print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------- GPU arm
def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.sequence:
        return run_sequence(args)
    import torch
    from paper_1812_03952_gb300 import build as B
    from paper_1812_03952_gb300 import synthetic as S
    from paper_1812_03952_gb300 import trs

    B.build()
    trs.load()
    rank, world, local = dist_setup(args.gpus)
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream()
    sysm = make_workload(args.workload)
    ds = trs.DeviceSystem(sysm, dev)
    A = ds.assemble()
    M = trs.CPR(A, precision=args.precision, cheb_degree=args.cheb_degree, decoupling=args.decoupling,
                ilu_fill=args.ilu_fill)
    x = torch.zeros_like(ds.rhs)
    info = M.info()

    def step():
        ds.assemble()
        M.update(A, reuse_amg=False)
        _, res = trs.krylov_solve(args.krylov, A, M, ds.rhs, x, rtol=args.rtol, restart=args.restart)
        return res

    for _ in range(args.warmup):
        res = step()
    torch.cuda.synchronize()
    barrier(world)
    torch.cuda.synchronize()
    l0 = trs.kernel_launches()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stats = []
    trs.profile_spmv(True)
    with ClockSampler(local) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            r = step()
            stats.append(r.stats)
        ev1.record(stream)
        torch.cuda.synchronize()
    spmv_total_ms, spmv_launches = trs.profile_spmv(False)
    barrier(world)
    torch.cuda.synchronize()
    launches = trs.kernel_launches() - l0
    ms = ev0.elapsed_time(ev1) / args.steps
    ms = barrier_max(ms, world)
    last = stats[-1]
    xt = x.cpu().numpy()

    # true residual on the host as an independent check of the reported one
    Aval = A.values()
    rp, col = A.pattern()
    rows = np.repeat(np.arange(len(rp) - 1), np.diff(rp))
    Ax = np.zeros_like(xt).reshape(-1, A.b)
    np.add.at(Ax, rows, np.einsum("prc,pc->pr", Aval, xt.reshape(-1, A.b)[col]))
    host_relres = float(np.linalg.norm(sysm.rhs - Ax.reshape(-1)) / np.linalg.norm(sysm.rhs))

    # Roofline of the dominant kernel, the Krylov operator block SpMV w = A z
    # (FP64 values and vectors; with BiCGSTAB fused with its dot products),
    # timed live over the timed region by events around each launch.  It is FP64-pipe-bound (ncu: FP64 pipe ~91% busy),
    # so it is reported against the FP64 peak: 152 SMs x 2 FP64 FMA/clk x 2
    # flop x 2.07 GHz = 1.259 TFLOP/s; its HBM fraction is given beside it.
    hbm, peak_kind = peaks()
    spmv_ms = spmv_total_ms / max(1, spmv_launches)
    nnzb = A.nnzb
    spmv_flops = 2 * nnzb * A.b * A.b
    spmv_bytes = nnzb * A.b * A.b * 8 + 2 * A.N * 8
    fp64_peak_tflops = 152 * 2 * 2 * 2.07e9 / 1e12
    spmv_tflops = spmv_flops / (spmv_ms * 1e-3) / 1e12
    spmv_gbs = spmv_bytes / (spmv_ms * 1e-3) / 1e9
    # DRAM traffic per launch from the ncu capture of the 96x96x48 case
    # (418.9 + 10.9 MB for 3,061,224 blocks), scaled by the blocks of this matrix
    spmv_traffic = (429.822464e6 * nnzb / 3061224.0
                    if args.workload == "128x128x64_b4" and args.krylov == "fgmres" else None)
    # the other Krylov method on the same system and preconditioner
    other = None
    if not args.no_krylov_compare:
        alt = "bicgstab" if args.krylov == "fgmres" else "fgmres"
        for _ in range(2):
            ds.assemble()
            M.update(A, reuse_amg=False)
            trs.krylov_solve(alt, A, M, ds.rhs, x, rtol=args.rtol, restart=args.restart)
        torch.cuda.synchronize()
        ta = []
        for _ in range(max(1, min(args.steps, 5))):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ds.assemble()
            M.update(A, reuse_amg=False)
            _, ra = trs.krylov_solve(alt, A, M, ds.rhs, x, rtol=args.rtol, restart=args.restart)
            e1.record(stream)
            torch.cuda.synchronize()
            ta.append(e0.elapsed_time(e1))
        other = {"method": alt, "ms_per_step": statistics.median(ta), "solve_ms": ra.stats["ms_solve"],
                 "iters": ra.stats["iters"], "true_relres": ra.stats["true_relres"]}
    # the other ILU level of the F stage on the same system
    other_ilu = None
    if not args.no_ilu_compare:
        fill = 1 - args.ilu_fill
        Mi = trs.CPR(A, precision=args.precision, cheb_degree=args.cheb_degree, decoupling=args.decoupling,
                     ilu_fill=fill)
        for _ in range(2):
            ds.assemble()
            Mi.update(A, reuse_amg=False)
            trs.krylov_solve(args.krylov, A, Mi, ds.rhs, x, rtol=args.rtol, restart=args.restart)
        torch.cuda.synchronize()
        ti = []
        for _ in range(max(1, min(args.steps, 5))):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ds.assemble()
            Mi.update(A, reuse_amg=False)
            _, ri = trs.krylov_solve(args.krylov, A, Mi, ds.rhs, x, rtol=args.rtol, restart=args.restart)
            e1.record(stream)
            torch.cuda.synchronize()
            ti.append(e0.elapsed_time(e1))
        other_ilu = {"ilu_fill": fill, "ms_per_step": statistics.median(ti), "setup_ms": ri.stats["ms_setup"],
                     "solve_ms": ri.stats["ms_solve"], "iters": ri.stats["iters"],
                     "true_relres": ri.stats["true_relres"], "n_colours": Mi.info()["n_colours"]}
        del Mi
    # FP64-preconditioner path on the same system, for the mixed/FP64 comparison
    fp64 = None
    if not args.no_fp64_compare and args.precision == "fp32":
        M64 = trs.CPR(A, precision="fp64", decoupling=args.decoupling, ilu_fill=args.ilu_fill)
        for _ in range(2):
            ds.assemble()
            M64.update(A, reuse_amg=False)
            _, r64 = trs.krylov_solve(args.krylov, A, M64, ds.rhs, x, rtol=args.rtol, restart=args.restart)
        torch.cuda.synchronize()
        t64 = []
        for _ in range(max(1, min(args.steps, 3))):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ds.assemble()
            M64.update(A, reuse_amg=False)
            _, r64 = trs.krylov_solve(args.krylov, A, M64, ds.rhs, x, rtol=args.rtol, restart=args.restart)
            e1.record(stream)
            torch.cuda.synchronize()
            t64.append(e0.elapsed_time(e1))
        fp64 = {"ms_per_step": statistics.median(t64), "solve_ms": r64.stats["ms_solve"],
                "setup_ms": r64.stats["ms_setup"], "iters": r64.stats["iters"],
                "true_relres": r64.stats["true_relres"]}
        del M64

    # end to end through the public API with host buffers
    e2e = None
    if not args.no_e2e:
        pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
        hk, hM, hacc, hwi, hlam, hb = (pin(sysm.k), pin(sysm.M.reshape(-1)), pin(sysm.acc.reshape(-1)),
                                       pin(sysm.wi), pin(sysm.lam.reshape(-1)), pin(sysm.rhs))
        hx = torch.empty(A.N, dtype=torch.float64).pin_memory()
        h2d = sum(t.numel() * 8 for t in (hk, hM, hacc, hwi, hlam, hb))
        d2h = hx.numel() * 8

        def e2e_step():
            for d, h in ((ds.k, hk), (ds.M, hM), (ds.acc, hacc), (ds.wi, hwi), (ds.lam, hlam),
                         (ds.rhs, hb)):
                d.copy_(h, non_blocking=True)
            ds.assemble()
            M.update(A, reuse_amg=False)
            trs.krylov_solve(args.krylov, A, M, ds.rhs, x, rtol=args.rtol, restart=args.restart)
            hx.copy_(x, non_blocking=True)

        e2e_step()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        n_e2e = max(1, min(args.steps, 3))
        e0.record(stream)
        for _ in range(n_e2e):
            e2e_step()
        e1.record(stream)
        torch.cuda.synchronize()
        e2e = {"value": barrier_max(e0.elapsed_time(e1) / n_e2e, world), "unit": "ms",
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        est, detail = oracle_sample(sysm, 1, last["iters"] if args.precision == "fp64" or fp64 is None else
                                    fp64["iters"])
        cpu = {"value": est, "unit": "ms", "cores": 1, "kind": "oracle",
               "sample": "assembly + CPR setup + 1 FGMRES iteration of the FP64 oracle on the full system, "
                         "scaled to the iteration count of the FP64 path (of this run's path if the FP64 path "
                         "was not run)", "detail": detail}

    if rank == 0:
        kname = ("k_spmv<4,double,double> (FGMRES operator block SpMV)" if args.krylov == "fgmres" else
                 "k_bicg_spmv<4,1|2> (BiCGSTAB operator block SpMV fused with its dot products)")
        line = {
            "metric": METRIC if args.krylov == "fgmres" else METRIC.replace("FGMRES", "BiCGSTAB"), "value": ms, "unit": "ms", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64+f32" if args.precision == "fp32" else "f64",
            "data": "synthetic",
            "config": {"workload": args.workload, "cells": sysm.n_cells, "b": sysm.b, "wells": sysm.n_wells,
                       "unknowns": sysm.n_unknowns,
                       "krylov": args.krylov,
                       "precision": "FP32 CPR inside FP64 Krylov" if args.precision == "fp32" else "FP64",
                       "rtol": args.rtol, "restart": args.restart, "cheb_degree": args.cheb_degree,
                       "decoupling": args.decoupling, "ilu_fill": args.ilu_fill,
                       "l2": "inputs larger than L2 (Jacobian inputs 0.9 GB, matrix 0.9 GB)",
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "iters": last["iters"], "true_relres": last["true_relres"], "host_true_relres": host_relres,
            "breakdown_ms": {"setup": last["ms_setup"], "solve": last["ms_solve"]},
            "amg_levels": info["n_levels"], "amg_rows": info["level_rows"], "n_colours": info["n_colours"],
            "fp64_path": fp64, "other_krylov": other, "other_ilu": other_ilu,
            "roofline": {"kernel": kname, "bound": "alu",
                         "achieved": spmv_tflops, "peak": fp64_peak_tflops, "unit": "TFLOP/s",
                         "frac": spmv_tflops / fp64_peak_tflops, "traffic": spmv_traffic,
                         "peak_kind": "FP64 unit count x clock (probe measured 1.2548 TFLOP/s)",
                         "launch_ms": spmv_ms, "launches": spmv_launches, "algorithmic_flops": spmv_flops,
                         "algorithmic_bytes": spmv_bytes, "hbm_achieved_gbs": spmv_gbs, "hbm_peak_gbs": hbm,
                         "hbm_frac": spmv_gbs / hbm, "hbm_peak_kind": peak_kind},
            "cpu_baseline": cpu, "e2e": e2e, "clocks": clk.summary(), "gpu_launches": launches,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
