#!/usr/bin/env python
"""Benchmark of one Newton-step linear solve on a GB300.

A step is one pass of the whole hot path over the 128x128x64, b = 4 synthetic
thermal Jacobian (1,048,576 cells, 8 SAGD wells, 4,194,336 unknowns with the
wells padded to b x b blocks): transmissibility/Jacobian assembly on the GPU,
full CPR setup (decoupling, pressure AMG, colouring, block ILU), and
FGMRES(30) to a true FP64 relative residual of 1e-6 -- with the CPR stored and
applied in FP32 (the default) or FP64 (--precision fp64).  value = device
milliseconds per step (lower is better), inputs resident in HBM.

Multi-GPU: the path is one system per GPU ("replicas"); every rank solves its
own copy and the step time is the maximum over ranks.

--impl reference times the CPU oracle (plain C, FP64, single thread): full
solves (assembly + CPR setup + FGMRES to the same tolerance) of the same
system, as many as fit a few minutes.
--sweep times every CPR stage ordering x decoupling pair on the workload.
--sequence N times a Newton-like sequence of N systems (forward + adjoint).
"""
from __future__ import annotations

import argparse
import json
import os
import platform
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
#: FP64 FMA units: 152 SMs x 2 FP64 FMA per clock (4 flop per SM per clock)
FP64_FLOP_PER_CLOCK = 152 * 2 * 2
#: reference-arm step cap: full oracle solves of the 128x128x64 system take
#: about 16 s each on the GPU host's cores
REF_MAX_STEPS, REF_MAX_WARMUP = 3, 1
#: resident memory of one oracle solve per unknown (5.1 GB at 4.19M unknowns)
ORACLE_BYTES_PER_UNKNOWN = 1300


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
    p.add_argument("--no-cpu-all-cores", action="store_true",
                   help="skip the all-core column of the oracle baseline (one solve per core)")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-fp64-compare", action="store_true")
    p.add_argument("--sequence", type=int, default=0,
                   help="time a sequence of this many Newton-like systems (accumulation blocks rescaled by "
                        "seeded +-20%% factors, AMG hierarchy rebuilt every --reuse steps, forward and adjoint "
                        "solve per system) instead of single solves")
    p.add_argument("--reuse", type=int, default=5)
    p.add_argument("--stages", default="fpf", choices=["fpf", "fp", "pf"],
                   help="CPR stage ordering of the forward CPR")
    p.add_argument("--decoupling", default="abf", choices=["abf", "none", "frs", "frs+abf"],
                   help="decoupling of the forward CPR")
    p.add_argument("--adjoint-decoupling", default="none", choices=["abf", "none", "frs", "frs+abf"],
                   help="decoupling of the CPR built on A^T for the adjoint solves")
    p.add_argument("--ilu-fill", type=int, default=None, choices=[0, 1],
                   help="level of fill of the block ILU stage (default: 0, 1 for --sequence and --jacobian physics)")
    p.add_argument("--no-ilu-compare", action="store_true",
                   help="skip timing the other ILU level on the same system")
    p.add_argument("--restart", type=int, default=None,
                   help="FGMRES restart length (default: 30, 60 for --sequence and --jacobian physics)")
    p.add_argument("--cheb-degree", type=int, default=2, help="Chebyshev smoother degree")
    p.add_argument("--krylov", default="fgmres", choices=["fgmres", "bicgstab"],
                   help="outer Krylov method of the timed step")
    p.add_argument("--no-krylov-compare", action="store_true",
                   help="skip timing the other Krylov method on the same system")
    p.add_argument("--sweep", action="store_true",
                   help="time every CPR stage ordering x decoupling pair (FP32 and FP64 CPR) instead")
    p.add_argument("--jacobian", default="synthetic", choices=["synthetic", "physics"],
                   help="physics: the step assembles the thermal model's Jacobian and residual "
                        "(water + heavy oil + energy) on the workload's grid and wells and solves J d = R")
    a = p.parse_args()
    # block ILU(1) and FGMRES(60) for the Newton-like sequence and the physics
    # Jacobian step (the single-system runs where ILU(0)/FGMRES(30) stalls or
    # needs ten times the iterations); the synthetic single solve and the sweep
    # keep the configuration's block ILU(0) and FGMRES(30)
    stronger = bool(a.sequence) or (a.jacobian == "physics" and not a.sweep)
    if a.ilu_fill is None:
        a.ilu_fill = 1 if stronger else 0
    if a.restart is None:
        a.restart = 60 if stronger else 30
    return a


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


def host_info():
    model = platform.processor() or platform.machine()
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    return {"cpu_model": model, "nproc": os.cpu_count(), "machine": platform.machine()}


def mem_available_bytes():
    """Memory this process may still use: MemAvailable, bounded by a cgroup limit."""
    avail = None
    try:
        with open("/proc/meminfo") as f:
            for line in f:
                if line.startswith("MemAvailable:"):
                    avail = int(line.split()[1]) * 1024
    except OSError:
        pass
    for path in ("/sys/fs/cgroup/memory.max", "/sys/fs/cgroup/memory/memory.limit_in_bytes"):
        try:
            with open(path) as f:
                v = f.read().strip()
            if v.isdigit():
                lim = int(v)
                with open(path.replace("memory.max", "memory.current").replace("limit_in_bytes",
                                                                               "usage_in_bytes")) as f:
                    used = int(f.read().strip())
                avail = min(avail, lim - used) if avail else lim - used
        except (OSError, ValueError):
            pass
    return avail or 0


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
def oracle_full_solve(sysm, rtol, restart=30):
    """One full FP64 oracle solve (assembly + CPR setup + FGMRES to the true
    relative residual rtol), single thread; returns (ms, detail, x)."""
    from oracle import oracle as O
    O.build()
    t0 = time.perf_counter()
    Ao = O.assemble(sysm)
    t1 = time.perf_counter()
    cpr = O.CPR(Ao)
    t2 = time.perf_counter()
    res = O.fgmres(Ao, cpr, sysm.rhs, rtol=rtol, restart=restart)
    t3 = time.perf_counter()
    detail = {"assemble_s": t1 - t0, "setup_s": t2 - t1, "solve_s": t3 - t2, "iters": res.iters,
              "true_relres": res.true_relres, "converged": res.converged}
    return 1e3 * (t3 - t0), detail, res.x


def _replica_main(workload, rtol, restart, barrier_, queue):
    """One oracle replica: generate the system, wait for the others, solve."""
    sysm = make_workload(workload)
    from oracle import oracle as O
    O.build()
    barrier_.wait()
    t0 = time.time()
    Ao = O.assemble(sysm)
    cpr = O.CPR(Ao)
    res = O.fgmres(Ao, cpr, sysm.rhs, rtol=rtol, restart=restart)
    queue.put((t0, time.time(), res.iters, res.true_relres))


def oracle_all_cores(workload, rtol, restart, n_unknowns):
    """The oracle on all host cores: one independent full solve per core (the
    oracle is sequential), started together; value = wall time of the set /
    number of solves.  The replica count is bounded by the memory available."""
    import multiprocessing as mp
    cores = os.cpu_count() or 1
    per = ORACLE_BYTES_PER_UNKNOWN * n_unknowns + (1 << 30)
    fit = int(0.6 * mem_available_bytes() // per)
    P = max(1, min(cores, fit))
    ctx = mp.get_context("spawn")
    bar = ctx.Barrier(P)
    q = ctx.Queue()
    procs = [ctx.Process(target=_replica_main, args=(workload, rtol, restart, bar, q)) for _ in range(P)]
    for p in procs:
        p.start()
    out = [q.get(timeout=1800) for _ in range(P)]
    for p in procs:
        p.join()
    wall = max(o[1] for o in out) - min(o[0] for o in out)
    return {"value": 1e3 * wall / P, "unit": "ms", "cores": P, "kind": "oracle",
            "sample": f"{P} independent full oracle solves (assembly + CPR setup + FGMRES to rtol {rtol}) "
                      f"of this workload run together, one per core; value = wall time / {P}",
            "wall_s": wall, "iters": sorted({o[2] for o in out}),
            "memory_bound": P < cores, **host_info()}


def run_reference(args):
    """The reference arm: full FP64 oracle solves of the same system, at most
    REF_MAX_STEPS timed after REF_MAX_WARMUP untimed, so that the run takes a
    few minutes; the line states the steps it ran."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    sysm = make_workload(args.workload)
    warm, steps = min(args.warmup, REF_MAX_WARMUP), max(1, min(args.steps, REF_MAX_STEPS))
    times = []
    detail = None
    for step in range(warm + steps):
        ms, detail, _ = oracle_full_solve(sysm, args.rtol, args.restart)
        if step >= warm:
            times.append(ms)
    value = statistics.median(times)
    sample = (f"full FP64 oracle solve (assembly + CPR setup + FGMRES to true rel. res. {args.rtol}) of the "
              f"{args.workload} system, single thread; median of {steps} after {warm} untimed "
              f"({args.steps} steps and {args.warmup} warm-up requested, capped so the run takes minutes)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "ms", "n_gpus": args.gpus,
            "steps": steps, "warmup": warm, "steps_requested": args.steps, "warmup_requested": args.warmup,
            "ms_per_step": value, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic", "oracle_precision": "FP64 throughout",
            "config": config_of(args, sysm, 1),
            "cpu_baseline": {"value": value, "unit": "ms", "cores": 1, "kind": "oracle", "sample": sample,
                             "detail": detail, **host_info()},
            "e2e": {"value": value, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def l2_note(sysm):
    """Whether the step's inputs exceed the 129 MB L2 (no flush needed between steps)."""
    stored = (7 * sysm.n_cells + 2 * len(sysm.perf_cell) + sysm.n_wells) * sysm.b * sysm.b * 8
    inputs = sysm.M.nbytes + sysm.acc.nbytes + sysm.k.nbytes
    if stored + inputs > 129e6:
        return (f"inputs larger than L2 (Jacobian inputs {inputs / 1e9:.2f} GB, matrix {stored / 1e9:.2f} GB): "
                "no flush between steps")
    return f"inputs fit in L2 ({(stored + inputs) / 1e6:.1f} MB): latency-bound case, no flush"


def config_of(args, sysm, world):
    return {"workload": args.workload, "cells": sysm.n_cells, "b": sysm.b, "wells": sysm.n_wells,
            "unknowns": sysm.n_unknowns, "krylov": args.krylov,
            "precision": "FP32 CPR inside FP64 Krylov" if args.precision == "fp32" else "FP64",
            "rtol": args.rtol, "restart": args.restart, "cheb_degree": args.cheb_degree,
            "stages": args.stages, "decoupling": args.decoupling, "ilu_fill": args.ilu_fill,
            "l2": l2_note(sysm),
            "parallelism": "replicas" if world > 1 else "single GPU"}


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
                stages=args.stages, ilu_fill=args.ilu_fill)
    AT = A.transpose()
    MT = trs.CPR(AT, precision=args.precision, cheb_degree=args.cheb_degree, decoupling=args.adjoint_decoupling,
                 stages=args.stages, ilu_fill=args.ilu_fill)
    x = torch.zeros_like(ds.rhs)
    records = []

    def run_all(record, time_phases=False):
        for k in range(args.sequence):
            torch.mul(acc0.view(-1, bb), scales[k].view(-1, 1), out=ds.acc.view(-1, bb))
            ds.assemble()
            reuse = (k % args.reuse) != 0
            M.update(A, reuse_amg=reuse)
            _, rf = trs.krylov_solve(args.krylov, A, M, ds.rhs, x, rtol=args.rtol, restart=args.restart,
                                     time_phases=time_phases)
            A.transpose(into=AT)
            MT.update(AT, reuse_amg=reuse)
            lam, _, ra = trs.solve_adjoint(A, AT, MT, g, x, rtol=args.rtol, restart=args.restart,
                                           method=args.krylov)
            trs.chain_theta(A, ds.k, ds.M, lam, x, sysm.kvkh, sysm.c_t)
            if record:
                rec = {"step": k, "amg": "reused" if reuse else "rebuilt",
                       "fwd_iters": rf.stats["iters"], "fwd_relres": rf.stats["true_relres"],
                       "adj_iters": ra.stats["iters"], "adj_relres": ra.stats["true_relres"],
                       "fwd_ms": rf.stats["ms_solve"], "adj_ms": ra.stats["ms_solve"]}
                if time_phases:
                    rec.update({k2: rf.stats[k2] for k2 in ("ms_precond", "ms_spmv", "ms_orth", "spmv_launches")})
                records.append(rec)

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
    launches = trs.kernel_launches() - l0
    converged = all(r["fwd_relres"] <= args.rtol and r["adj_relres"] <= args.rtol for r in records)
    # phase split of the forward solves, in a separate pass after the timed region
    records.clear()
    run_all(True, time_phases=True)
    torch.cuda.synchronize()
    phases = {k: sum(r[k] for r in records) for k in ("ms_precond", "ms_spmv", "ms_orth", "spmv_launches")}
    hbm, peak_kind = peaks()
    spmv_bytes = A.nnzb * A.b * A.b * 8 + 2 * A.N * 8
    spmv_ms = phases["ms_spmv"] / max(1, phases["spmv_launches"])
    if rank == 0:
        line = {"metric": f"Newton-like sequence of {args.sequence} systems: forward + adjoint CPR-"
                          f"{args.krylov.upper()} total ms",
                "value": ms, "unit": "ms", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": ms, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
                "dtype": "f64+f32" if args.precision == "fp32" else "f64", "data": "synthetic",
                "config": {"workload": args.workload, "cells": sysm.n_cells, "b": sysm.b, "wells": sysm.n_wells,
                           "unknowns": sysm.n_unknowns, "systems": args.sequence, "amg_rebuild_every": args.reuse,
                           "rtol": args.rtol, "precision": args.precision, "stages": args.stages,
                           "decoupling": args.decoupling, "adjoint_decoupling": args.adjoint_decoupling,
                           "restart": args.restart, "ilu_fill": args.ilu_fill,
                           "l2": "inputs larger than L2", "parallelism": "replicas" if world > 1 else "single GPU"},
                "all_converged": converged, "per_system": records,
                "forward_phases_ms": phases,
                "spmv": {"launch_ms": spmv_ms, "algorithmic_bytes": spmv_bytes,
                         "hbm_gbs": spmv_bytes / (spmv_ms * 1e-3) / 1e9 if spmv_ms else None,
                         "hbm_peak_gbs": hbm, "hbm_peak_kind": peak_kind},
                "clocks": clk.summary(), "gpu_launches": launches}
        print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------ CPR sweep
def run_sweep(args):
    """Every CPR stage ordering x decoupling pair on one system (Sec.
    "Numerical Performance" compares them): iterations, setup and solve ms,
    true residual, for the FP32 and FP64 CPR."""
    import torch
    from paper_1812_03952_gb300 import build as B
    from paper_1812_03952_gb300 import trs
    B.build()
    trs.load()
    rank, world, local = dist_setup(args.gpus)
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream()
    sysm = make_workload(args.workload)
    if args.jacobian == "physics":
        from paper_1812_03952_gb300 import synthetic as S
        phys = trs.ThermalSystem(sysm, S.thermal_state(sysm, S.SEED_BASE + 77), S.SWT, S.SLT)
        rhs = phys.assemble()
        A = phys.A
        assemble = phys.assemble
    else:
        ds = trs.DeviceSystem(sysm, dev)
        A = ds.assemble()
        rhs = ds.rhs
        assemble = ds.assemble
    x = torch.zeros_like(rhs)
    rows = []
    with ClockSampler(local) as clk:
        for precision in ("fp32", "fp64"):
            for stages in ("fpf", "fp", "pf"):
                for dec in ("abf", "none", "frs", "frs+abf"):
                    M = trs.CPR(A, precision=precision, stages=stages, decoupling=dec,
                                cheb_degree=args.cheb_degree, ilu_fill=args.ilu_fill)
                    ts, res = [], None
                    for k in range(args.warmup + args.steps):
                        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                        e0.record(stream)
                        assemble()
                        M.update(A, reuse_amg=False)
                        _, res = trs.krylov_solve(args.krylov, A, M, rhs, x, rtol=args.rtol,
                                                  restart=args.restart, maxit=1000)
                        e1.record(stream)
                        torch.cuda.synchronize()
                        if k >= args.warmup:
                            ts.append(e0.elapsed_time(e1))
                    rows.append({"precision": precision, "stages": stages, "decoupling": dec,
                                 "iters": res.stats["iters"], "converged": bool(res.stats["converged"]),
                                 "true_relres": res.stats["true_relres"], "setup_ms": res.stats["ms_setup"],
                                 "solve_ms": res.stats["ms_solve"], "ms_per_step": statistics.median(ts)})
                    del M
    if rank == 0:
        print(json.dumps({"metric": "CPR stage ordering x decoupling sweep: ms per step (assembly + CPR setup + "
                                    f"{args.krylov.upper()} to true rel. res. {args.rtol})"
                                    + (", physics Jacobian" if args.jacobian == "physics" else ""),
                          "unit": "ms", "higher_is_better": False, "n_gpus": world, "steps": args.steps,
                          "warmup": args.warmup, "data": "synthetic",
                          "config": config_of(args, sysm, world), "rows": rows, "clocks": clk.summary()}),
              flush=True)
    return 0


# ------------------------------------------------- physics Jacobian step
def run_physics(args):
    """One Newton step of the thermal model: the Jacobian dR/du and residual
    R(u) assembled on the GPU (water + heavy oil + energy, Sec. "Mathematical
    Model"), CPR setup on it, and the CPR-Krylov solve of J d = R."""
    import torch
    from paper_1812_03952_gb300 import build as B
    from paper_1812_03952_gb300 import synthetic as S
    from paper_1812_03952_gb300 import trs
    B.build()
    trs.load()
    rank, world, local = dist_setup(args.gpus)
    stream = torch.cuda.current_stream()
    sysm = make_workload(args.workload)
    if sysm.b != 4:
        raise SystemExit("the thermal model has b = 4")
    state = S.thermal_state(sysm, S.SEED_BASE + 77)
    ts = trs.ThermalSystem(sysm, state, S.SWT, S.SLT)
    R = ts.assemble()
    M = trs.CPR(ts.A, precision=args.precision, cheb_degree=args.cheb_degree, stages=args.stages,
                decoupling=args.decoupling, ilu_fill=args.ilu_fill)
    d = torch.zeros_like(R)
    ea, eb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    asm = []

    def step(record=False):
        if record:
            ea.record(stream)
        ts.assemble()
        if record:
            eb.record(stream)
        M.update(ts.A, reuse_amg=False)
        _, res = trs.krylov_solve(args.krylov, ts.A, M, R, d, rtol=args.rtol, restart=args.restart)
        if record:
            asm.append(ea.elapsed_time(eb))
        return res

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    barrier(world)
    l0 = trs.kernel_launches()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        e0.record(stream)
        for _ in range(args.steps):
            res = step()
        e1.record(stream)
        torch.cuda.synchronize()
    ms = barrier_max(e0.elapsed_time(e1) / args.steps, world)
    launches = trs.kernel_launches() - l0
    for _ in range(max(1, min(args.steps, 5))):
        step(record=True)
    asm_ms = statistics.median(asm)
    if rank == 0:
        line = {"metric": "Newton step with the physics Jacobian: thermal assembly + CPR setup + CPR-"
                          f"{args.krylov.upper()} to true rel. res. {args.rtol} (ms)",
                "value": ms, "unit": "ms", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": ms, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
                "dtype": "f64+f32" if args.precision == "fp32" else "f64", "data": "synthetic",
                "config": {**config_of(args, sysm, world), "jacobian": "physics (water + heavy oil + energy)",
                           "gas_cells": int(state.gas.sum()), "dt_day": state.params["dt"]},
                "iters": res.stats["iters"], "converged": bool(res.stats["converged"]),
                "true_relres": res.stats["true_relres"],
                "breakdown_ms": {"assembly": asm_ms, "setup": res.stats["ms_setup"], "solve": res.stats["ms_solve"]},
                "clocks": clk.summary(), "gpu_launches": launches}
        print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------- GPU arm
def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.sequence:
        return run_sequence(args)
    if args.sweep:
        return run_sweep(args)
    if args.jacobian == "physics":
        return run_physics(args)
    import torch
    from paper_1812_03952_gb300 import build as B
    from paper_1812_03952_gb300 import trs

    B.build()
    trs.load()
    rank, world, local = dist_setup(args.gpus)
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream()
    sysm = make_workload(args.workload)
    ds = trs.DeviceSystem(sysm, dev)
    A = ds.assemble()
    cpr_kw = dict(precision=args.precision, cheb_degree=args.cheb_degree, stages=args.stages,
                  decoupling=args.decoupling, ilu_fill=args.ilu_fill)
    M = trs.CPR(A, **cpr_kw)
    x = torch.zeros_like(ds.rhs)
    info = M.info()

    def step(time_phases=False):
        ds.assemble()
        M.update(A, reuse_amg=False)
        _, res = trs.krylov_solve(args.krylov, A, M, ds.rhs, x, rtol=args.rtol, restart=args.restart,
                                  time_phases=time_phases)
        return res

    for _ in range(args.warmup):
        res = step()
    torch.cuda.synchronize()
    barrier(world)
    torch.cuda.synchronize()
    l0 = trs.kernel_launches()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stats = []
    with ClockSampler(local) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            r = step()
            stats.append(r.stats)
        ev1.record(stream)
        torch.cuda.synchronize()
    barrier(world)
    torch.cuda.synchronize()
    launches = trs.kernel_launches() - l0
    ms = ev0.elapsed_time(ev1) / args.steps
    ms = barrier_max(ms, world)
    last = stats[-1]
    x32 = x.cpu().numpy()
    clocks = clk.summary()

    # Roofline pass, after the timed region: the same steps again with CUDA
    # events between the solve's phases (opts.time_phases) on the solve's
    # stream; gives the operator SpMV's average launch time and the phase split.
    n_rp = max(1, min(args.steps, 5))
    pev0, pev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ph = {"ms_precond": 0.0, "ms_spmv": 0.0, "ms_orth": 0.0, "spmv_launches": 0, "ms_solve": 0.0,
          "ms_setup": 0.0}
    with ClockSampler(local) as clk_rp:
        pev0.record(stream)
        for _ in range(n_rp):
            r = step(time_phases=True)
            for k in ph:
                ph[k] += r.stats[k]
        pev1.record(stream)
        torch.cuda.synchronize()
    rp_step_ms = pev0.elapsed_time(pev1) / n_rp
    phases = {k: v / n_rp for k, v in ph.items() if k != "spmv_launches"}
    phases["spmv_launches_per_step"] = ph["spmv_launches"] / n_rp

    # true residual on the host as an independent check of the reported one
    Aval = A.values()
    rp, col = A.pattern()
    rows = np.repeat(np.arange(len(rp) - 1), np.diff(rp))
    Ax = np.zeros_like(x32).reshape(-1, A.b)
    np.add.at(Ax, rows, np.einsum("prc,pc->pr", Aval, x32.reshape(-1, A.b)[col]))
    host_relres = float(np.linalg.norm(sysm.rhs - Ax.reshape(-1)) / np.linalg.norm(sysm.rhs))

    # Roofline of the dominant kernel, the Krylov operator block SpMV w = A z
    # (FP64 values and vectors; with BiCGSTAB fused with its dot products).
    # It is FP64-pipe-bound (ncu: FP64 pipe ~89% busy), so it is reported
    # against the FP64 peak at the SM clock sampled during the roofline pass:
    # 152 SMs x 2 FP64 FMA/clk x 2 flop x f; its HBM fraction is given beside it.
    hbm, peak_kind = peaks()
    spmv_ms = ph["ms_spmv"] / max(1, ph["spmv_launches"])
    nnzb = A.nnzb
    spmv_flops = 2 * nnzb * A.b * A.b
    spmv_bytes = nnzb * A.b * A.b * 8 + 2 * A.N * 8
    rp_clock = clk_rp.summary().get("sm_mhz") or clocks.get("sm_mhz") or 2070.0
    fp64_peak_tflops = FP64_FLOP_PER_CLOCK * rp_clock * 1e6 / 1e12
    spmv_tflops = spmv_flops / (spmv_ms * 1e-3) / 1e12
    spmv_gbs = spmv_bytes / (spmv_ms * 1e-3) / 1e9
    # DRAM traffic per launch of k_spmv<4,double,double> on this 128x128x64
    # system, from ncu (see SPMV_TRAFFIC_128)
    spmv_traffic = (SPMV_TRAFFIC_128 if args.workload == "128x128x64_b4" and args.krylov == "fgmres"
                    else None)

    def timed_legs(Mx, solver, n):
        for _ in range(2):
            ds.assemble()
            Mx.update(A, reuse_amg=False)
            trs.krylov_solve(solver, A, Mx, ds.rhs, x, rtol=args.rtol, restart=args.restart)
        torch.cuda.synchronize()
        ts, rr = [], None
        for _ in range(n):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ds.assemble()
            Mx.update(A, reuse_amg=False)
            _, rr = trs.krylov_solve(solver, A, Mx, ds.rhs, x, rtol=args.rtol, restart=args.restart)
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return statistics.median(ts), rr

    # the other Krylov method on the same system and preconditioner
    other = None
    if not args.no_krylov_compare:
        alt = "bicgstab" if args.krylov == "fgmres" else "fgmres"
        t, ra = timed_legs(M, alt, max(1, min(args.steps, 5)))
        other = {"method": alt, "ms_per_step": t, "solve_ms": ra.stats["ms_solve"],
                 "iters": ra.stats["iters"], "true_relres": ra.stats["true_relres"]}
    # the other ILU level of the F stage on the same system
    other_ilu = None
    if not args.no_ilu_compare:
        fill = 1 - args.ilu_fill
        Mi = trs.CPR(A, **{**cpr_kw, "ilu_fill": fill})
        t, ri = timed_legs(Mi, args.krylov, max(1, min(args.steps, 5)))
        other_ilu = {"ilu_fill": fill, "ms_per_step": t, "setup_ms": ri.stats["ms_setup"],
                     "solve_ms": ri.stats["ms_solve"], "iters": ri.stats["iters"],
                     "true_relres": ri.stats["true_relres"], "n_colours": Mi.info()["n_colours"]}
        del Mi
    # FP64-preconditioner path on the same system, for the mixed/FP64 comparison
    fp64 = None
    x64 = None
    if not args.no_fp64_compare and args.precision == "fp32":
        M64 = trs.CPR(A, **{**cpr_kw, "precision": "fp64"})
        t, r64 = timed_legs(M64, args.krylov, max(1, min(args.steps, 3)))
        x64 = x.cpu().numpy()
        fp64 = {"ms_per_step": t, "solve_ms": r64.stats["ms_solve"], "setup_ms": r64.stats["ms_setup"],
                "iters": r64.stats["iters"], "true_relres": r64.stats["true_relres"]}
        del M64

    # End to end through the C ABI with host buffers: trs_bsr_assemble_host
    # (assembly inputs copied from pinned host memory inside the call),
    # trs_cpr_update, and trs_fgmres_solve_host / trs_bicgstab_solve_host (b
    # copied in, x copied out inside the call).
    e2e = None
    if not args.no_e2e:
        pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
        hk, hM, hacc, hwi, hlam, hb = (pin(sysm.k), pin(sysm.M.reshape(-1)), pin(sysm.acc.reshape(-1)),
                                       pin(sysm.wi), pin(sysm.lam.reshape(-1)), pin(sysm.rhs))
        hx = torch.empty(A.N, dtype=torch.float64).pin_memory()
        h2d = sum(t.numel() * 8 for t in (hk, hM, hacc, hwi, hlam, hb))
        d2h = hx.numel() * 8
        host_solve = trs.fgmres_solve_host if args.krylov == "fgmres" else trs.bicgstab_solve_host
        skw = {"restart": args.restart} if args.krylov == "fgmres" else {}

        def e2e_step():
            A.assemble_host(hk, hM, hacc, hwi, hlam, sysm.kvkh, sysm.c_t)
            M.update(A, reuse_amg=False)
            return host_solve(A, M, hb, rtol=args.rtol, x=hx, **skw)[1]

        for _ in range(2):
            e2e_step()
        torch.cuda.synchronize()
        n_e2e = max(1, min(args.steps, 5))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0 = time.perf_counter()
        e0.record(stream)
        for _ in range(n_e2e):
            re = e2e_step()
        e1.record(stream)
        torch.cuda.synchronize()
        wall = (time.perf_counter() - t0) * 1e3 / n_e2e
        e2e = {"value": barrier_max(e0.elapsed_time(e1) / n_e2e, world), "unit": "ms",
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "host_wall_ms": wall,
               "api": "trs_bsr_assemble_host + trs_cpr_update + trs_%s_solve_host" % args.krylov,
               "true_relres": re.stats["true_relres"]}

    cpu = None
    cpu_all = None
    err = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cms, detail, xo = oracle_full_solve(sysm, args.rtol, args.restart)
        cpu = {"value": cms, "unit": "ms", "cores": 1, "kind": "oracle",
               "sample": f"one full FP64 oracle solve of this system (assembly + CPR setup + FGMRES to true rel. "
                         f"res. {args.rtol}), single thread", "detail": detail, **host_info()}
        nx = np.linalg.norm(xo)
        err = {"vs": f"the oracle's FP64 CPR-FGMRES solution at rtol {args.rtol}",
               "timed_path": float(np.linalg.norm(x32 - xo) / nx),
               "fp64_path": float(np.linalg.norm(x64 - xo) / nx) if x64 is not None else None}
        if not args.no_cpu_all_cores:
            cpu_all = oracle_all_cores(args.workload, args.rtol, args.restart, sysm.n_unknowns)

    if rank == 0:
        kname = ("k_spmv<4,double,double> (FGMRES operator block SpMV)" if args.krylov == "fgmres" else
                 "k_bicg_spmv<4,1|2> (BiCGSTAB operator block SpMV fused with its dot products)")
        line = {
            "metric": METRIC if args.krylov == "fgmres" else METRIC.replace("FGMRES", "BiCGSTAB"), "value": ms,
            "unit": "ms", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64+f32" if args.precision == "fp32" else "f64",
            "data": "synthetic",
            "config": config_of(args, sysm, world),
            "iters": last["iters"], "true_relres": last["true_relres"], "host_true_relres": host_relres,
            "err_vs_oracle": err,
            "breakdown_ms": {"setup": last["ms_setup"], "solve": last["ms_solve"]},
            "solve_phases_ms": phases, "phase_pass_ms_per_step": rp_step_ms,
            "amg_levels": info["n_levels"], "amg_rows": info["level_rows"], "n_colours": info["n_colours"],
            "fp64_path": fp64, "other_krylov": other, "other_ilu": other_ilu,
            "roofline": {"kernel": kname, "bound": "alu",
                         "achieved": spmv_tflops, "peak": fp64_peak_tflops, "unit": "TFLOP/s",
                         "frac": spmv_tflops / fp64_peak_tflops, "traffic": spmv_traffic,
                         "peak_kind": f"FP64 unit count x sampled SM clock {rp_clock:.0f} MHz "
                                      "(152 SMs x 4 flop/clk; a probe measured 1.2548 TFLOP/s at 2070 MHz)",
                         "sm_mhz": rp_clock, "launch_ms": spmv_ms, "launches": ph["spmv_launches"],
                         "timing": f"CUDA events around each launch over {n_rp} steps after the timed region",
                         "algorithmic_flops": spmv_flops,
                         "algorithmic_bytes": spmv_bytes, "hbm_achieved_gbs": spmv_gbs, "hbm_peak_gbs": hbm,
                         "hbm_frac": spmv_gbs / hbm, "hbm_peak_kind": peak_kind},
            "cpu_baseline": cpu, "cpu_baseline_all_cores": cpu_all, "e2e": e2e, "clocks": clocks,
            "gpu_launches": launches,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


#: ncu dram__bytes_read.sum + dram__bytes_write.sum of one k_spmv<4,double,double>
#: launch on the 128x128x64 system (one-pass capture of this bench's own
#: command: 994.32 MB read, 30.50 MB written)
SPMV_TRAFFIC_128 = (994.32 + 30.50) * 1e6


if __name__ == "__main__":
    sys.exit(main())
