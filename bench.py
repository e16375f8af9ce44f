"""Benchmark of the SQ hot path on one GB300 (or N replicas under torchrun).

Metric: SQ density throughput in grid points per second -- columns taken through the whole path in
one step: Hamiltonian set-up (projector tables, spectral bounds), the K-step Chebyshev recursion of
every column with moments and force moments, moment sums, Fermi level, weights, density, band
energy/entropy and nonlocal forces.  Workload: the 95-atom mono-vacancy hcp Mg-like cell
(48x42x59 grid = 118,944 points, 12th-order FD, s+p projectors, R_cut = 6 bohr -> 25^3 cubes,
K = 60, kT = 0.005 Ha).  The main line is the FP32 recursion (FP64 Fermi solve and reductions); the
FP64 recursion is measured in the same run under "fp64".

  python bench.py [--steps K] [--warmup W] [--precision fp32|fp64|both] [--impl ours|reference]
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2011_13517_gb300 import cells  # noqa: E402

METRIC = "SQ density grid-points/sec (FP32 vs FP64) at stated rho error; % of roofline"
UNIT = "grid-points/s"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
# FP32 FMA roofline from unit counts: 152 SMs x 128 FP32 lanes x 2 flop x 2070 MHz max SM clock
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12
# FP64 roofline: the nominal GB300 FP64 rate (1.25 TFLOP/s)
FP64_PEAK_TFLOPS = 1.25
# DRAM bytes (read + write) of one full-size vacancy launch, from one ncu capture of the same kernel
# version (dram__bytes_read.sum 3.41 MB + dram__bytes_write.sum 846.59 KB); a kernel without a
# capture of its current version reports null
MEASURED_TRAFFIC = {"slab_kernel<25,6>": 3.41e6 + 846.59e3}


def workload_config(cell):
    return {
        "workload": (f"{cell.name}: hcp Mg-like mono-vacancy, {cell.n[0]}x{cell.n[1]}x{cell.n[2]} grid "
                     f"({cell.N_d} points), {cell.fd_order}th-order FD, s+p KB projectors, "
                     f"R_cut={cell.R_cut} bohr ({cell.n_c[0]}^3 cubes), K={cell.K}, kT={cell.kT} Ha"),
        "grid_points": cell.N_d, "atoms": cell.natom, "K": cell.K, "cube": int(cell.n_c[0]),
        "fd_order": cell.fd_order, "projectors_per_atom": 4,
        "l2": "flushed (256 MiB write) between timed steps",
        "data": "synthetic seeded hcp cell (Gaussian wells + smooth noise); stands in for the paper's "
                "Troullier-Martins Mg systems",
    }


def support_mask(R_a, L_a, n_a, rc):
    """Grid indices of one axis inside the projector support: some periodic image of the atom lies
    closer than the window radius rc (the window (1 - t^2/rc^2)^3 vanishes from |t| = rc on)."""
    x = np.arange(n_a) * (L_a / n_a)
    t = x - R_a
    t = t - L_a * np.round(t / L_a)               # nearest image
    inside = np.abs(t) < rc
    for shift in (-L_a, L_a):                     # further images, for windows wider than half the box
        inside |= np.abs(t + shift) < rc
    return inside


def algorithmic_flops(cell):
    """FLOPs of one recursion-kernel launch counted from the method's definition: per column and
    recursion step, the FD stencil (3 n_o + 1 FMAs per cube point) plus the Chebyshev update (1 FMA),
    plus for each projector 2 |supp chi ^ C_q| FMAs (chi^T v and the rank-1 update); force moments
    add 3 |supp ^ C_q| FMAs per projector of the atoms whose projectors are nonzero at x_q, at each of
    the K+1 vectors.  FLOPs = 2 x FMAs."""
    nc3 = int(np.prod(cell.n_c))
    nproj = 1 if cell.lmax == 0 else 4
    stencil = cell.K * nc3 * (3 * cell.fd_order + 2)
    m = cell.m
    # per atom, axis and window start s: overlap length of the support with [s, s + nc)
    ov = []
    inq = []
    for J in range(cell.natom):
        per_axis, per_axis_q = [], []
        for a in range(3):
            g = support_mask(cell.R[J, a], cell.box[a], int(cell.n[a]), cell.proj_rc)
            n = int(cell.n[a])
            nc = int(cell.n_c[a])
            g2 = np.concatenate([g, g]).astype(np.int64)
            cs = np.concatenate([[0], np.cumsum(g2)])
            starts = (np.arange(n) - m[a]) % n            # window start of a column at index q_a
            per_axis.append(cs[starts + nc] - cs[starts])
            per_axis_q.append(g.astype(np.int64))
        ov.append(per_axis)
        inq.append(per_axis_q)
    total_nl = 0
    total_force = 0
    for J in range(cell.natom):
        ox, oy, oz = ov[J]
        box = oz[:, None, None] * oy[None, :, None] * ox[None, None, :]
        total_nl += int(box.sum())
        qin = inq[J][2][:, None, None] * inq[J][1][None, :, None] * inq[J][0][None, None, :]
        total_force += int((box * qin).sum())
    fma = (cell.N_d * stencil + cell.K * 2 * nproj * total_nl + (cell.K + 1) * 3 * nproj * total_force)
    return 2.0 * fma


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for name, val in zip(names, f[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_baseline(cell, target_seconds=15.0):
    """The FP64 oracle, as it stands, on a bounded sample of columns of the same workload."""
    from oracle import oracle
    lo, hi = oracle.spectral_bounds(cell)
    omega, tau = oracle.scale_shift(lo, hi)
    threads = oracle.max_threads()
    rng = np.random.Generator(np.random.PCG64([23, 5]))
    probe = rng.choice(cell.N_d, size=max(2 * threads, 8), replace=False)
    t0 = time.perf_counter()
    oracle.moments(cell, omega, tau, cols=probe, force=True)
    per_col = (time.perf_counter() - t0) / probe.size
    ncols = int(min(cell.N_d, max(probe.size, target_seconds / max(per_col, 1e-9))))
    ncols = max(threads, (ncols // threads) * threads)
    cols = rng.choice(cell.N_d, size=ncols, replace=False)
    t0 = time.perf_counter()
    oracle.moments(cell, omega, tau, cols=cols, force=True)
    dt = time.perf_counter() - t0
    # the same oracle on one core, on a sample of about a quarter of the time
    n1 = max(2, int(0.25 * target_seconds * ncols / dt / threads))
    t0 = time.perf_counter()
    oracle.moments(cell, omega, tau, cols=cols[:n1], force=True, nthreads=1)
    one_core = n1 / (time.perf_counter() - t0)
    return {"value": ncols / dt, "unit": UNIT, "cores": threads, "kind": "oracle", "value_one_core": one_core,
            "sample": f"{ncols} random columns of the {cell.N_d}-point workload (moments + force moments, "
                      f"K={cell.K}; one-core figure on the first {n1} of them); Fermi solve and observables are "
                      f"O(K M) per step and not sampled",
            "seconds": dt}


def run_reference(args, rank, world):
    cell = cells.vacancy_cell()
    if rank != 0:
        return
    samples = []
    base = None
    for i in range(args.warmup + args.steps):
        base = cpu_baseline(cell, target_seconds=args.ref_seconds)
        if i >= args.warmup:
            samples.append(base["value"])
    value = statistics.mean(samples)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * cell.N_d / value,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(cell),
            "cpu_baseline": dict(base, value=value),
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_batch(args, sq, torch, world, rank, barrier, dist):
    """32 independent defect cells (48-288 sites, 0-2 vacancies, 0-2 Al, R_cut 5/6/7, K 40/60/80) in
    one batch: one persistent recursion launch, autotuned (in FP32 the 21^3/25^3 cells take slab
    launches), captured in a CUDA graph and replayed.  About 4 minutes per FP32 replay."""
    precision = sq.SQ_FP64 if args.precision == "fp64" else sq.SQ_FP32
    cs = cells.batch_cells(32)
    if args.profile:   # small case for ncu: the first four cells with K = 8
        cs = cs[:4]
        for c in cs:
            c.K = 8
    handles = [sq.build_for_cell(c) for c in cs]
    b = sq.sq_batch_create(handles, [c.K for c in cs], [c.kT for c in cs], [c.N_e for c in cs], precision, 0)
    rhos = [torch.empty(c.N_d, dtype=torch.float64, device="cuda") for c in cs]
    t0 = time.perf_counter()
    sq.sq_batch_density(b, rhos)            # autotune + capture + first replay
    first = time.perf_counter() - t0
    if args.profile:
        torch.cuda.synchronize()
        print(json.dumps({"profile_case": "batch", "cells": len(cs), "K": 8, "first_call_s": first,
                          "autotuned": sq.sq_batch_info(b)}), flush=True)
        b.close()
        return
    for _ in range(args.warmup):
        sq.sq_batch_density(b, rhos)
    stream = torch.cuda.current_stream()
    times = []
    with ClockSampler(int(os.environ.get("LOCAL_RANK", "0"))) as clk:
        for _ in range(args.steps):
            torch.cuda.synchronize()
            barrier()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            sq.sq_batch_density(b, rhos)
            e1.record(stream)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
    ms = statistics.mean(times)
    pts = sum(c.N_d for c in cs)
    info = sq.sq_batch_info(b)
    if rank == 0:
        print(json.dumps({"metric": METRIC, "value": world * pts / (ms * 1e-3), "unit": UNIT, "n_gpus": world,
                          "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
                          "scaling": "weak", "vs_baseline": None, "dtype": "f32" if precision else "f64",
                          "data": "synthetic",
                          "config": {"workload": "batch of 32 seeded hcp defect cells (48-288 sites, 0-2 vacancies, "
                                                 "0-2 Al, R_cut 5/6/7 bohr, K 40/60/80), one persistent launch "
                                                 "(FP32: 21^3/25^3 cells as slab launches), CUDA graph",
                                     "grid_points": pts, "first_call_s": first,
                                     "autotuned": info},
                          "clocks": clk.summary()}), flush=True)
    b.close()


def run_adjoint(args, sq, torch, world, rank, barrier, dist):
    """Reverse-mode derivative of (rho, U) wrt V_eff on the vacancy cell (K = 60, checkpoint every 8
    steps): one forward sq_density plus one sq_density_vjp per step."""
    precision = sq.SQ_FP64 if args.precision == "fp64" else sq.SQ_FP32
    c = cells.vacancy_cell()
    kc = 8
    if args.profile:   # small case for ncu: K = 8, checkpoint every 4 steps, one forward + VJP
        c.K, kc = 8, 4
    d_veff = torch.from_numpy(np.ascontiguousarray(c.veff.reshape(-1))).cuda()
    # the derivative holds the spectral bounds fixed: take the library's bounds once and pass them in
    h0 = sq.build_for_cell(c, d_veff=d_veff)
    bounds = sq.sq_get_spectral_bounds(h0)
    h0.close()
    rho = torch.empty(c.N_d, dtype=torch.float64, device="cuda")
    rbar = torch.from_numpy(np.random.default_rng(9).standard_normal(c.N_d)).cuda()
    vbar = torch.empty_like(rho)
    stream = torch.cuda.current_stream()

    def step():
        h = sq.build_for_cell(c, bounds=bounds, d_veff=d_veff)
        sq.sq_density(h, c.K, c.kT, c.N_e, precision, 0, rho)
        sq.sq_density_vjp(h, rbar, 0.25, kc, vbar)
        h.close()

    if args.profile:
        step()
        torch.cuda.synchronize()
        print(json.dumps({"profile_case": "adjoint", "K": c.K, "checkpoint_k": kc}), flush=True)
        return

    for _ in range(args.warmup):
        step()
    times = []
    for _ in range(args.steps):
        torch.cuda.synchronize()
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    ms = statistics.mean(times)
    if rank == 0:
        print(json.dumps({"metric": "SQ forward + vector-Jacobian product grid-points/sec", "value": world * c.N_d / (ms * 1e-3),
                          "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                          "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                          "dtype": "f32" if precision else "f64", "data": "synthetic",
                          "config": dict(workload_config(c), checkpoint_k=kc)}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["fp32", "fp64", "both"], default="both")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ref-seconds", type=float, default=10.0)
    ap.add_argument("--fp64-steps", type=int, default=1,
                    help="timed steps of the secondary FP64 measurement (0: same as --steps)")
    ap.add_argument("--workload", choices=["vacancy", "batch", "adjoint"], default="vacancy",
                    help="vacancy: the headline line; batch: 32 defect cells in one graph-captured batch; "
                         "adjoint: the reverse-mode derivative of the vacancy cell")
    ap.add_argument("--profile", action="store_true",
                    help="small case for ncu, no timing loop: one sq_density of the same cell with K=8 "
                         "(batch: the first four cells, K=8; adjoint: K=8, checkpoint every 4 steps)")
    args = ap.parse_args()

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import torch
    from paper_2011_13517_gb300 import sq

    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    def barrier():
        if dist is not None:
            dist.barrier()

    if args.workload == "batch":
        run_batch(args, sq, torch, world, rank, barrier, dist)
        return
    if args.workload == "adjoint":
        run_adjoint(args, sq, torch, world, rank, barrier, dist)
        return
    cell = cells.vacancy_cell()
    if args.profile:
        cell.K = 8
    stream = torch.cuda.current_stream()
    d_veff = torch.from_numpy(np.ascontiguousarray(cell.veff.reshape(-1))).cuda()
    rho = torch.empty(cell.N_d, dtype=torch.float64, device="cuda")
    force = torch.empty((cell.natom, 3), dtype=torch.float64, device="cuda")
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")

    def step(precision):
        h = sq.build_for_cell(cell, d_veff=d_veff)
        lam = sq.sq_density(h, cell.K, cell.kT, cell.N_e, precision, sq.SQ_WANT_FORCE, rho)
        U, S, F = sq.sq_energy(h)
        sq.sq_nonlocal_force(h, force)
        timing = sq.sq_get_timing(h)
        kname = sq.sq_kernel_name(h)
        h.close()
        return lam, U, S, timing, kname

    def measure(precision, steps, warmup):
        for _ in range(warmup):
            step(precision)
        torch.cuda.synchronize()
        times, rec = [], []
        launches0 = sq.sq_kernel_launches()
        res = None
        with ClockSampler(local_rank) as clk:
            for _ in range(steps):
                flush.zero_()
                torch.cuda.synchronize()
                barrier()
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                res = step(precision)
                e1.record(stream)
                torch.cuda.synchronize()
                barrier()
                times.append(e0.elapsed_time(e1))
                rec.append(res[3][0])
        launches = (sq.sq_kernel_launches() - launches0) / steps
        ms = statistics.mean(times)
        if dist is not None:
            t = torch.tensor([ms], device="cuda")
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            ms = float(t.item())
        return ms, statistics.mean(rec), clk.summary(), launches, res

    def measure_e2e(precision, steps):
        """Through the public API with host buffers: V_eff from pinned host memory in, rho and forces
        back to pinned host memory, all inside the timed region."""
        host_veff = torch.from_numpy(np.ascontiguousarray(cell.veff.reshape(-1))).pin_memory()
        host_rho = torch.empty(cell.N_d, dtype=torch.float64).pin_memory()
        host_f = torch.empty((cell.natom, 3), dtype=torch.float64).pin_memory()
        dv = torch.empty_like(d_veff)
        times = []
        for i in range(steps + 1):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            dv.copy_(host_veff, non_blocking=True)
            h = sq.build_for_cell(cell, d_veff=dv)
            sq.sq_density(h, cell.K, cell.kT, cell.N_e, precision, sq.SQ_WANT_FORCE, rho)
            sq.sq_energy(h)
            sq.sq_nonlocal_force(h, force)
            host_rho.copy_(rho, non_blocking=True)
            host_f.copy_(force, non_blocking=True)
            torch.cuda.synchronize()
            h.close()
            if i > 0:
                times.append(time.perf_counter() - t0)
        bi = cell.N_d * 8 + cell.natom * 3 * 8
        bo = cell.N_d * 8 + cell.natom * 3 * 8
        return cell.N_d / statistics.mean(times), bi, bo

    if args.profile:
        for p in (["fp32", "fp64"] if args.precision == "both" else [args.precision]):
            lam, U, S, timing, kname = step(sq.SQ_FP32 if p == "fp32" else sq.SQ_FP64)
            torch.cuda.synchronize()
            print(json.dumps({"profile_case": p, "K": cell.K, "kernel": kname, "recursion_ms": timing[0], "lambda_f": lam}))
        return
    flops = algorithmic_flops(cell)
    results = {}
    precs = ["fp32", "fp64"] if args.precision == "both" else [args.precision]
    for p in precs:
        code = sq.SQ_FP32 if p == "fp32" else sq.SQ_FP64
        # the FP64 recursion runs at the GB300's FP64 rate (~33 s per step here): a single timed step
        steps = args.steps if (p == precs[0] or args.fp64_steps <= 0) else args.fp64_steps
        ms, rec_ms, clocks, launches, res = measure(code, steps, args.warmup)
        torch.cuda.synchronize()
        rho_out, force_out = rho.cpu().numpy().copy(), force.cpu().numpy().copy()   # after the timed region
        peak = FP32_PEAK_TFLOPS if p == "fp32" else FP64_PEAK_TFLOPS
        achieved = flops / (rec_ms * 1e-3) / 1e12
        results[p] = dict(ms=ms, rec_ms=rec_ms, clocks=clocks, launches=launches, lam_f=res[0], U=res[1], steps=steps,
                          rho=rho_out, force=force_out,
                          S=res[2], value=world * cell.N_d / (ms * 1e-3),
                          roofline={"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                                    "frac": achieved / peak, "traffic": MEASURED_TRAFFIC.get(res[4]),
                                    "kernel": res[4],
                                    "algorithmic_tflop_per_launch": flops / 1e12,
                                    "kernel_ms": rec_ms,
                                    "peak_source": ("FP32 unit count: 152 SM x 128 lanes x 2 x 2.07 GHz"
                                                    if p == "fp32" else "nominal GB300 FP64 rate")})
    main_p = precs[0]
    m = results[main_p]
    e2e_value, bi, bo = measure_e2e(sq.SQ_FP32 if main_p == "fp32" else sq.SQ_FP64, max(1, min(args.steps, 2)))
    line = {
        "metric": METRIC, "value": m["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": m["ms"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32" if main_p == "fp32" else "f64", "data": "synthetic",
        "config": dict(workload_config(cell), parallelism=f"replicas x{world}" if world > 1 else "single GPU",
                       recursion_precision=main_p),
        "roofline": m["roofline"], "clocks": m["clocks"], "gpu_launches": m["launches"],
        "e2e": {"value": world * e2e_value, "unit": UNIT, "h2d_bytes_per_step": bi, "d2h_bytes_per_step": bo},
        "results": {"lambda_f": m["lam_f"], "U": m["U"], "S": m["S"]},
    }
    for p in precs[1:]:
        r = results[p]
        line[p] = {"value": r["value"], "ms_per_step": r["ms"], "steps": r["steps"], "warmup": args.warmup,
                   "roofline": r["roofline"], "clocks": r["clocks"],
                   "gpu_launches": r["launches"], "results": {"lambda_f": r["lam_f"], "U": r["U"], "S": r["S"]}}
    if "fp32" in results and "fp64" in results:
        # the rho error stated with the FP32 throughput, against the FP64 path of the same run (which
        # the parity tests hold to the FP64 oracle at 1e-10 relative)
        r32, r64 = results["fp32"], results["fp64"]
        drho = np.abs(r32["rho"] - r64["rho"])
        line["fp32_vs_fp64"] = {"rho_rel_l1": float(drho.sum() * float(np.prod(cell.h)) / cell.N_e),
                                "rho_max_rel": float((drho / np.maximum(np.abs(r64["rho"]), 1e-300)).max()),
                                "dU_per_atom": abs(r32["U"] - r64["U"]) / cell.natom,
                                "force_max_abs": float(np.abs(r32["force"] - r64["force"]).max()),
                                "dlambda_f": abs(r32["lam_f"] - r64["lam_f"]),
                                "units": "rho_rel_l1 = sum|d rho| dV / N_e; dU Ha/atom; force Ha/bohr; lambda_f Ha",
                                "speedup": r32["value"] / r64["value"]}
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(cell)
    if dist is not None:
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
