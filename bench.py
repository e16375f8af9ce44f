"""Benchmark of the SQ hot path on one GB300 (or N replicas under torchrun).

Metric: SQ density throughput in grid points per second -- columns taken through the whole path in
one step: Hamiltonian set-up (projector tables, spectral bounds), the K-step Chebyshev recursion of
every column with moments and force moments, moment sums, Fermi level, weights, density, band
energy/entropy and nonlocal forces.  Headline workload: the 286-atom precision cell (6x6x4 hcp Mg-like
cell with a divacancy and 2 Al-like solutes, 73x63x79 grid = 363,321 points, 12th-order FD, s+p
projectors, R_cut = 7 bohr -> 29^3 cubes, K = 80, kT = 0.005 Ha).  The main line is the FP32
recursion (FP64 Fermi solve and reductions); the FP64 recursion is measured in the same run under
"fp64", and both are compared with the FP64 oracle's golden values of the same cell.  The 95-atom
vacancy cell (25^3 cubes, K = 60) is reported as an extra key.

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
GOLDEN = os.path.join(ROOT, "tests", "golden")
# FP32 FMA roofline from unit counts: 152 SMs x 128 FP32 lanes x 2 flop x 2070 MHz max SM clock
FP32_UNIT_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12
# FP64: the nominal GB300 rate (1.25 TFLOP/s)
FP64_NOMINAL_TFLOPS = 1.25
# DRAM bytes (read + write) of one full-size launch, from one ncu capture of the same kernel version;
# a kernel without a capture of its current version reports null.  cluster_kernel<29,6,mma>: the
# K = 8 precision-cell launch read 8.98 MB and wrote 148.51 MB (register spills that leave L1, and
# the moments); both scale with the recursion steps per column, so the K = 80 launch is taken as
# 81/9 of that (an upper bound: the per-column set-up reads do not grow with K)
MEASURED_TRAFFIC = {"cluster_kernel<29,6,mma>": (8.97536e6 + 148.50688e6) * 81 / 9}
TRAFFIC_NOTE = {"cluster_kernel<29,6,mma>": "ncu capture of the K = 8 launch (157.5 MB) scaled by 81/9 column-steps; "
                                            "upper bound"}


DESCRIPTION = {
    "precision_286atom": "hcp Mg-like 6x6x4 cell, divacancy + 2 Al-like solutes",
    "vacancy_95atom": "hcp Mg-like mono-vacancy",
}


def workload_config(cell):
    return {
        "workload": (f"{cell.name}: {DESCRIPTION.get(cell.name, 'hcp cell')}, {cell.n[0]}x{cell.n[1]}x{cell.n[2]} "
                     f"grid ({cell.N_d} points), {cell.fd_order}th-order FD, s+p KB projectors, "
                     f"R_cut={cell.R_cut} bohr ({cell.n_c[0]}^3 cubes), K={cell.K}, kT={cell.kT} Ha"),
        "grid_points": cell.N_d, "atoms": cell.natom, "K": cell.K, "cube": int(cell.n_c[0]),
        "fd_order": cell.fd_order, "projectors_per_atom": 4,
        "l2": "flushed (256 MiB write) between timed steps",
        "data": "synthetic seeded hcp cell (Gaussian wells + smooth noise); stands in for the paper's "
                "Troullier-Martins Mg/Al systems",
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


def ball_support(cell, J):
    """Grid points within the projector cut-off radius r_c of atom J (some periodic image closer than
    r_c), as a dense mask on the smallest index box that holds the ball."""
    lo = np.floor((cell.R[J] - cell.proj_rc) / cell.h).astype(int)
    hi = np.ceil((cell.R[J] + cell.proj_rc) / cell.h).astype(int)
    axes = [np.arange(lo[a], hi[a] + 1) * cell.h[a] - cell.R[J, a] for a in range(3)]
    r2 = axes[2][:, None, None] ** 2 + axes[1][None, :, None] ** 2 + axes[0][None, None, :] ** 2
    return r2 < cell.proj_rc ** 2


def algorithmic_flops_ball(cell):
    """FLOPs of one recursion-kernel launch with each projector's support taken as the ball r < r_c
    (the count of the hot-path measurement plan): per column and step (3 n_o + 2) FMAs per cube point,
    2 |B_J ^ C_q| FMAs per projector (chi^T v and the rank-1 update), and for the force moments
    3 |B_J ^ C_q| FMAs per projector of the atoms whose ball holds x_q, at each of the K+1 vectors.
    Every grid point lies in exactly n_c^3 cubes, so sum_q |B ^ C_q| = |B| n_c^3; the force term is
    the autocorrelation of the ball's mask summed over the cube's offsets."""
    from scipy.signal import fftconvolve
    nc3 = int(np.prod(cell.n_c))
    nproj = 1 if cell.lmax == 0 else 4
    m = cell.m
    total_nl = 0
    total_force = 0
    for J in range(cell.natom):
        b = ball_support(cell, J).astype(np.float64)
        total_nl += int(b.sum()) * nc3
        ac = fftconvolve(b, b[::-1, ::-1, ::-1])
        c = np.array(b.shape) - 1
        win = ac[max(c[0] - m[2], 0):c[0] + m[2] + 1, max(c[1] - m[1], 0):c[1] + m[1] + 1,
                 max(c[2] - m[0], 0):c[2] + m[0] + 1]
        total_force += int(np.rint(win.sum()))
    fma = (cell.N_d * cell.K * nc3 * (3 * cell.fd_order + 2) + cell.K * 2 * nproj * total_nl
           + (cell.K + 1) * 3 * nproj * total_force)
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


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_baseline(cell, target_seconds=15.0, threads=None):
    """The FP64 oracle, as it stands, on a bounded sample of columns of the same workload: the moments
    and force moments of a random set of columns, on `threads` host threads (all cores by default),
    with the number of columns chosen from a short probe so the sample takes about target_seconds."""
    from oracle import oracle
    lo, hi = oracle.spectral_bounds(cell)
    omega, tau = oracle.scale_shift(lo, hi)
    threads = threads or host_cores()
    rng = np.random.Generator(np.random.PCG64([23, 5]))
    probe = rng.choice(cell.N_d, size=max(2 * threads, 8), replace=False)
    t0 = time.perf_counter()
    oracle.moments(cell, omega, tau, cols=probe, force=True, nthreads=threads)
    per_col = (time.perf_counter() - t0) / probe.size
    ncols = int(min(cell.N_d, max(probe.size, target_seconds / max(per_col, 1e-9))))
    ncols = max(threads, (ncols // threads) * threads)
    cols = rng.choice(cell.N_d, size=ncols, replace=False)
    t0 = time.perf_counter()
    oracle.moments(cell, omega, tau, cols=cols, force=True, nthreads=threads)
    dt = time.perf_counter() - t0
    return {"value": ncols / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"{ncols} random columns of the {cell.N_d}-point workload (moments + force moments, "
                      f"K={cell.K}) in {dt:.1f} s on {threads} threads; the Fermi solve and observables are "
                      f"O(K M) per step and not sampled",
            "seconds": dt, "columns": ncols}


def run_reference(args, rank, world):
    """The oracle as the reference arm: each step is a bounded sample of columns of the workload,
    timed on the host cores; value = sampled columns per second of wall time."""
    if rank != 0:
        return
    cell = cells.precision_cell()
    per_step = max(2.0, 150.0 / max(1, args.steps + args.warmup))
    samples, secs, base = [], [], None
    for i in range(args.warmup + args.steps):
        base = cpu_baseline(cell, target_seconds=per_step)
        if i >= args.warmup:
            samples.append(base["value"])
            secs.append(base["seconds"])
    value = statistics.mean(samples)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(secs),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(cell),
            "step": f"one step = the oracle on a random sample of about {base['columns']} columns "
                    f"(not the whole {cell.N_d}-point grid); ms_per_step is the sample's measured wall time",
            "cpu_baseline": dict(base, value=value),
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_batch(args, sq, torch, world, rank, barrier, dist):
    """32 independent defect cells (48-288 sites, 0-2 vacancies, 0-2 Al, R_cut 5/6/7, K 40/60/80) in
    one batch: one persistent recursion launch, autotuned (in FP32 the 21^3/25^3/29^3 cells take slab
    or cluster launches), captured in a CUDA graph and replayed."""
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
    launches0 = sq.sq_kernel_launches()
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
                                                 "(FP32: 21^3/25^3/29^3 cells as their own launches), CUDA graph",
                                     "grid_points": pts, "first_call_s": first,
                                     "autotuned": info},
                          "gpu_launches": (sq.sq_kernel_launches() - launches0) / max(1, args.steps),
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


def run_gauss(args, sq, torch, world, rank, barrier, dist):
    """Gauss (Lanczos) spectral quadrature for rho, U and S (SQ_GAUSS) on the vacancy cell at its K:
    per column K Lanczos steps, the Jacobi matrix's Gauss rule, the Fermi level over all nodes and the
    observables, timed like the Chebyshev step (inputs resident, L2 flushed between steps)."""
    precision = sq.SQ_FP64 if args.precision == "fp64" else sq.SQ_FP32
    c = cells.vacancy_cell()
    if args.profile:   # small case for ncu
        c.K = 8
    d_veff = torch.from_numpy(np.ascontiguousarray(c.veff.reshape(-1))).cuda()
    rho = torch.empty(c.N_d, dtype=torch.float64, device="cuda")
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    h = sq.build_for_cell(c, d_veff=d_veff)

    def step():
        return sq.sq_density(h, c.K, c.kT, c.N_e, precision, sq.SQ_GAUSS, rho)

    if args.profile:
        step()
        torch.cuda.synchronize()
        print(json.dumps({"profile_case": "gauss", "K": c.K, "kernel": sq.sq_kernel_name(h)}), flush=True)
        h.close()
        return
    for _ in range(args.warmup):
        step()
    times, lam = [], None
    launches0 = sq.sq_kernel_launches()
    with ClockSampler(int(os.environ.get("LOCAL_RANK", "0"))) as clk:
        for _ in range(args.steps):
            flush.fill_(1.0)
            torch.cuda.synchronize()
            barrier()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            lam = step()
            e1.record(stream)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
    launches = (sq.sq_kernel_launches() - launches0) / max(1, args.steps)
    U, S, _ = sq.sq_energy(h)
    kname = sq.sq_kernel_name(h)
    tim = sq.sq_get_timing(h)
    h.close()
    ms = statistics.mean(times)
    if rank == 0:
        print(json.dumps({"metric": "SQ density grid-points/sec, Gauss (Lanczos) quadrature", "unit": UNIT,
                          "value": world * c.N_d / (ms * 1e-3), "n_gpus": world, "steps": args.steps,
                          "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
                          "vs_baseline": None, "dtype": "f32" if precision else "f64", "data": "synthetic",
                          "config": dict(workload_config(c), quadrature="Gauss (Lanczos), SQ_GAUSS",
                                         l2="flushed between steps (256 MiB write)"),
                          "kernel": kname, "timing_ms": tim, "gpu_launches": launches,
                          "results": {"lambda_f": lam, "U": U, "S": S}, "clocks": clk.summary()}), flush=True)


def run_scf(args, sq, torch, world, rank, barrier, dist):
    """The SCF loop of the vacancy cell (Sec. 3 flow): per iteration the build of V_in, the SQ density
    (FP32 unless --precision fp64), the effective potential (pseudocharges, Poisson, LDA) and an Anderson
    step (beta 0.3, history 5), until |V_out - V_in| / |V_out| <= 1e-6 or 40 iterations.  One step of
    this workload is one SCF iteration."""
    precision = sq.SQ_FP64 if args.precision == "fp64" else sq.SQ_FP32
    c = cells.vacancy_cell()
    if args.profile:
        c.K = 8
    N, sig = c.N_d, 1.0
    Z = np.array([float(cells.VALENCE[int(t)]) for t in c.species])
    b = torch.empty(N, dtype=torch.float64, device="cuda")
    sq.sq_pseudocharge(c.n, c.box, c.R, Z, sig, b)
    v_in = torch.from_numpy(np.ascontiguousarray(c.veff.reshape(-1))).cuda()
    rho, phi, exc, vxc, v_out = [torch.empty(N, dtype=torch.float64, device="cuda") for _ in range(5)]
    mixer = sq.sq_mixer_create(N, history=5, beta=0.3)
    stream = torch.cuda.current_stream()

    def iteration():
        h = sq.build_for_cell(c, d_veff=v_in)
        sq.sq_density(h, c.K, c.kT, c.N_e, precision, 0, rho)
        h.close()
        sq.sq_effective_potential(c.n, c.box, c.fd_order, rho, b, phi, exc, vxc, v_out, tol=1e-10)
        return sq.sq_mixer_step(mixer, v_in, v_out, v_in)

    errs = [iteration() for _ in range(max(args.warmup, 3))]
    times = []
    with ClockSampler(int(os.environ.get("LOCAL_RANK", "0"))) as clk:
        for _ in range(args.steps):
            torch.cuda.synchronize()
            barrier()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            errs.append(iteration())
            e1.record(stream)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
    mixer.close()
    ms = statistics.mean(times)
    if rank == 0:
        print(json.dumps({"metric": "SCF iterations (SQ density + effective potential + mixing) grid-points/sec",
                          "value": world * N / (ms * 1e-3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
                          "warmup": max(args.warmup, 3), "ms_per_step": ms, "higher_is_better": True,
                          "scaling": "weak", "vs_baseline": None, "dtype": "f32" if precision else "f64",
                          "data": "synthetic", "config": dict(workload_config(c), mixing="Anderson, beta 0.3, history 5",
                                                              pseudocharge_sigma=sig),
                          "scf_errors": errs, "clocks": clk.summary()}), flush=True)


def golden_errors(cell, lam, U, S, rho, force):
    """Errors of one result against the FP64 oracle's golden values of the same cell (written by
    tests/golden/make_golden.py): the rho error stated beside each throughput number."""
    path = os.path.join(GOLDEN, f"{cell.name}.json")
    if not os.path.exists(path):
        return None
    g = json.load(open(path))
    if g.get("digest") != cell.digest():
        return {"error": "golden file does not match the generated cell"}
    idx = np.array(g["rho_idx"])
    gr = np.array(g["rho"])
    d = np.abs(rho[idx] - gr)
    return {"dlambda_f": abs(lam - g["lam_f"]), "dU_per_atom": abs(U - g["U"]) / cell.natom,
            "dS_rel": abs(S - g["S"]) / abs(g["S"]),
            "force_max_abs": float(np.max(np.abs(force - np.array(g["force"])))),
            "rho_max_rel": float(d.max() / np.abs(gr).max()),
            "rho_rel_l1": float(d.sum() / np.abs(gr).sum()),
            "rho_points": int(idx.size),
            "units": "lambda_f Ha; U Ha/atom; force Ha/bohr; rho over the sampled points: max |d rho| / max rho "
                     "and sum |d rho| / sum rho"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["fp32", "fp64", "both"], default="both")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-vacancy", action="store_true", help="skip the extra vacancy-cell line")
    ap.add_argument("--fp64-steps", type=int, default=1,
                    help="timed steps of the secondary FP64 measurement (0: same as --steps)")
    ap.add_argument("--workload", choices=["precision", "vacancy", "batch", "adjoint", "gauss", "scf"], default="precision",
                    help="precision: the headline line (286-atom cell, 29^3 cubes, K=80); vacancy: the 95-atom "
                         "cell alone; batch: 32 defect cells in one graph-captured batch; adjoint: the "
                         "reverse-mode derivative of the vacancy cell; gauss: Gauss (Lanczos) quadrature on "
                         "the vacancy cell; scf: SCF iterations of the vacancy cell")
    ap.add_argument("--kb", choices=["mma", "fma"], default="mma",
                    help="projector term of the FP32 cluster kernel (29^3 cubes): tensor cores (3xTF32 warp MMAs) "
                         "or CUDA-core FMAs (SQ_KB_FMA)")
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
    if args.workload == "gauss":
        run_gauss(args, sq, torch, world, rank, barrier, dist)
        return
    if args.workload == "scf":
        run_scf(args, sq, torch, world, rank, barrier, dist)
        return
    stream = torch.cuda.current_stream()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    KB_FLAGS = sq.SQ_KB_FMA if args.kb == "fma" else 0

    class Workload:
        def __init__(self, cell):
            self.cell = cell
            self.d_veff = torch.from_numpy(np.ascontiguousarray(cell.veff.reshape(-1))).cuda()
            self.rho = torch.empty(cell.N_d, dtype=torch.float64, device="cuda")
            self.force = torch.empty((cell.natom, 3), dtype=torch.float64, device="cuda")

        def step(self, precision, K=None):
            c = self.cell
            h = sq.build_for_cell(c, d_veff=self.d_veff)
            lam = sq.sq_density(h, c.K if K is None else K, c.kT, c.N_e, precision, sq.SQ_WANT_FORCE | KB_FLAGS,
                                self.rho)
            U, S, F = sq.sq_energy(h)
            sq.sq_nonlocal_force(h, self.force)
            timing = sq.sq_get_timing(h)
            kname = sq.sq_kernel_name(h)
            h.close()
            return lam, U, S, timing, kname

        def measure(self, precision, steps, warmup, warm_K=None):
            for _ in range(warmup):
                self.step(precision, K=warm_K)
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
                    res = self.step(precision)
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
            torch.cuda.synchronize()
            out = dict(ms=ms, rec_ms=statistics.mean(rec), clocks=clk.summary(), launches=launches,
                       lam_f=res[0], U=res[1], S=res[2], kernel=res[4], steps=steps,
                       rho=self.rho.cpu().numpy().copy(), force=self.force.cpu().numpy().copy(),
                       value=world * self.cell.N_d / (ms * 1e-3))
            return out

        def e2e(self, precision, steps):
            """Through the public API with host buffers: V_eff from pinned host memory in, rho and forces
            back to pinned host memory, all inside the timed region."""
            c = self.cell
            host_veff = torch.from_numpy(np.ascontiguousarray(c.veff.reshape(-1))).pin_memory()
            host_rho = torch.empty(c.N_d, dtype=torch.float64).pin_memory()
            host_f = torch.empty((c.natom, 3), dtype=torch.float64).pin_memory()
            dv = torch.empty_like(self.d_veff)
            times = []
            for i in range(steps + 1):
                flush.zero_()
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                dv.copy_(host_veff, non_blocking=True)
                h = sq.build_for_cell(c, d_veff=dv)
                sq.sq_density(h, c.K, c.kT, c.N_e, precision, sq.SQ_WANT_FORCE | KB_FLAGS, self.rho)
                sq.sq_energy(h)
                sq.sq_nonlocal_force(h, self.force)
                host_rho.copy_(self.rho, non_blocking=True)
                host_f.copy_(self.force, non_blocking=True)
                torch.cuda.synchronize()
                h.close()
                if i > 0:
                    times.append(time.perf_counter() - t0)
            bi = c.N_d * 8
            bo = c.N_d * 8 + c.natom * 3 * 8
            return c.N_d / statistics.mean(times), bi, bo

    main_cell = cells.vacancy_cell() if args.workload == "vacancy" else cells.precision_cell()
    wl = Workload(main_cell)
    if args.profile:
        for p in (["fp32", "fp64"] if args.precision == "both" else [args.precision]):
            lam, U, S, timing, kname = wl.step(sq.SQ_FP32 if p == "fp32" else sq.SQ_FP64, K=8)
            torch.cuda.synchronize()
            print(json.dumps({"profile_case": p, "cell": main_cell.name, "K": 8, "kernel": kname,
                              "recursion_ms": timing[0], "lambda_f": lam}))
        return

    # measured FMA ceilings of this GPU (outside the timed region)
    fma = {"fp32": sq.sq_fma_throughput(sq.SQ_FP32)[0], "fp64": sq.sq_fma_throughput(sq.SQ_FP64)[0]}
    mma = {"tf32_m16n8k8": sq.sq_mma_throughput(0)[0], "bf16_m16n8k16": sq.sq_mma_throughput(1)[0]}
    flops_ball = algorithmic_flops_ball(main_cell)
    flops_box = algorithmic_flops(main_cell)

    def roofline(p, r, fb, fx):
        peak = fma[p]
        unit_peak = FP32_UNIT_TFLOPS if p == "fp32" else FP64_NOMINAL_TFLOPS
        ach = fb / (r["rec_ms"] * 1e-3) / 1e12
        ach_box = fx / (r["rec_ms"] * 1e-3) / 1e12
        return {"bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
                "traffic": MEASURED_TRAFFIC.get(r["kernel"]), "traffic_note": TRAFFIC_NOTE.get(r["kernel"]),
                "kernel": r["kernel"], "kernel_ms": r["rec_ms"],
                "count": "ball supports r < r_c (the hot-path measurement plan's count)",
                "algorithmic_tflop_per_launch": fb / 1e12,
                "achieved_box_count": ach_box, "frac_box_count": ach_box / peak,
                "algorithmic_tflop_per_launch_box_count": fx / 1e12,
                "peak_source": f"measured: sq_fma_throughput({p}) on this GPU in this run",
                "peak_unit_count": unit_peak, "frac_of_unit_count": ach / unit_peak,
                "unit_count_source": ("152 SM x 128 FP32 lanes x 2 x 2.07 GHz" if p == "fp32"
                                      else "nominal GB300 FP64 rate"),
                "projector_term": ("tensor cores: 3xTF32 warp MMAs (m16n8k8), FP32 accumulation; the stencil "
                                   "and the rest on the FP32 pipes" if r["kernel"].endswith(",mma>")
                                   else "FMA pipes")}

    precs = ["fp32", "fp64"] if args.precision == "both" else [args.precision]
    results = {}
    for p in precs:
        code = sq.SQ_FP32 if p == "fp32" else sq.SQ_FP64
        if p == precs[0]:
            r = wl.measure(code, args.steps, args.warmup)
            r["warmup"] = args.warmup
        else:
            # the FP64 recursion runs at the GPU's FP64 rate (minutes per step on this cell): a single
            # timed step, after one warm-up step at K = 2 (module load, buffers, every kernel once)
            steps = args.steps if args.fp64_steps <= 0 else args.fp64_steps
            r = wl.measure(code, steps, 1, warm_K=2)
            r["warmup"] = "1 step at K=2"
        r["roofline"] = roofline(p, r, flops_ball, flops_box)
        r["vs_oracle"] = golden_errors(main_cell, r["lam_f"], r["U"], r["S"], r["rho"], r["force"])
        results[p] = r
    main_p = precs[0]
    m = results[main_p]
    e2e_value, bi, bo = wl.e2e(sq.SQ_FP32 if main_p == "fp32" else sq.SQ_FP64, max(1, min(args.steps, 2)))
    line = {
        "metric": METRIC, "value": m["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": m["ms"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32" if main_p == "fp32" else "f64", "data": "synthetic",
        "config": dict(workload_config(main_cell), parallelism=f"replicas x{world}" if world > 1 else "single GPU",
                       recursion_precision=main_p, projector_path=args.kb),
        "roofline": m["roofline"], "clocks": m["clocks"], "gpu_launches": m["launches"],
        "e2e": {"value": world * e2e_value, "unit": UNIT, "h2d_bytes_per_step": bi, "d2h_bytes_per_step": bo},
        "results": {"lambda_f": m["lam_f"], "U": m["U"], "S": m["S"]},
        "vs_oracle": m["vs_oracle"],
        "fma_peaks_tflops": fma,
        "warp_mma_peaks_tflops": mma,
    }
    for p in precs[1:]:
        r = results[p]
        line[p] = {"value": r["value"], "ms_per_step": r["ms"], "steps": r["steps"], "warmup": r["warmup"],
                   "roofline": r["roofline"], "clocks": r["clocks"], "gpu_launches": r["launches"],
                   "results": {"lambda_f": r["lam_f"], "U": r["U"], "S": r["S"]}, "vs_oracle": r["vs_oracle"]}
    if "fp32" in results and "fp64" in results:
        r32, r64 = results["fp32"], results["fp64"]
        drho = np.abs(r32["rho"] - r64["rho"])
        line["fp32_vs_fp64"] = {"rho_rel_l1": float(drho.sum() * float(np.prod(main_cell.h)) / main_cell.N_e),
                                "rho_max_rel": float(drho.max() / np.abs(r64["rho"]).max()),
                                "dU_per_atom": abs(r32["U"] - r64["U"]) / main_cell.natom,
                                "force_max_abs": float(np.abs(r32["force"] - r64["force"]).max()),
                                "dlambda_f": abs(r32["lam_f"] - r64["lam_f"]),
                                "units": "rho_rel_l1 = sum|d rho| dV / N_e over all points; rho_max_rel = "
                                         "max|d rho| / max rho; dU Ha/atom; force Ha/bohr; lambda_f Ha",
                                "speedup": r32["value"] / r64["value"]}
    if args.workload == "precision" and not args.no_vacancy and "fp32" in precs:
        vc = cells.vacancy_cell()
        wv = Workload(vc)
        rv = wv.measure(sq.SQ_FP32, 3, 3)
        fv = algorithmic_flops_ball(vc)
        line["vacancy_fp32"] = {"workload": workload_config(vc)["workload"], "value": rv["value"],
                                "ms_per_step": rv["ms"], "steps": 3, "warmup": 3,
                                "roofline": roofline("fp32", rv, fv, algorithmic_flops(vc)),
                                "vs_oracle": golden_errors(vc, rv["lam_f"], rv["U"], rv["S"], rv["rho"], rv["force"])}
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(main_cell)
    if dist is not None:
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
