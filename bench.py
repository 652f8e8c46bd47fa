"""Benchmark of the fused MUSCL-Hancock step (one JSON line on rank 0).

Workload (default): 1D periodic grid of N = 2^22 cells, h = 1/1024 (L = 4096
base wavelengths), FP32 state, gamma 1.4, C_k 0.1, tau_rho -1, tau_T -1.5,
Q/I exponents 0, S 1, tau0 0.08, CFL 0.4, seeded sum of 64 random-phase
acoustic modes with k_i = 2 pi i / 32 (i = 1..64) and amplitudes 1e-3 / i.
A "step" is one MUSCL-Hancock time step of the whole grid (one launch of the
fused kernel).  The state (64 MiB per buffer) fits in L2, so L2 is flushed by a
256 MiB write before every timed step and each step is timed alone with CUDA
events on the solver's stream.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--precision fp32|fp64|fp32_p64|fp32_pc|fp32_ps] [--n CELLS]

Under torchrun (N > 1) every rank runs an independent replica (the 1D problem
is not sharded: "replicas only"); value = all ranks' cell-updates / max time.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "cell-updates/s"
L2_FLUSH_BYTES = 256 << 20

# DRAM bytes (read + write) of one launch of the 1D FP32 step at N = 2^22, per launch
# configuration (a substring of its description), from one ncu capture of the current kernels
# with ncu's default cache control (caches flushed before the launch, as the benchmark's steps):
# the block tiles read the state once (plus the first tile of the other buffer, 2.5 MB) and write
# part of it back during the launch (the rest is still dirty in L2 when it ends); the sliding warps
# re-read their chunk halos.  Only valid for that workload and precision; other lines, and
# configurations without a capture, report null.
TRAFFIC_1D_FP32_N22 = {
    "512-cell block tiles, 2 cells per thread, 78 registers, 3 blocks/SM": 89.7e6,
    "512-cell block tiles, 2 cells per thread, 2 blocks/SM": 89.9e6,
    "1024-cell block tiles, 4 cells per thread, 2 blocks/SM": 86.2e6,
    "512-cell block tiles, 2 cells per thread, 64 registers, 4 blocks/SM": 90.0e6,
    "warps sliding over 64-cell chunks": 91.6e6,
}
# The same launch in steady state back to back (ncu --cache-control none on launches 100-102 of
# `bench.py --b2b --steps 64`, 3-blocks/SM tiles): each step writes back the previous step's dirty
# lines and finds ~5 MB of its input still in L2, 129.2 MB per launch against the algorithmic
# 134.2 MB.
TRAFFIC_B2B_1D_FP32_N22 = 129.2e6
# The 3D FP32 step at 512^3 (the field-pair kernel, segments of 128 planes), one-pass capture of
# the benchmark command itself: 4370.8 MB read + 3196.3 MB written against the algorithmic
# 6442.5 MB (the tiles' halo columns and rows are read by two blocks, each segment reads two
# extra planes).
TRAFFIC_3D_FP32_512 = {"segments of 128 planes": 7567.1e6}


def traffic_of(workload: str, ncell: int, precision: str, config: str):
    if precision != "fp32":
        return None
    if workload == "1d" and ncell == 1 << 22:
        table = TRAFFIC_1D_FP32_N22
    elif workload == "3d" and ncell == 512 ** 3:
        table = TRAFFIC_3D_FP32_512
    else:
        return None
    return next((v for k, v in table.items() if k in config), None)

# FP64 flops one updated cell costs in the FP64 step kernels of the benchmark grids (2 DFMA +
# DMUL + DADD, ncu warp-instruction counts x 32 lanes, the tiles' halo work included): step1d_kernel
# at N = 2^22 itself; stepnd_kernel on 4224^2 (2D) and 180^3 (3D), whose x-y tiles cover the grid
# with the same redundancy as 8192^2 and 512^3 do (a capture of the full FP64 grids would hold
# 5-6 GB), both scaled to the marching segments the benchmark grids run (two warm-up planes per
# segment: 2D 793.5 counted with 64-row segments, x (258/256) / (66/64) for the 256-row segments
# of 8192^2; 3D 1575.8 counted with 60-plane segments, x (520/512) / (186/180) for the 128-plane
# segments of 512^3).  With the paper's closure exponents (tau_rho = -1,
# tau_T = -1.5: the power laws of eq. 6 as products).  These kernels are bound by GB300's FP64 pipe
# (ncu: 86 % of its peak busy), so FP64 lines report an "alu" roofline.
FP64_FLOPS_PER_CELL = {1: 422.9, 2: 775.5, 3: 1548.8}

# --precision names -> sv_params.precision (SV_FP32, SV_FP64, SV_FP32_P64,
# SV_FP32_PC, SV_FP32_PS of include/sv.h) and the arithmetic type reported as "dtype"
PRECISIONS = {"fp32": 0, "fp64": 1, "fp32_p64": 2, "fp32_pc": 3, "fp32_ps": 4}
DTYPES = {"fp32": "f32", "fp64": "f64", "fp32_p64": "f32", "fp32_pc": "f32", "fp32_ps": "f32"}


def fp64_roofline(dim: int, ncell: int, step_s: float, hbm_frac: float, peak: float) -> dict:
    """The FP64 step as an ALU-bound kernel: FP64 flops per launch
    (FP64_FLOPS_PER_CELL) over the FP64 FMA rate the library's probe measured
    in this run (`peak`, TFLOP/s)."""
    flops = FP64_FLOPS_PER_CELL[dim] * ncell
    achieved = flops / step_s / 1e12
    return {"bound": "alu", "achieved": achieved, "peak": peak,
            "peak_src": "measured: DFMA-chain probe of the library (sv_measure_fp64_peak), this run",
            "unit": "TFLOP/s", "frac": achieved / peak, "traffic": None,
            "flops_per_launch": flops, "hbm_frac": hbm_frac}


def workload(n_cells: int, gamma: float, Ck: float, S: float):
    from paper_1805_03442_gb300 import inputs
    h = 1.0 / 1024
    L = n_cells * h
    m0 = max(1, int(round(L / 32.0)))            # k_1 = 2 pi / 32
    modes = inputs.random_phase_modes(2024, inputs.acoustic_shape(gamma), 64, m0, 1e-3, m_step=m0)
    U0 = inputs.waves_1d(gamma, n_cells, L, inputs.equilibrium_primitive(Ck, S), modes)
    return U0, h, L


# Workloads: name -> (grid, params, description, steps of the per-field error run
# against FP64).  The 1D line is the default.
WORKLOADS = {
    "1d": dict(dims=lambda a: (a.n,), params=dict(tau0=0.08, S=1.0, cfl=0.4), err_steps=200,
               desc="1D periodic MUSCL-Hancock step, N={cells} cells, h=1/1024, 64 random-phase "
                    "acoustic modes (k^-1, 1e-3), S=1, tau0=0.08, CFL 0.4"),
    "2d": dict(dims=lambda a: (a.side or 8192,) * 2, params=dict(tau0=0.01, S=1.0, cfl=0.4),
               err_steps=50,
               desc="2D periodic unsplit MUSCL-Hancock step, {side}x{side}, plane wave (7,4) at 29.7 deg "
                    "amplitude 1e-3 + white noise 1e-5, S=1, tau0=0.01, CFL 0.4"),
    "3d": dict(dims=lambda a: (a.side or 512,) * 3, params=dict(tau0=0.08, S=1.0, cfl=0.3),
               err_steps=20,
               desc="3D periodic unsplit MUSCL-Hancock step, {side}^3, isotropic k^-2 random density/"
                    "velocity perturbations amplitude 1e-3, S=1, tau0=0.08, CFL 0.3"),
}


def make_state(name: str, dims, gamma: float, Ck: float, S: float):
    """Initial state (nf, ncell) float64, cell size h, lengths L."""
    from paper_1805_03442_gb300 import inputs
    base = inputs.equilibrium_primitive(Ck, S)
    if name == "1d":
        U0, h, L = workload(dims[0], gamma, Ck, S)
        return U0, h, (L,)
    n = dims[0]
    h = 1.0 / n
    if name == "2d":
        return inputs.plane_wave_2d(gamma, dims[0], dims[1], 1.0, base, 7, 4, 1e-3, 1e-5, 3), h, (1.0, 1.0)
    return inputs.random_field_3d(gamma, n, 1.0, base, 1e-3, seed=5), h, (1.0, 1.0, 1.0)


def peaks() -> dict:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return {"hbm_gbs": float(d["hbm_gbs"]), "src": "measured"}
    except Exception:
        return {"hbm_gbs": 6800.0, "src": "fallback"}


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.p = None
        self.index = index

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "100"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.p = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        self.result = {"sm_mhz": None, "sm_max_mhz": None, "reasons": []}
        if self.p is None:
            return
        time.sleep(0.2)
        self.p.terminate()
        try:
            out, _ = self.p.communicate(timeout=5)
        except Exception:
            self.p.kill()
            out = ""
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower() == "active":
                    reasons.add(nm)
        if sm:
            self.result = {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                           "reasons": sorted(reasons), "samples": len(sm)}


def cpu_baseline(name: str, args, budget_s: float = 10.0) -> dict:
    """The FP64 oracle, as it stands, on the same workload: whole-grid steps
    until `budget_s` of wall time (at least one).  2D / 3D use a periodic
    sub-grid of the same generator (2048^2 / 128^3) to stay within budget."""
    from oracle import orc as O
    W = WORKLOADS[name]
    P = O.Params(**W["params"])
    dims = W["dims"](args)
    if name == "2d":
        dims = (2048, 2048)
    elif name == "3d":
        dims = (128, 128, 128)
    U, h, _ = make_state(name, dims, P.gamma, P.Ck, P.S)
    ncell = int(np.prod(dims))

    def timed(U, budget):
        steps, t0 = 0, time.perf_counter()
        while True:
            dt = O.dt_cfl(P, U, dims, h)
            U, rc = O.step(P, U, dims, h, dt)
            steps += 1
            el = time.perf_counter() - t0
            if el >= budget:
                return U, steps, el

    cores = O.threads()
    U1, steps, el = timed(U, budget_s)
    # the same oracle on one thread (shorter sample), then all cores again
    O.set_threads(1)
    try:
        _, steps1, el1 = timed(U, max(3.0, budget_s / 3))
    finally:
        O.set_threads(cores)
    return {"value": ncell * steps / el, "unit": METRIC, "cores": cores, "kind": "oracle",
            "single_thread_value": ncell * steps1 / el1,
            "sample": f"{steps} whole-grid FP64 oracle steps of the {name} workload on "
                      f"{'x'.join(map(str, dims))} cells ({el:.1f} s wall; one thread: "
                      f"{steps1} steps, {el1:.1f} s)"}


def wc_problem(N: int):
    """Colliding shock waves (Sec. 2.4): rho = 1, u = 0, p = 1000 / 0.01 / 100 on
    [0, 0.1) / [0.1, 0.9] / (0.9, 1], passive e_nu 0.3, frozen gas, walls."""
    from paper_1805_03442_gb300 import inputs
    x = inputs.cell_centres(N, 1.0)
    p = np.where(x < 0.1, 1000.0, np.where(x <= 0.9, 0.01, 100.0))
    U0 = inputs.prim_to_cons(1.4, np.ones(N), [np.zeros(N)], p, np.full(N, 0.3))
    return dict(tau0=math.inf, S=0.0), U0, 0.038


def driven_problem(N: int, gamma: float = 1.4, Ck: float = 0.1, S: float = 0.5):
    """Forced source (Sec. 3): the uniform equilibrium of S = 0.5, tau0 =
    0.0135, and the boundary wave of wavelength 0.1 (frozen acoustic shape,
    amplitude 1e-4): (params, U0, base state, amplitude vector, omega, k)."""
    from paper_1805_03442_gb300 import inputs
    rho0, p0, ev0 = inputs.equilibrium_primitive(Ck, S)
    base = inputs.prim_to_cons(gamma, np.array([rho0]), [np.array([0.0])], np.array([p0]),
                               np.array([ev0]))[:, 0]
    w = 2 * math.pi / 0.1 * math.sqrt(gamma)
    shape = inputs.acoustic_shape(gamma)          # rho', u', p', e_nu' of a frozen wave
    amp = 1e-4 * np.array([shape[0], shape[1], shape[2] / (gamma - 1.0) + ev0 * shape[0],
                           ev0 * shape[0]])
    U0 = np.repeat(base[:, None], N, axis=1)
    return dict(S=S, tau0=0.0135), U0, base, amp, w, w / math.sqrt(gamma)


def oracle_rate(advance, ncell: int, budget_s: float):
    """Cell-updates/s of the oracle: `advance(k)` runs k more steps and returns
    the number it ran (0 once its run has ended); called with growing k until
    `budget_s` of wall time.  Returns (rate, steps, seconds)."""
    steps, k, t0 = 0, 4, time.perf_counter()
    while True:
        done = advance(k)
        steps += done
        el = time.perf_counter() - t0
        if el >= budget_s or done == 0:
            break
        k = min(2 * k, 4096)
    return (ncell * steps / el if steps else 0.0), steps, el


def oracle_special(name: str, args, budget_s: float) -> dict:
    """The FP64 oracle, as it stands, on the colliding-shock, forced-source,
    active-sector and sweep workloads: a bounded sample of the same run(s).
    The sweep's value is runs/s, extrapolated from the oracle's cell-update
    rate over a stratified sample to the cell-updates the whole sweep needs
    (each run: N cells x t_end / its initial eq.-16 step)."""
    from oracle import orc as O
    from paper_1805_03442_gb300 import inputs
    if name == "wc":
        N = args.n if args.n != 1 << 22 else 100000
        prm, U, t_end = wc_problem(N)
        Po = O.Params(**prm)
        st = {"U": U, "t": 0.0}

        def adv(k):
            U2, t, n, rc = O.run_bc1(Po, st["U"], N, 1.0 / N, t_end, O.REFLECT, O.REFLECT,
                                     t0=st["t"], max_steps=k)[:4]
            st["U"], st["t"] = U2, t
            return n if rc == 0 and t < t_end else 0
        rate, steps, el = oracle_rate(adv, N, budget_s)
        return {"value": rate, "unit": METRIC, "cores": O.threads(), "kind": "oracle",
                "sample": f"first {steps} oracle steps of the colliding-shock run, N={N} "
                          f"({el:.1f} s wall)"}
    if name == "driven":
        N = args.n if args.n != 1 << 22 else 1 << 16
        prm, U, base, amp, w, kk = driven_problem(N)
        Po = O.Params(**prm)
        drv = O.drive(w, kk, base, amp)
        st = {"U": U, "t": 0.0}

        def adv(k):
            U2, t, n, rc = O.run_driven(Po, st["U"], N, 1.0 / N, 1.0, drv, t0=st["t"],
                                        max_steps=k)[:4]
            st["U"], st["t"] = U2, t
            return n if rc == 0 and t < 1.0 else 0
        rate, steps, el = oracle_rate(adv, N, budget_s)
        return {"value": rate, "unit": METRIC, "cores": O.threads(), "kind": "oracle",
                "sample": f"first {steps} oracle steps of the forced-source run, N={N} "
                          f"({el:.1f} s wall)"}
    if name == "sector":
        pb = inputs.sector_problem(args.side or 2048)
        Po = O.Params(S=1.0, tau0=0.0135)
        U = inputs.sector_rest_state(Po.gamma, Po.Ck, Po.S, pb.nx, pb.ny)
        lo, hi, dlo, dhi = pb.maps
        med = O.Medium2(lo, hi, dlo, dhi, pb.omega, pb.amp)
        st = {"U": U, "t": 0.0}

        def adv(k):
            U2, t, n, rc = O.run2m(Po, st["U"], pb.nx, pb.ny, pb.h, 1.2, pb.bc, med, t0=st["t"],
                                   max_steps=k)[:4]
            st["U"], st["t"] = U2, t
            return n if rc == 0 and t < 1.2 else 0
        rate, steps, el = oracle_rate(adv, pb.nx * pb.ny, budget_s)
        return {"value": rate, "unit": METRIC, "cores": O.threads(), "kind": "oracle",
                "sample": f"first {steps} oracle steps of the active-sector run, "
                          f"{pb.nx}x{pb.ny} ({el:.1f} s wall)"}
    if name == "sweep":
        runs, states = sweep_inputs(args.runs)
        cost = [r.N * r.t_end / O.dt_cfl(_oracle_params(O, r), st, r.N, 1.0 / r.N)
                for r, st in zip(runs, states)]
        order = sorted(range(len(runs)), key=lambda i: cost[i])
        sample = order[:: max(1, len(runs) // 64)]
        cells, t0, used = 0, time.perf_counter(), 0
        for i in sample:
            r = runs[i]
            _, _, n, _ = O.run(_oracle_params(O, r), states[i], r.N, 1.0 / r.N, r.t_end,
                               max_steps=max(1, int(2e6 // r.N)))[:4]
            cells += n * r.N
            used += 1
            if time.perf_counter() - t0 >= budget_s:
                break
        el = time.perf_counter() - t0
        rate = cells / el
        return {"value": len(runs) / (sum(cost) / rate), "unit": "runs/s", "cores": O.threads(),
                "kind": "oracle", "cell_updates_per_s": rate,
                "sample": f"up to 2e6 cell-updates of each of {used} runs of a cost-stratified "
                          f"sample ({el:.1f} s wall), extrapolated to the sweep's "
                          f"{sum(cost):.3g} cell-updates (N t_end / initial dt per run)"}
    raise ValueError(name)


def _oracle_params(O, r):
    return O.Params(S=r.S, tau0=r.tau0, tau_rho=r.tau_rho, tau_T=r.tau_T, Q_rho=r.Q_rho,
                    Q_T=r.Q_T, I_rho=r.I_rho, I_T=r.I_T)


def dist_init():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws <= 1:
        return 0, 1, None
    import torch.distributed as dist
    backend = "nccl"
    try:
        import torch
        if not torch.cuda.is_available():
            backend = "gloo"
    except Exception:
        backend = "gloo"
    dist.init_process_group(backend)
    return dist.get_rank(), dist.get_world_size(), dist


def aggregate(local_seconds: float, local_units: float, dist=None, device: str = "cpu"):
    """Whole-job figures over ranks: (max time over ranks, units of all ranks).
    Works with gloo (CPU tensors) and nccl (CUDA tensors)."""
    if dist is None:
        return local_seconds, local_units
    import torch
    t = torch.tensor([local_seconds], dtype=torch.float64, device=device)
    u = torch.tensor([local_units], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def run_reference(args):
    rank, ws, dist = dist_init()
    if rank != 0:
        return
    from oracle import orc as O
    if args.workload not in WORKLOADS:
        # bounded samples of the same runs; value in the GPU line's unit
        base = oracle_special(args.workload, args, budget_s=max(args.cpu_budget, 10.0))
        unit = base["unit"]
        line = {"impl": "reference", "metric": "batched sweep runs/s" if unit == "runs/s" else METRIC,
                "value": base["value"], "unit": unit, "n_gpus": 1, "steps": 1, "warmup": 0,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic", "config": {"workload": args.workload},
                "cpu_baseline": base,
                "e2e": {"value": base["value"], "unit": unit, "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return
    W = WORKLOADS[args.workload]
    P = O.Params(**W["params"])
    dims = W["dims"](args)
    # bounded sample: 2D / 3D steps on a periodic sub-grid of the same
    # generator (an oracle step of the full 8192^2 / 512^3 grid takes seconds)
    if args.workload == "2d":
        dims = (min(dims[0], 2048),) * 2
    elif args.workload == "3d":
        dims = (min(dims[0], 128),) * 3
    U, h, _ = make_state(args.workload, dims, P.gamma, P.Ck, P.S)
    ncell = int(np.prod(dims))
    for _ in range(args.warmup):
        U, _ = O.step(P, U, dims, h, O.dt_cfl(P, U, dims, h))
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        U, _ = O.step(P, U, dims, h, O.dt_cfl(P, U, dims, h))
        times.append(time.perf_counter() - t0)
    tot = sum(times)
    value = ncell * args.steps / tot
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": W["desc"].format(cells=ncell, side=dims[0]), "cells": ncell,
                       "precision": args.precision},
            "cpu_baseline": {"value": value, "unit": METRIC, "cores": O.threads(), "kind": "oracle",
                             "sample": f"{args.steps} whole-grid FP64 oracle steps of the "
                                       f"workload on {'x'.join(map(str, dims))} cells"},
            "e2e": {"value": value, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def timed_flushed_steps(solver, stream, flush, steps: int, warmup: int) -> list:
    """Per-step seconds of `steps` single steps, each after an L2-evicting
    write (outside its CUDA-event window), after `warmup` untimed steps."""
    import torch
    for _ in range(warmup):
        with torch.cuda.stream(stream):
            flush.fill_(1.0)
        solver.step(1)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    for i in range(steps):
        with torch.cuda.stream(stream):
            flush.fill_(float(i))
            ev[i][0].record(stream)
        solver.step(1)
        with torch.cuda.stream(stream):
            ev[i][1].record(stream)
    torch.cuda.synchronize()
    return [a.elapsed_time(b) * 1e-3 for a, b in ev]


def back_to_back(solver, stream, flush, steps: int, alg_bytes: int, hbm_gbs: float) -> dict:
    """`steps` steps replayed back to back from the solver's CUDA graph with
    no flush between them (one CUDA-event window after one L2-evicting write):
    the write-back of each step's dirty lines is paid inside the window, and
    part of each step's input is still in L2 from the step before."""
    import torch
    with torch.cuda.stream(stream):
        flush.fill_(2.0)
    solver.step(steps)                      # warm: the graph is built and replayed once
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        flush.fill_(3.0)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    solver.step(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    t = e0.elapsed_time(e1) * 1e-3 / steps
    out = {"value": solver.ncell / t, "unit": METRIC, "ms_per_step": 1e3 * t, "steps": steps,
           "l2": "one flush before the window, none between steps",
           "alg_gbs": alg_bytes / t / 1e9, "frac": alg_bytes / t / 1e9 / hbm_gbs}
    if solver.ncell == 1 << 22 and solver.params.precision == 0:
        out["traffic"] = TRAFFIC_B2B_1D_FP32_N22
    return out


def precision_leg(sv, args, prec_name: str, U0, dims, L, stream, flush, pk: dict) -> dict:
    """The default workload in another arithmetic policy, timed as the main
    line (L2 flushed before each step): FP64 (roofline of the FP64 pipe,
    measured by the library's probe, and one step against the oracle on
    sampled cells) or a float pressure policy (HBM roofline, per-field error
    against the FP64 kernels)."""
    from paper_1805_03442_gb300 import tune
    W = WORKLOADS[args.workload]
    prec = PRECISIONS[prec_name]
    P = sv.Params(precision=prec, **W["params"])
    ncell = int(np.prod(dims))
    with sv.Solver(P, dims, L, stream=stream) as s:
        s.write_state(U0)
        tuned = tune.tune_solver(s, tune.solver_key(P, dims), tune.device_name(), cold=True)
        times = timed_flushed_steps(s, stream, flush, args.steps, args.warmup)
        status = s.status()
    step_s = sum(times) / len(times)
    esize = 8 if prec == sv.FP64 else 4
    alg = 2 * (len(dims) + 3) * esize * ncell
    out = {"precision": prec_name, "value": ncell / step_s, "unit": METRIC,
           "ms_per_step": 1e3 * step_s, "steps": len(times), "launch_config": tuned["config"],
           "status_flags": status}
    if prec == sv.FP64:
        peak = sv.measure_fp64_peak(stream)
        flops = FP64_FLOPS_PER_CELL[len(dims)] * ncell
        out["roofline"] = {"bound": "alu", "achieved": flops / step_s / 1e12, "peak": peak,
                           "peak_src": "measured: DFMA-chain probe of the library "
                                       "(sv_measure_fp64_peak), this run",
                           "unit": "TFLOP/s", "frac": flops / step_s / 1e12 / peak,
                           "traffic": None, "flops_per_launch": flops,
                           "hbm_frac": alg / step_s / 1e9 / pk["hbm_gbs"]}
        out["error_vs_oracle"] = fp64_sampled_parity(sv, P, dims, L, U0)
    else:
        out["roofline"] = {"bound": "hbm", "achieved": alg / step_s / 1e9, "peak": pk["hbm_gbs"],
                           "unit": "GB/s", "frac": alg / step_s / 1e9 / pk["hbm_gbs"],
                           "traffic": None}
        if args.err_steps >= 0:
            out["error_vs_fp64"] = precision_error(sv, P, dims, L, U0,
                                                   args.err_steps or W["err_steps"])
    return out


def fp64_sampled_parity(sv, P, dims, L, U0, nsample: int = 64) -> dict:
    """One FP64 step of the workload against the oracle's one-cell evaluation
    on sampled cells: max |gpu - oracle| / max(|field|, 1) over the sample."""
    from oracle import orc as O
    Po = O.Params(gamma=P.gamma, Ck=P.Ck, S=P.S, tau0=P.tau0, tau_rho=P.tau_rho, tau_T=P.tau_T,
                  Q_rho=P.Q_rho, Q_T=P.Q_T, I_rho=P.I_rho, I_T=P.I_T, cfl=P.cfl, c_tau=P.c_tau,
                  limiter=P.limiter)
    ncell = int(np.prod(dims))
    h = L[0] / dims[0]
    with sv.Solver(P, dims, L) as s:
        s.write_state(U0)
        dt = s.dt()
        s.step(1)
        U, _ = s.read_state()
    rng = np.random.default_rng(1)
    idx = np.unique(np.concatenate([[0, 1, ncell - 1], rng.integers(0, ncell, nsample)]))
    scale = np.maximum(np.max(np.abs(U0), axis=1), 1.0)
    err = max(float(np.max(np.abs(U[:, i] - O.step_cell(Po, U0, dims, h, dt, int(i))) / scale))
              for i in idx)
    return {"max_rel": err, "cells": int(len(idx)), "dt_rel": abs(dt - O.dt_cfl(Po, U0, dims, h))
            / O.dt_cfl(Po, U0, dims, h), "norm": "max |gpu - oracle| / max(|field|, 1)"}


def run_ours(args):
    import torch
    rank, ws, dist = dist_init()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    from paper_1805_03442_gb300 import sv
    from paper_1805_03442_gb300.build import build
    if rank == 0 or not os.path.exists(sv.LIB_PATH):
        build()
    if dist is not None:
        dist.barrier()
    prec = PRECISIONS[args.precision]
    esize = 8 if prec == sv.FP64 else 4
    W = WORKLOADS[args.workload]
    P = sv.Params(precision=prec, **W["params"])
    dims = W["dims"](args)
    ncell = int(np.prod(dims))
    U0, h, L = make_state(args.workload, dims, P.gamma, P.Ck, P.S)
    stream = torch.cuda.Stream()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    solver = sv.Solver(P, dims, L, stream=stream)
    solver.write_state(U0)
    # launch configuration from the autotuner (timed on the initial state, which
    # it restores), outside the timed region; its trials flush L2 before every
    # step as the timed steps below do
    from paper_1805_03442_gb300 import tune
    if args.config >= 0:                     # a configuration named on the command line
        solver.set_config(args.config)
        tuned = {"config": solver.configs()[args.config], "index": args.config, "us": None,
                 "cached": False}
    else:
        tuned = tune.tune_solver(solver, tune.solver_key(P, dims), tune.device_name(), cold=True)
    torch.cuda.synchronize()
    timed_flushed_steps(solver, stream, flush, 0, args.warmup)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    with Clocks(local) as clk:
        if args.b2b:
            # diagnostic mode: the K steps replayed back to back from the
            # solver's graph in one CUDA-event window after one flush (the
            # graph is built by an untimed replay first)
            solver.step(args.steps)
            with torch.cuda.stream(stream):
                flush.fill_(3.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            solver.step(args.steps)
            e1.record(stream)
            torch.cuda.synchronize()
            times = [e0.elapsed_time(e1) * 1e-3 / args.steps] * args.steps
        else:
            times = timed_flushed_steps(solver, stream, flush, args.steps, 0)
    if dist is not None:
        dist.barrier()
    tot, units = aggregate(sum(times), float(ncell * args.steps), dist, device="cuda")
    status = solver.status()
    t_sim, nsteps = solver.time()

    # end to end through the C ABI: pinned host state in, one step, state out;
    # float host buffers for the float policies (their device state is float:
    # exact both ways, half the bytes of double buffers), double for FP64
    nf = len(dims) + 3
    f32_host = prec != sv.FP64

    def e2e_rate(host_f32: bool, steps: int):
        dt_ = torch.float32 if host_f32 else torch.float64
        hin = torch.from_numpy(U0.reshape(-1)).to(dt_).pin_memory()
        hout = torch.empty_like(hin).pin_memory()
        wr = solver.write_state_ptr_f32 if host_f32 else solver.write_state_ptr
        rd = solver.read_state_ptr_f32 if host_f32 else solver.read_state_ptr
        wr(hin.data_ptr())
        solver.step(1)
        rd(hout.data_ptr())
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(steps):
            wr(hin.data_ptr())
            solver.step(1)
            rd(hout.data_ptr())
        el = time.perf_counter() - t0
        return el, int(hin.numel() * hin.element_size()), int(hout.numel() * hout.element_size())

    e2e_steps = max(2, min(args.steps, 10))
    e2e_t, e2e_bi, e2e_bo = e2e_rate(f32_host, e2e_steps)
    e2e_f64 = e2e_rate(False, e2e_steps) if f32_host else None
    pk = peaks()
    fp64_peak = sv.measure_fp64_peak(stream) if args.precision == "fp64" else None
    esize_alg = 2 * nf * esize * ncell
    extras = ws == 1 and not args.no_extras and args.workload == "1d" and args.precision == "fp32"
    b2b = back_to_back(solver, stream, flush, 64, esize_alg, pk["hbm_gbs"]) if extras else None
    solver.close()

    if rank != 0:
        return
    err = None
    if prec != sv.FP64 and args.err_steps >= 0:
        err = precision_error(sv, P, dims, L, U0, args.err_steps or W["err_steps"])
    step_s = tot / args.steps
    alg_bytes = 2 * nf * esize * ncell             # read + write every conserved field once
    achieved = alg_bytes / step_s / 1e9
    value = units / tot
    line = {
        "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * step_s, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": DTYPES[args.precision],
        "data": "synthetic",
        "config": {"workload": W["desc"].format(cells=ncell, side=dims[0]), "cells": ncell,
                   "precision": args.precision,
                   "l2": ("one 256 MiB write before the window, steps back to back" if args.b2b
                          else "flushed by a 256 MiB write before every timed step"),
                   "parallelism": "replicas" if ws > 1 else "single GPU",
                   "launch_config": tuned["config"]},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": pk["hbm_gbs"],
                     "peak_src": f"{pk['src']} hbm_gbs (burst copy)", "unit": "GB/s",
                     "frac": achieved / pk["hbm_gbs"],
                     "traffic": traffic_of(args.workload, ncell, args.precision, tuned["config"]),
                     "alg_bytes_per_launch": alg_bytes},
        **({"roofline": fp64_roofline(len(dims), ncell, step_s, achieved / pk["hbm_gbs"],
                                      fp64_peak)}
           if args.precision == "fp64" else {}),
        "e2e": {"value": ws * ncell * e2e_steps / e2e_t, "unit": METRIC,
                "h2d_bytes_per_step": e2e_bi, "d2h_bytes_per_step": e2e_bo,
                "host_dtype": "f32" if f32_host else "f64",
                **({"value_f64_host_buffers": ws * ncell * e2e_steps / e2e_f64[0]}
                   if e2e_f64 else {})},
        "gpu_launches": args.steps,
        "clocks": getattr(clk, "result", None),
        "status_flags": status, "sim_time": t_sim,
    }
    if err is not None:
        line["error_vs_fp64"] = err
    if extras:
        # the rest of the metric on the same box: the same step back to back,
        # the FP64 kernels, the compensated-float pressure policy (the float
        # stand-in for the FP64 pressure island) and the batched sweep
        line["back_to_back"] = b2b
        line["fp64"] = precision_leg(sv, args, "fp64", U0, dims, L, stream, flush, pk)
        line["fp32_pc"] = precision_leg(sv, args, "fp32_pc", U0, dims, L, stream, flush, pk)
        del flush
        torch.cuda.empty_cache()
        line["sweep"] = sweep_summary(sweep_measure(args, stream, reps=1))
    if not args.no_cpu_baseline and ws == 1:
        line["cpu_baseline"] = cpu_baseline(args.workload, args, budget_s=args.cpu_budget)
    print(json.dumps(line), flush=True)


def precision_error(sv, P, dims, L, U0, steps: int) -> dict:
    """Per-field error of a float policy against the FP64 kernels (which match
    the FP64 oracle to 1e-12) on the benchmark's own workload: the float run
    takes `steps` steps of its own dt, the FP64 run is advanced to the same
    time (its last step clamped onto it), and rho, v, p, E_nu are compared cell
    by cell.  Absolute errors: L1 = mean over cells, Linf = maximum (v: every
    component)."""
    import dataclasses
    with sv.Solver(P, dims, L) as s:
        s.write_state(U0)
        s.step(steps)
        Uf, t = s.read_state()
        st = s.status()
    P64 = dataclasses.replace(P, precision=sv.FP64)
    with sv.Solver(P64, dims, L) as s:
        s.write_state(U0)
        rc, k = s.run_to(t, check=False)
        Ud, _ = s.read_state()
    dim = len(dims)

    def fields(U):
        U = U.reshape(dim + 3, -1)
        rho = U[0]
        v = np.stack([U[1 + a] / rho for a in range(dim)])
        kin = sum(U[1 + a] * v[a] for a in range(dim))
        return {"rho": rho, "v": v, "p": (P.gamma - 1.0) * (U[1 + dim] - 0.5 * kin - U[2 + dim]),
                "E_nu": U[2 + dim]}

    ff, fd = fields(Uf), fields(Ud)
    del Uf, Ud
    out = {}
    for name in ff:
        d = np.abs(ff[name] - fd[name])
        out[name] = {"l1": float(np.mean(d)), "linf": float(np.max(d))}
    return {"reference": "FP64 kernels", "steps": steps, "fp64_steps": int(k), "t": t,
            "status": [int(st), int(rc)], "norm": "absolute, L1 = mean over cells", "fields": out}


def sweep_inputs(nruns: int, seed: int = 2026):
    """Stability sweep: N ~ U[256, 16384], tau0 log-uniform [1e-3, 1e1], S in
    [0, 2], eq. 6 exponents spanning stable and unstable regions, mode m in 1..8
    on L = 1, frozen acoustic wave of amplitude 1e-3, t_end = 5 periods."""
    from paper_1805_03442_gb300 import inputs
    runs = inputs.sweep_runs(seed, nruns)
    shape = inputs.acoustic_shape(1.4)
    states = [inputs.waves_1d(1.4, r.N, 1.0,
                              inputs.equilibrium_primitive(0.1, r.S),
                              [inputs.Mode(m=r.m, shape=shape, scale=1e-3)]) for r in runs]
    return runs, states


class _R:
    def __init__(self, r):
        self.__dict__.update(r.__dict__)
        self.n = r.N


def sweep_measure(args, stream, reps: int = 2) -> dict:
    """Batched sweep: one persistent launch for all runs (the best of `reps`
    timed runs), next to the same runs looped through single 1D solvers on a
    stratified subset.  Returns the raw figures."""
    import torch
    from paper_1805_03442_gb300 import sv
    from paper_1805_03442_gb300.build import build
    build()
    runs, states = sweep_inputs(args.runs)
    runs = [_R(r) for r in runs]
    prec = PRECISIONS[args.precision]
    P = sv.Params(precision=prec)
    # per-run step cap: about twice the expected CFL step count plus the tau bound
    max_steps = 30 * max(r.n for r in runs) + 20000
    # launch configuration (block size per run) from the autotuner: a strided
    # sample of 256 runs to 2% of their end times, each configuration timed once
    from paper_1805_03442_gb300 import tune
    import copy
    sample = list(range(0, len(runs), max(1, len(runs) // 256)))
    s_runs = []
    for i in sample:
        r = copy.copy(runs[i])
        r.t_end = 0.02 * r.t_end
        s_runs.append(r)
    tuned = tune.tune_batch(
        lambda: sv.Batch(P, s_runs, [states[i] for i in sample], log_cap=64, stream=stream,
                         max_steps=max_steps),
        tune.batch_key(P), tune.device_name())
    b = sv.Batch(P, runs, states, log_cap=64, stream=stream, max_steps=max_steps)
    b.set_config(tuned["index"])
    times = []
    with Clocks(int(os.environ.get("LOCAL_RANK", "0"))) as clk:
        for rep in range(max(1, reps)):
            if rep:
                b.reset(states)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            b.run()
            e1.record(stream)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1) * 1e-3)
    t_batch = min(times)
    cells = cells_done = 0
    flags = {}
    completed = blown = capped = 0
    for i, r in enumerate(runs):
        _, t, k, f = b.read(i, state=False)
        cells += k * r.n
        flags[f] = flags.get(f, 0) + 1
        if f == 0 and t == r.t_end:
            completed += 1
            cells_done += k * r.n
        elif f & (sv.FLAG_NONPHYS | sv.FLAG_DT):
            blown += 1
        elif f & sv.FLAG_MAXSTEPS:
            capped += 1
    b.close()
    # looped single runs vs the batch on the same stratified subset
    order = sorted(range(len(runs)), key=lambda i: -(runs[i].n ** 2) * runs[i].t_end)
    sub = order[:: max(1, len(runs) // args.subset)][: args.subset]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in sub:
        r = runs[i]
        Pi = sv.Params(precision=prec, S=r.S, tau0=r.tau0, tau_rho=r.tau_rho, tau_T=r.tau_T,
                       Q_rho=r.Q_rho, Q_T=r.Q_T, I_rho=r.I_rho, I_T=r.I_T)
        with sv.Solver(Pi, (r.n,), (1.0,), stream=stream) as s:
            s.write_state(states[i])
            s.run_to(r.t_end, max_steps=max_steps, check=False)
    torch.cuda.synchronize()
    t_loop = time.perf_counter() - t0
    sb = sv.Batch(P, [runs[i] for i in sub], [states[i] for i in sub], log_cap=64, stream=stream,
                  max_steps=max_steps)
    sb.set_config(tuned["index"])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    sb.run()
    sb.sync()
    t_sub = time.perf_counter() - t0
    sb.close()
    return {"runs": len(runs), "t_batch": t_batch, "reps": len(times), "cells": cells,
            "cells_completed": cells_done, "completed": completed, "blown_up": blown,
            "capped": capped, "flags": {str(k): v for k, v in sorted(flags.items())},
            "tuned": tuned, "sub": len(sub), "t_loop": t_loop, "t_sub": t_sub,
            "clocks": getattr(clk, "result", None)}


def sweep_summary(m: dict) -> dict:
    """The sweep's figures for a JSON line: runs/s over all runs and over the
    runs that reach their end time, cell-updates/s, the blown-up and
    step-capped counts, and the batch against looped single runs."""
    t = m["t_batch"]
    return {"metric": "batched sweep runs/s", "runs_per_s": m["runs"] / t,
            "completed_runs_per_s": m["completed"] / t, "cell_updates_per_s": m["cells"] / t,
            "completed_cell_updates_per_s": m["cells_completed"] / t, "seconds": t,
            "runs": m["runs"], "completed": m["completed"], "blown_up": m["blown_up"],
            "blown_up_frac": m["blown_up"] / m["runs"], "capped": m["capped"],
            "launches": 1, "graph": "the persistent launch is replayed from a CUDA graph",
            "launch_config": m["tuned"]["config"],
            "vs_looped_subset": {"runs": m["sub"], "looped_single_runs_s": m["t_loop"],
                                 "batched_s": m["t_sub"], "speedup": m["t_loop"] / m["t_sub"]}}


def run_sweep(args):
    """The sweep as its own line (runs/s), with the oracle's bounded sample."""
    import torch
    stream = torch.cuda.Stream()
    m = sweep_measure(args, stream, reps=max(1, min(args.steps, 2)))
    sm = sweep_summary(m)
    line = {"metric": "batched sweep runs/s", "value": sm["runs_per_s"], "unit": "runs/s",
            "n_gpus": 1, "steps": m["reps"], "warmup": 0, "ms_per_step": 1e3 * m["t_batch"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": DTYPES[args.precision], "data": "synthetic",
            "config": {"workload": f"batched 1D stability sweep, {m['runs']} runs, N~U[256,16384], "
                                   "tau0 log-uniform [1e-3,1e1], S in [0,2], exponents in "
                                   "[-2.5,1], m in 1..8, 5 periods", "runs": m["runs"],
                       "precision": args.precision,
                       "launch_config": m["tuned"]["config"], "tuning_us": m["tuned"]["us"]},
            **{k: v for k, v in sm.items() if k not in ("metric", "runs_per_s")},
            "cell_updates": m["cells"], "run_flags": m["flags"],
            "gpu_launches": 2, "clocks": m["clocks"]}
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = oracle_special("sweep", args, args.cpu_budget)
    print(json.dumps(line), flush=True)


def run_wc(args):
    """The paper's colliding-shock test at its reference resolution: N = 10^5
    cells between solid walls, run to t = 0.038 (time to solution and
    cell-updates/s; the 3.2 MB state stays in L2 during the run)."""
    import torch
    from paper_1805_03442_gb300 import inputs, sv
    from paper_1805_03442_gb300.build import build
    build()
    N = args.n if args.n != 1 << 22 else 100000
    prec = PRECISIONS[args.precision]
    prm, U0, _ = wc_problem(N)
    P = sv.Params(precision=prec, **prm)
    stream = torch.cuda.Stream()
    s = sv.Solver(P, (N,), (1.0,), stream=stream, bc=(sv.BC_REFLECT, sv.BC_REFLECT))
    s.write_state(U0)
    s.run_to(0.004)                    # warm-up (graph capture, clocks)
    s.write_state(U0)
    torch.cuda.synchronize()
    with Clocks(int(os.environ.get("LOCAL_RANK", "0"))) as clk:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        t0 = time.perf_counter()
        rc, steps = s.run_to(0.038)
        e1.record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
    gpu_s = e0.elapsed_time(e1) * 1e-3
    s.close()
    line = {"metric": "cell-updates/s", "value": N * steps / wall, "unit": "cell-updates/s",
            "n_gpus": 1, "steps": steps, "warmup": 1, "ms_per_step": 1e3 * wall / steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": DTYPES[args.precision],
            "data": "synthetic",
            "config": {"workload": f"colliding shock waves, N={N} cells, solid walls, t_end 0.038",
                       "cells": N, "l2": "not flushed: whole run timed (3.2 MB state)"},
            "time_to_solution_s": wall, "gpu_event_s": gpu_s, "gpu_launches": steps,
            "clocks": getattr(clk, "result", None)}
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = oracle_special("wc", args, args.cpu_budget)
    print(json.dumps(line), flush=True)


def run_sector(args):
    """The paper's 2D active-sector problem (Sec. 3) as set up in the inputs
    module: a pulsating source (wavelength 0.1) at the apex of a 30-degree
    sector of active medium (S = 1, tau0 = 0.0135; frozen outside), solid wall
    at x = Lx reached by the front near t = 1, free outflow on the other
    sides; args.side cells across (default 2048, ~148 cells per wavelength),
    run to t = 1.2 (time to solution; amplitude in and outside the sector)."""
    import torch
    from paper_1805_03442_gb300 import inputs, sv
    from paper_1805_03442_gb300.build import build
    build()
    nx = args.side or 2048
    prec = PRECISIONS[args.precision]
    pb = inputs.sector_problem(nx)
    P = sv.Params(precision=prec, S=1.0, tau0=0.0135)
    U0 = inputs.sector_rest_state(P.gamma, P.Ck, P.S, pb.nx, pb.ny)
    lo, hi, dlo, dhi = pb.maps
    stream = torch.cuda.Stream()
    n = (pb.nx, pb.ny)
    s = sv.Solver(P, n, (pb.nx * pb.h, pb.ny * pb.h), stream=stream, bc=pb.bc)
    s.set_medium2d(lo, hi, dlo, dhi, pb.omega, pb.amp)
    from paper_1805_03442_gb300 import tune
    tuned = tune.tune_solver(s, tune.solver_key(P, n) + "/bnd", tune.device_name())
    s.write_state(U0)
    s.run_to(0.01)                     # warm-up (graph capture, clocks)
    s.write_state(U0)
    torch.cuda.synchronize()
    t_end = 1.2
    with Clocks(int(os.environ.get("LOCAL_RANK", "0"))) as clk:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        t0 = time.perf_counter()
        rc, steps = s.run_to(t_end, check=False)
        e1.record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
    U, t = s.read_state()
    status = s.status()
    s.close()
    # wave amplitude on the arc 0.8 < r < 1.0 from the source: inside the sector
    # (|angle| < 10 deg) and outside it (40-90 deg off the axis)
    rho = U[0].reshape(pb.ny, pb.nx) - 1.0
    X, Y = np.meshgrid((np.arange(pb.nx) + 0.5) * pb.h - pb.apex[0],
                       (np.arange(pb.ny) + 0.5) * pb.h - pb.apex[1])
    r, ang = np.hypot(X, Y), np.degrees(np.abs(np.arctan2(Y, X)))
    arc = (r > 0.8) & (r < 1.0)
    amp_in = float(np.abs(rho[arc & (ang < 10)]).max())
    amp_out = float(np.abs(rho[arc & (ang > 40) & (ang < 90)]).max())
    cells = pb.nx * pb.ny
    line = {"metric": "cell-updates/s", "value": cells * steps / wall, "unit": "cell-updates/s",
            "n_gpus": 1, "steps": steps, "warmup": 1, "ms_per_step": 1e3 * wall / steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": DTYPES[args.precision],
            "data": "synthetic",
            "config": {"workload": f"2D active sector, {pb.nx}x{pb.ny} cells, walls/outflow, "
                                   f"pulsating source lambda 0.1, S=1, tau0=0.0135, t_end {t_end}",
                       "cells": cells, "l2": "not flushed: whole run timed",
                       "launch_config": tuned["config"]},
            "time_to_solution_s": wall, "gpu_event_s": e0.elapsed_time(e1) * 1e-3,
            "status": rc, "status_flags": status, "sim_time": t,
            "amplitude_in_sector": amp_in, "amplitude_outside": amp_out,
            "gpu_launches": steps, "clocks": getattr(clk, "result", None)}
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = oracle_special("sector", args, args.cpu_budget)
    print(json.dumps(line), flush=True)


def run_driven(args):
    """The forced-source problem of the paper's Sec. 3: a wave of wavelength
    ~0.1 driven into the active medium (S = 0.5, tau0 = 0.0135) at x = 0, free
    outflow at x = 1, N = args.n cells (default 2^16), run to t = 1 (time to
    solution; the state stays in L2).  The boundary wave (eigenvector of eq. 8
    for real omega) is computed by the inputs module's caller: here from the
    closed form of the frozen acoustic wave, which the medium then reshapes."""
    import torch
    from paper_1805_03442_gb300 import inputs, sv
    from paper_1805_03442_gb300.build import build
    build()
    N = args.n if args.n != 1 << 22 else 1 << 16
    prec = PRECISIONS[args.precision]
    prm, U0, base, amp, w, kk = driven_problem(N)
    P = sv.Params(precision=prec, **prm)
    stream = torch.cuda.Stream()
    s = sv.Solver(P, (N,), (1.0,), stream=stream, bc=(sv.BC_DRIVEN, sv.BC_OUTFLOW))
    s.set_drive(w, kk, base, amp)
    s.write_state(U0)
    s.run_to(0.01)
    s.write_state(U0)
    torch.cuda.synchronize()
    with Clocks(int(os.environ.get("LOCAL_RANK", "0"))) as clk:
        t0 = time.perf_counter()
        rc, steps = s.run_to(1.0)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
    s.close()
    line = {"metric": "cell-updates/s", "value": N * steps / wall, "unit": "cell-updates/s",
            "n_gpus": 1, "steps": steps, "warmup": 1, "ms_per_step": 1e3 * wall / steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": DTYPES[args.precision],
            "data": "synthetic",
            "config": {"workload": f"forced-source wave, N={N} cells, driven x=0, outflow x=1, "
                                   "S=0.5, tau0=0.0135, t_end 1", "cells": N,
                       "l2": "not flushed: whole run timed"},
            "time_to_solution_s": wall, "gpu_launches": steps, "status": rc,
            "clocks": getattr(clk, "result", None)}
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = oracle_special("driven", args, args.cpu_budget)
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64", "fp32_p64", "fp32_pc", "fp32_ps"])
    ap.add_argument("--n", type=int, default=1 << 22, help="cells of the 1d workload")
    ap.add_argument("--workload", default="1d",
                    choices=sorted(WORKLOADS) + ["sweep", "wc", "driven", "sector"])
    ap.add_argument("--side", type=int, default=0,
                    help="cells per axis of the 2d / 3d workloads (default 8192 / 512)")
    ap.add_argument("--runs", type=int, default=4096, help="runs of the sweep workload")
    ap.add_argument("--subset", type=int, default=64, help="looped comparison subset of the sweep")
    ap.add_argument("--cpu-budget", type=float, default=10.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--b2b", action="store_true",
                    help="diagnostic: time the steps back to back (graph replay, no flush between "
                         "them) instead of one flushed step at a time")
    ap.add_argument("--no-extras", action="store_true",
                    help="default 1D line only: skip the back-to-back, FP64, compensated-pressure "
                         "and sweep figures")
    ap.add_argument("--config", type=int, default=-1,
                    help="launch configuration index of the grid workloads (default: autotuner)")
    ap.add_argument("--err-steps", type=int, default=0,
                    help="steps of the per-field error run against FP64 (0: workload default, "
                         "-1: skip)")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "sweep":
        run_sweep(args)
    elif args.workload == "wc":
        run_wc(args)
    elif args.workload == "sector":
        run_sector(args)
    elif args.workload == "driven":
        run_driven(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
