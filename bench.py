#!/usr/bin/env python
"""Benchmark of the FAM time step on B300.

Workload (default): 2D Euler (gamma = 1.4), FAM5, periodic 4096 x 4096 grid,
smooth density wave rho = 1 + 0.2 sin(2 pi (x + y)), u = v = p = 1, FP64,
CFL 0.55, Type-II OE after every step.  One "step" = one full time step:
three SSP-RK3 stage kernels + the OE kernel (with the fused CFL reduction).
Metric: cell-stage updates per second (cells x 3 stages x steps / time).

Arms:
  --impl fam        (default) the CUDA library through its C ABI.
  --impl reference  the FP64 CPU oracle on the host cores, each step one
                    oracle time step on a bounded sub-grid sample of the
                    same workload (rank 0 only).

Launch: python bench.py [--gpus N --steps K --warmup W]; for N > 1 under
torch.distributed.run, one independent replica per GPU ("replicas only":
the FAM step has no cross-GPU exchange in this build), barrier + max over
ranks of the timed region.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "2D Euler k=5 cell-stage updates/s"
UNIT = "cell-stage/s"

# Algorithmic FP64 work per cell and stage of the stage kernel: the
# DFMA / DADD / DMUL instructions of one launch per cell, counted by ncu
# (2048^2 FAM5, 16x8 tiles; profiles/stage2d_k5_f64_2048.md) when every
# multiply still ran on the FP64 unit: 1102.5 DFMA + 445.2 DADD + 437.0 DMUL
# = 3087.2 FLOP with a DFMA counted as 2, minus the 240 FLOP per cell that
# the ring cells around each 16x8 tile spend recomputing face traces (48
# ring cells x 4 components x 160 FLOP / 128 cells).  The count excludes the
# ring, so it does not depend on the tile shape.  The products the kernel
# now computes on the integer pipes (bit-identical) are still FLOP of the
# method and stay in the count.
# The FP32 kernel is the same code instantiated in float: the same count
# (its reciprocals and roots are single hardware operations in FP32, a few
# FLOP fewer per cell).
FLOP_PER_CELL_STAGE = {(5, 64): 2847.2, (5, 32): 2847.2}
# FP64-unit instructions (DFMA + DADD + DMUL) per cell of one stage launch,
# counted by ncu on the current kernel (2048^2 FAM5, 16x8 tiles: 1071.0 DFMA
# + 485.2 DADD + 200.5 DMUL): the FP64 unit's own busy fraction is these at
# one instruction per FP64 lane and cycle (half the FLOP peak).
FP64_UNIT_INST_PER_CELL = {(5, 64): 1756.7}
# DRAM bytes per launch of the stage kernel per cell (dram__bytes_read.sum +
# dram__bytes_write.sum of the current kernel, 1.1847 GB / 4.19 M cells);
# traffic grows with the cell count, so it scales to the 4096^2 launch.
DRAM_BYTES_PER_CELL = {(5, 64): 282.5}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="fam", choices=["fam", "reference"])
    ap.add_argument("--n", type=int, default=4096)
    ap.add_argument("--k", type=int, default=5)
    ap.add_argument("--precision", type=int, default=64, choices=[64, 32])
    ap.add_argument("--cfl", type=float, default=None)
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--tile", default="auto", choices=["auto", "0", "1", "2"],
                    help="2D tile shape: the autotuner's pick, or an index into fam.TILES_2D")
    ap.add_argument("--fused", default="0", choices=["0", "1"],
                    help="with a fixed --tile: 1 runs the final stage and the OE as one fused launch")
    ap.add_argument("--pp", action="store_true",
                    help="run the workload with the BP/PP safeguard (option pp_limiter) on")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched-vs-plain report")
    ap.add_argument("--no-adjoint", action="store_true", help="skip the adjoint-vs-plain report")
    ap.add_argument("--no-configs", action="store_true", help="skip the throughput of the other workloads")
    ap.add_argument("--batched-steps", type=int, default=500)
    ap.add_argument("--batched2d-steps", type=int, default=50)
    ap.add_argument("--adjoint-steps", type=int, default=200)
    ap.add_argument("--adjoint-n", type=int, default=1024)
    ap.add_argument("--oracle-rate-only", type=float, default=None, help=argparse.SUPPRESS)
    ap.add_argument("--adjoint-only", action="store_true",
                    help="run only the adjoint-vs-plain report and print it as one JSON line")
    return ap.parse_args()


def workload_config(a):
    return {"workload": f"2D Euler FAM{a.k} periodic {a.n}x{a.n}, smooth density wave "
                        f"rho=1+0.2sin(2pi(x+y)), u=v=p=1, CFL {cfl_of(a)}, Type-II OE"
                        + (", BP/PP safeguard on" if getattr(a, "pp", False) else ""),
            "grid": [a.n, a.n], "k": a.k, "equation": "euler2d", "gamma": 1.4, "oe": "type2",
            "cells": a.n * a.n, "bytes_per_state": 4 * 3 * a.n * a.n * (a.precision // 8),
            "l2": "state buffers (>= 1.6 GB) far larger than L2; no flush needed"}


def cfl_of(a):
    if a.cfl is not None:
        return a.cfl
    return 0.4 if a.k <= 4 else 0.55


# --------------------------------------------------------------------------
# clocks sampled during the timed region
# --------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.3)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.flush()
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx = float(r[2])
                for nm, v in zip(names, r[5:9]):
                    if v.strip().lower() == "active":
                        reasons.add(nm)
            except (ValueError, IndexError):
                pass
        if not sm:
            return None
        loaded = [s for s in sm if s > 0.5 * (mx or max(sm))] or sm
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# --------------------------------------------------------------------------
# oracle (CPU) baseline
# --------------------------------------------------------------------------
def oracle_rate(a, target_s: float, steps: int | None = None, sample_n: int = 256):
    """Cell-stage/s of the FP64 oracle on a sample_n x sample_n sub-grid of the
    workload (same mesh width), all host cores."""
    import oracle
    from paper_2609_26194_b300 import inputs
    cores = os.cpu_count() or 1
    os.environ.setdefault("OMP_NUM_THREADS", str(cores))
    full_n = a.n
    U = inputs.euler2d_smooth(full_n)[:, :, :sample_n, :sample_n].copy() if full_n <= 4096 else None
    dx = 1.0 / full_n
    P = oracle.Problem(d=2, nx=sample_n, ny=sample_n, x0=0.0, x1=dx * sample_n, y0=0.0, y1=dx * sample_n,
                       k=a.k, eq=oracle.EULER)
    dt = oracle.dt(P, U, cfl_of(a))
    oracle.step(P, U, dt)  # warm-up (loads the library)
    t0 = time.perf_counter()
    n = 0
    times = []
    while True:
        s0 = time.perf_counter()
        U = oracle.step(P, U, dt)
        times.append(time.perf_counter() - s0)
        n += 1
        if (steps is not None and n >= steps) or (steps is None and time.perf_counter() - t0 >= target_s):
            break
    el = time.perf_counter() - t0
    return {"value": 3.0 * sample_n * sample_n * n / el, "unit": UNIT, "cores": int(os.environ["OMP_NUM_THREADS"]),
            "kind": "oracle",
            "sample": f"{n} oracle time steps (3 stages + OE) on a {sample_n}x{sample_n} periodic sub-grid of the "
                      f"{full_n}x{full_n} FAM{a.k} workload, {el:.1f} s"}, times


def oracle_single_thread(a, seconds: float):
    """The same oracle sample on one host thread (a child process started
    with OMP_NUM_THREADS=1, since OpenMP fixes its thread count at load)."""
    env = dict(os.environ, OMP_NUM_THREADS="1")
    cmd = [sys.executable, os.path.abspath(__file__), "--oracle-rate-only", str(seconds), "--n", str(a.n),
           "--k", str(a.k)]
    try:
        out = subprocess.run(cmd, env=env, capture_output=True, text=True, timeout=300, check=True).stdout
        r = json.loads(out.strip().splitlines()[-1])
        return {"value": r["value"], "unit": r["unit"], "cores": r["cores"], "sample": r["sample"]}
    except (subprocess.SubprocessError, ValueError, KeyError, IndexError) as e:
        return {"value": None, "error": str(e)[:200]}


def run_reference(a):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    steps, warm = a.steps, a.warmup
    # each step: one oracle step on a 256 x 256 sample of the workload
    base, times = oracle_rate(a, 0, steps=warm + steps)
    t = sum(times[warm:])
    val = 3.0 * 256 * 256 * steps / t
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": a.gpus,
            "steps": steps, "warmup": warm, "ms_per_step": 1e3 * t / steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(a),
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": base["cores"], "kind": "oracle",
                             "sample": f"each step: one oracle time step on a 256x256 periodic sub-grid of the "
                                       f"{a.n}x{a.n} workload"},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------------------
# GPU arm
# --------------------------------------------------------------------------
def max_over_ranks(x: float, dist=None, device: str = "cpu") -> float:
    """Max of a per-rank scalar over all ranks (the timed region's length)."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_value(world: int, cells: int, steps: int, ms: float) -> float:
    """Whole-job cell-stage updates/s of `world` independent replicas, each
    advancing `cells` cells by `steps` steps of 3 stages, over the max time."""
    return world * 3.0 * cells * steps / (ms * 1e-3)


def batched_report(a, torch):
    """Many independent 1D Euler problems (4096 instances, N log-uniform in
    [64, 16384], k uniform in {3..6}, outflow, CFL 0.3, Riemann data), 500
    steps in one persistent launch, against the plain per-instance step loop."""
    from paper_2609_26194_b300 import fam, inputs
    insts = inputs.batched_1d(4096, seed=4)
    nx = [U.shape[-1] for _, U in insts]
    ks = [k for k, _ in insts]
    cells = sum(nx)
    b = fam.Batch(nx, ks, bc=fam.OUTFLOW)
    b.set_state([U for _, U in insts])
    tx, bps = b.tune(0.3, probe_steps=2)
    b.set_state([U for _, U in insts])
    b.run(0, 0.3)
    b.sync()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    b.run(a.batched_steps, 0.3)
    status = "ok"
    try:
        b.sync()
    except fam.FamError as e:  # a non-physical instance: timing stands, flag it
        status = str(e)
    batched_s = time.perf_counter() - t0
    info = b.info()
    _, dts, steps = b.times()
    b.close()
    # plain path: one handle per instance, fam_step per instance and step
    plain_steps = 5
    solvers = []
    for (k, U), n in zip(insts, nx):
        sv = fam.Solver(1, n, k=k, equation=fam.EULER, bc=fam.OUTFLOW)
        sv.set_state(U)
        sv.step(0.3)  # first step size + warm-up
        solvers.append(sv)
    for sv in solvers:
        sv.sync()
    t0 = time.perf_counter()
    for _ in range(plain_steps):
        for sv in solvers:
            sv.step(0.3)
    for sv in solvers:
        sv.sync()
    plain_s = time.perf_counter() - t0
    for sv in solvers:
        sv.close()
    bv = 3.0 * cells * a.batched_steps / batched_s
    pv = 3.0 * cells * plain_steps / plain_s
    # algorithmic HBM traffic of 1D Euler FP64: 8 state passes of 48 B per
    # cell per step = 128 B per cell-stage
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        pass
    hbm = peaks.get("hbm_gbs", 6400.0)
    return {"workload": "4096 x 1D Euler, N log-uniform [64,16384], k in {3,4,5,6}, outflow, CFL 0.3, "
                        "Riemann data (rho [0.7,1.5], |u| <= 0.3, p [0.7,2]), FP64", "instances": len(nx),
            "cells": cells,
            "steps": a.batched_steps, "value": bv, "unit": UNIT, "seconds": batched_s,
            "launch": {"tile_x": info["tile_x"], "grid_blocks": info["grid"], "tiles": info["tiles"],
                       "blocks_per_sm": bps, "kernel_launches": 1},
            "plain_loop": {"value": pv, "unit": UNIT, "steps": plain_steps, "seconds": plain_s,
                           "kernel_launches": 4 * len(nx) * plain_steps},
            "hbm_roofline": {"algorithmic_bytes_per_cell_stage": 128.0, "achieved_gbs": 128.0 * bv / 1e9,
                             "peak_gbs": hbm, "frac": 128.0 * bv / 1e9 / hbm},
            "speedup_vs_plain": bv / pv, "all_instances_advanced": bool(np.all(steps == a.batched_steps)),
            "status": status,
            "dt_spread": [float(np.min(dts)), float(np.max(dts))],
            "printed_ranges": batched_printed_ranges(a, nx, ks)}


def batched_printed_ranges(a, nx, ks):
    """The same instance sizes and orders with the Riemann generator at the
    shock workload's printed ranges (rho [0.1, 2], |u| <= 1, p [0.1, 10]).
    Without a positivity limiter some instances reach a non-physical state:
    each one stops after that step while the others go on.  Reported: how
    many completed, where the others stopped, and the face points whose
    Rusanov trace had no spectral radius."""
    from paper_2609_26194_b300 import fam, inputs
    states = [inputs.euler1d_riemann(n, seed=4 + i, rho=(0.1, 2.0), umax=1.0, p=(0.1, 10.0))
              for i, n in enumerate(nx)]
    b = fam.Batch(nx, ks, bc=fam.OUTFLOW)
    b.set_state(states)
    t0 = time.perf_counter()
    b.run(a.batched_steps, 0.3)
    try:
        b.sync()
        status = "ok"
    except fam.FamError as e:
        status = str(e)
    sec = time.perf_counter() - t0
    ntr, st, bad = b.health()
    _, _, steps = b.times()
    b.close()
    stopped = bad > 0
    out = {"rho": [0.1, 2.0], "umax": 1.0, "p": [0.1, 10.0], "steps": a.batched_steps, "status": status,
           "completed": int(np.sum(~stopped)), "stopped": int(np.sum(stopped)),
           "stop_step_quartiles": ([int(v) for v in np.percentile(bad[stopped], [0, 25, 50, 75, 100])]
                                   if stopped.any() else []),
           "nonphysical_traces": int(np.sum(ntr)),
           "instances_with_nonphysical_traces": int(np.sum(ntr > 0)),
           "cell_stages": int(3 * np.sum(np.asarray(nx) * steps)), "seconds": sec}
    # the same batch with the BP/PP safeguard, at the same CFL and at the
    # bound of its guarantee (1/12 for k = 5, 6)
    for cfl in (0.3, 1.0 / 12.0):
        b = fam.Batch(nx, ks, bc=fam.OUTFLOW)
        b.set_option("pp_limiter", 1)
        b.set_state(states)
        torch_sync()
        t0 = time.perf_counter()
        b.run(a.batched_steps, cfl)
        try:
            b.sync()
            status = "ok"
        except fam.FamError as e:
            status = str(e)
        sec = time.perf_counter() - t0
        ntr, _, bad = b.health()
        _, _, steps = b.times()
        rej = b.rejected_steps()
        b.close()
        # rejected attempts are not counted as work
        cs = 3.0 * float(np.sum(np.asarray(nx) * steps))
        out[f"safeguard_cfl_{cfl:.4g}"] = {"status": status, "completed": int(np.sum(bad == 0)),
                                           "stopped": int(np.sum(bad > 0)), "nonphysical_traces": int(np.sum(ntr)),
                                           "rejected_steps": int(np.sum(rej)),
                                           "instances_with_rejections": int(np.sum(rej > 0)),
                                           "value": cs / sec, "unit": UNIT, "seconds": sec}
    return out


def torch_sync():
    import torch
    torch.cuda.synchronize()


def batched2d_report(a, torch, prec: int = 64):
    """Many independent 2D Euler problems (1024 instances, nx, ny log-uniform
    in [16, 256] -- 256 to 65536 cells, the cell-count spread of the 1D batch
    -- k in {3..6}, periodic density waves) advanced 50 steps in one
    persistent launch, against the plain per-instance step loop."""
    from paper_2609_26194_b300 import fam, inputs
    insts = inputs.batched_2d(1024, seed=6, nmin=16, nmax=256)
    if prec == 32:
        insts = [(k, U.astype(np.float32)) for k, U in insts]
    nx = [U.shape[-1] for _, U in insts]
    ny = [U.shape[-2] for _, U in insts]
    ks = [k for k, _ in insts]
    cells = sum(x * y for x, y in zip(nx, ny))
    cfl, nsteps = 0.4, a.batched2d_steps
    b = fam.Batch(nx, ks, ny=ny, bc=fam.PERIODIC, precision=prec)
    b.set_state([U for _, U in insts])
    tx, bps = b.tune(cfl, probe_steps=2)
    b.set_state([U for _, U in insts])
    b.run(0, cfl)
    b.sync()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    b.run(nsteps, cfl)
    status = "ok"
    try:
        b.sync()
    except fam.FamError as e:
        status = str(e)
    batched_s = time.perf_counter() - t0
    info = b.info()
    _, dts, steps = b.times()
    b.close()
    plain_steps = 5
    solvers = []
    for (k, U), n, m in zip(insts, nx, ny):
        sv = fam.Solver(2, n, m, k=k, equation=fam.EULER, bc=fam.PERIODIC, precision=prec,
                        tile2d=fam.TILES_2D.index((info["tile_x"], info["tile_y"])))
        sv.set_state(U)
        sv.step(cfl)
        solvers.append(sv)
    for sv in solvers:
        sv.sync()
    t0 = time.perf_counter()
    for _ in range(plain_steps):
        for sv in solvers:
            sv.step(cfl)
    for sv in solvers:
        sv.sync()
    plain_s = time.perf_counter() - t0
    for sv in solvers:
        sv.close()
    bv = 3.0 * cells * nsteps / batched_s
    pv = 3.0 * cells * plain_steps / plain_s
    bpc = 256.0 if prec == 64 else 128.0  # algorithmic bytes per cell-stage
    return {"workload": "1024 x 2D Euler, nx, ny log-uniform [16,256], k in {3,4,5,6}, periodic, CFL 0.4, "
                        f"density waves (exact moments), FP{prec}", "instances": len(nx), "cells": cells,
            "steps": nsteps, "value": bv, "unit": UNIT, "seconds": batched_s,
            "launch": {"tile": [info["tile_x"], info["tile_y"]], "grid_blocks": info["grid"],
                       "tiles": info["tiles"], "blocks_per_sm": bps, "kernel_launches": 1},
            "plain_loop": {"value": pv, "unit": UNIT, "steps": plain_steps, "seconds": plain_s,
                           "kernel_launches": 4 * len(nx) * plain_steps},
            "hbm_roofline": {"algorithmic_bytes_per_cell_stage": bpc, "achieved_gbs": bpc * bv / 1e9,
                             "peak_gbs": _hbm_peak(), "frac": bpc * bv / 1e9 / _hbm_peak()},
            "speedup_vs_plain": bv / pv, "all_instances_advanced": bool(np.all(steps == nsteps)),
            "status": status}


# Warp instructions per cell of one FP32 stage launch (2D Euler FAM5, 32x8
# tiles), counted by ncu (smsp__inst_executed.sum / cells at 2048^2,
# profiles/stage2d_k5_f32_2048.md): the FP32 stage is issue-bound, so its
# roofline is the issue rate, one warp instruction per cycle per scheduler.
FP32_STAGE_WARP_INST_PER_CELL = {5: 82.16}


def _sm_clock_hz() -> float:
    """Current SM clock of GPU 0 (NVML), else the B300's maximum 2032 MHz."""
    try:
        import pynvml
        pynvml.nvmlInit()
        h = pynvml.nvmlDeviceGetHandleByIndex(int(os.environ.get("LOCAL_RANK", "0")))
        return float(pynvml.nvmlDeviceGetClockInfo(h, pynvml.NVML_CLOCK_SM)) * 1e6
    except Exception:
        return 2032e6


def _hbm_peak() -> float:
    try:
        return float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"])
    except (OSError, KeyError, ValueError):
        return 6400.0


def configs_report(a, torch):
    """Throughput of the other workloads (seeded synthetic grids shaped like
    the paper's tests), each timed on the device over a whole run."""
    from paper_2609_26194_b300 import fam, inputs

    def timed(solver, stream, run):
        # events on the solver's own stream bracket its launches
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        solver.sync()
        torch.cuda.synchronize()
        s0.record(stream)
        run()
        s1.record(stream)
        torch.cuda.synchronize()
        sec = s0.elapsed_time(s1) * 1e-3
        solver.sync()  # raises on a non-physical state: the run's number would not stand
        return sec

    out = {}
    # advection sine, N = 200, k = 3, CFL 0.2 to T = 1 (1000 steps; launch-bound by size)
    U = inputs.advection_sine(200)
    for prec in (64, 32):
        st = torch.cuda.Stream()
        s = fam.Solver(1, 200, k=3, equation=fam.ADVECTION, bc=fam.PERIODIC, gamma=1.0, precision=prec,
                       stream=st.cuda_stream)
        s.set_state(U.astype(np.float64 if prec == 64 else np.float32))
        s.run_steps(1000, 0.2)  # builds the graph of 1000 steps
        s.set_state(U.astype(np.float64 if prec == 64 else np.float32))
        sec = timed(s, st, lambda: s.run_steps(1000, 0.2))
        out[f"advection_N200_k3_f{prec}"] = {"value": 3.0 * 200 * 1000 / sec, "seconds": sec, "steps": 1000}
        s.close()
    # 1D Euler Riemann, N = 65536, k = 5, outflow, CFL 0.3, 1000 steps (one graph launch)
    U = inputs.euler1d_riemann(65536, seed=2)
    for prec in (64, 32):
        st = torch.cuda.Stream()
        s = fam.Solver(1, 65536, k=5, equation=fam.EULER, bc=fam.OUTFLOW, precision=prec, stream=st.cuda_stream)
        s.set_state(U.astype(np.float64 if prec == 64 else np.float32))
        s.run_steps(1000, 0.3)
        s.set_state(U.astype(np.float64 if prec == 64 else np.float32))
        sec = timed(s, st, lambda: s.run_steps(1000, 0.3))
        out[f"euler1d_riemann_N65536_k5_f{prec}"] = {"value": 3.0 * 65536 * 1000 / sec, "seconds": sec,
                                                     "steps": 1000}
        s.close()
    # 2D Euler 4096^2 periodic, k = 4 and 6: smooth wave and rectangles, 5 steps each (tuned tile)
    n, steps = 4096, 5
    data = {"smooth": inputs.euler2d_smooth(n),
            "rectangles": inputs.euler2d_rectangles(n, seed=3, nrect=64, **inputs.ADMISSIBLE_RECT)}
    for k in (4, 6):
        cfl = 0.4 if k == 4 else 0.55
        for prec in (64, 32):
            st = torch.cuda.Stream()
            s = fam.Solver(2, n, n, k=k, equation=fam.EULER, bc=fam.PERIODIC, precision=prec,
                           stream=st.cuda_stream)
            s.set_state(data["smooth"].astype(np.float64 if prec == 64 else np.float32))
            tile = fam.TILES_2D[s.tune(cfl, probe_steps=1)]
            for name, U in data.items():
                s.set_state(U.astype(np.float64 if prec == 64 else np.float32))
                s.run_steps(steps, cfl)
                s.set_state(U.astype(np.float64 if prec == 64 else np.float32))
                sec = timed(s, st, lambda: s.run_steps(steps, cfl))
                out[f"euler2d_{name}_4096_k{k}_f{prec}"] = {"value": 3.0 * n * n * steps / sec, "seconds": sec,
                                                            "steps": steps, "tile": list(tile)}
            s.close()
    # 2D Euler 4096^2, k = 5, FP32: the bench workload in single precision
    st = torch.cuda.Stream()
    s = fam.Solver(2, n, n, k=5, equation=fam.EULER, bc=fam.PERIODIC, precision=32, stream=st.cuda_stream)
    U32 = data["smooth"].astype(np.float32)
    s.set_state(U32)
    tile = fam.TILES_2D[s.tune(0.55, probe_steps=1)]
    s.set_state(U32)
    s.run_steps(steps, 0.55)
    s.set_state(U32)
    sec = timed(s, st, lambda: s.run_steps(steps, 0.55))
    s.set_option("profile", 1)
    s.set_state(U32)
    for _ in range(2):
        s.step(0.55)
    prof, pst = s.profile()
    stage_ms = sum(prof[:3]) / (3 * max(1, pst))
    clk = _sm_clock_hz()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    issue_peak = sms * 4 * clk  # warp instructions per second
    achieved = FP32_STAGE_WARP_INST_PER_CELL[5] * n * n / (stage_ms * 1e-3) if tile == (32, 8) else None
    out["euler2d_smooth_4096_k5_f32"] = {"value": 3.0 * n * n * steps / sec, "seconds": sec, "steps": steps,
                                         "tile": list(tile), "stage_ms": stage_ms,
                                         "issue_roofline": {"bound": "issue", "unit": "warp instructions/s",
                                                            "achieved": achieved, "peak": issue_peak,
                                                            "frac": achieved / issue_peak if achieved else None,
                                                            "instructions_per_cell": FP32_STAGE_WARP_INST_PER_CELL[5],
                                                            "source": "ncu count at 32x8 tiles; SM clock from NVML"}}
    s.close()
    # the bench workload (FP64, k = 5) with the BP/PP safeguard on: what the
    # per-stage scaling-factor kernel costs where it changes nothing
    st = torch.cuda.Stream()
    s = fam.Solver(2, n, n, k=5, equation=fam.EULER, bc=fam.PERIODIC, precision=64, pp_limiter=1,
                   stream=st.cuda_stream)
    s.set_state(data["smooth"])
    s.run_steps(steps, 0.55)
    s.set_state(data["smooth"])
    sec = timed(s, st, lambda: s.run_steps(steps, 0.55))
    out["euler2d_smooth_4096_k5_f64_safeguard"] = {"value": 3.0 * n * n * steps / sec, "seconds": sec,
                                                   "steps": steps}
    s.close()
    return {"unit": UNIT, "note": "each run: CUDA events around one graph-captured multi-step launch "
                                  "(after an untimed run of the same length)", "runs": out,
            "rectangles_printed_ranges": printed_rectangles_report(torch), "extreme_1d": extreme_1d_report(torch),
            "double_mach": double_mach_report(torch)}


def printed_rectangles_report(torch, n: int = 4096, max_steps: int = 20):
    """The rectangle workload at its printed ranges (rho, p in [0.1, 5],
    |u|, |v| <= 1), 4096^2, k = 4 and 6, FP64: stepped one step at a time
    until the state is flagged non-physical (no positivity limiter is built)
    or max_steps pass; reports where it stopped and the face points whose
    Rusanov trace had no spectral radius up to then (not a throughput)."""
    from paper_2609_26194_b300 import fam, inputs
    U = inputs.euler2d_rectangles(n, seed=3, nrect=64)
    out = {}
    for k in (4, 6):
        cfl = 0.4 if k == 4 else 0.55
        s = fam.Solver(2, n, n, k=k, equation=fam.EULER, bc=fam.PERIODIC, precision=64)
        s.set_state(U)
        status, done = "completed", max_steps
        for q in range(1, max_steps + 1):
            s.step(cfl)
            try:
                s.sync()
            except fam.FamError as e:
                status, done = f"{e} after step {q}", q
                break
        out[f"k{k}_f64"] = {"status": status, "steps": done, "nonphysical_traces": s.nonphysical_traces(),
                            "face_points_per_step": 3 * 2 * n * (n + 1) * 4}
        s.close()
    # the same data with the BP/PP safeguard (option pp_limiter) at the same
    # CFL: timed with CUDA events around one graph-captured run of max_steps
    for k, prec in ((4, 64), (6, 64), (5, 32)):
        cfl = 0.4 if k == 4 else 0.55
        Up = U.astype(np.float64 if prec == 64 else np.float32)
        st = torch.cuda.Stream()
        s = fam.Solver(2, n, n, k=k, equation=fam.EULER, bc=fam.PERIODIC, precision=prec, pp_limiter=1,
                       stream=st.cuda_stream)
        s.set_state(Up)
        s.run_steps(max_steps, cfl)  # builds the graph
        try:
            s.sync()
        except fam.FamError:
            pass
        s.set_state(Up)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        s.run_steps(max_steps, cfl)
        e1.record(st)
        torch.cuda.synchronize()
        sec = e0.elapsed_time(e1) * 1e-3
        try:
            s.sync()
            status = "completed"
        except fam.FamError as e:
            status = str(e)
        t, _, nst = s.time()
        out[f"k{k}_f{prec}_safeguard"] = {"status": status, "steps": nst, "t": t,
                                           "rejected_steps": s.rejected_steps(),
                                           "nonphysical_traces": s.nonphysical_traces(),
                                           "value": 3.0 * n * n * max_steps / sec, "unit": UNIT, "seconds": sec}
        s.close()
    return out


def extreme_1d_report(torch):
    """Example 4.7's extreme 1D tests (Sedov point blast on [-2, 2] to
    T = 1e-3, LeBlanc tube on [-10, 10] to T = 1e-4, outflow) with the BP/PP
    safeguard at the CFL of its guarantee, FP64: complete runs through
    fam_run (16-step graph chunks, synchronised between chunks), host wall
    clock.  The unlimited scheme stops in the first step on both."""
    from paper_2609_26194_b300 import fam, inputs
    out = {}
    for name, gen, n, x0, x1, T in (("sedov", inputs.sedov_1d, 801, -2.0, 2.0, 1e-3),
                                    ("leblanc", inputs.leblanc_1d, 800, -10.0, 10.0, 1e-4)):
        U = gen(n)
        for k in (3, 5, 6):
            cfl = 1 / 6 if k <= 4 else 1 / 12
            s = fam.Solver(1, n, box=(x0, x1, 0.0, 1.0), k=k, equation=fam.EULER, bc=fam.OUTFLOW, pp_limiter=1)
            s.set_state(U)
            s.run(T / 20, cfl)  # builds the chunk graph
            s.set_state(U)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            try:
                nst = s.run(T, cfl)
                s.sync()
                status = "completed"
            except fam.FamError as e:
                nst, status = s.time()[2], str(e)
            sec = time.perf_counter() - t0
            t, _, _ = s.time()
            out[f"{name}_k{k}"] = {"cells": n, "cfl": cfl, "T": T, "t": t, "steps": nst, "status": status,
                                   "rejected_steps": s.rejected_steps(),
                                   "seconds": sec, "value": 3.0 * n * nst / sec, "unit": UNIT}
            s.close()
    return out


def double_mach_report(torch, nx: int = 1440, ny: int = 480):
    """Example 4.8, double Mach reflection on [0, 3] x [0, 1] at the paper's
    1440 x 480 mesh, FAM5 with the BP/PP safeguard at CFL 1/12 (the unlimited
    scheme stops in its first step).  FP32: the complete run to T = 0.2
    through fam_run (host wall clock).  FP64: 200 steps in one graph (CUDA
    events) and one profiled step (stage launches include the safeguard's
    factor kernel and the front ghosts); the complete FP64 run is projected
    from the FP32 run's step count."""
    from paper_2609_26194_b300 import fam, inputs
    post, pre = inputs.double_mach_states()
    U = inputs.double_mach(nx, ny)
    cfl = 1.0 / 12.0

    def solver(prec, stream=None):
        s = fam.Solver(2, nx, ny, box=inputs.DMR_BOX, k=5, equation=fam.EULER, bc=fam.OUTFLOW, precision=prec,
                       pp_limiter=1, stream=stream)
        s.set_bc(0, fam.INFLOW, post)
        s.set_bc(2, fam.REFLECTIVE)
        s.set_bc_split(2, inputs.DMR_FRONT[0], post)
        s.set_bc_front(3, *inputs.DMR_FRONT, post, pre)
        return s

    out = {"mesh": [nx, ny], "k": 5, "cfl": cfl, "T": 0.2}
    s = solver(32)
    U32 = U.astype(np.float32)
    s.set_state(U32)
    s.run(0.002, cfl)  # builds the chunk graph
    s.set_state(U32)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    try:
        nst = s.run(0.2, cfl)
        s.sync()
        status = "completed"
    except fam.FamError as e:
        nst, status = s.time()[2], str(e)
    sec = time.perf_counter() - t0
    rho = s.get_state()[0, 0]
    out["f32_complete_run"] = {"status": status, "steps": nst, "seconds": sec,
                               "rejected_steps": s.rejected_steps(),
                               "value": 3.0 * nx * ny * nst / sec, "unit": UNIT,
                               "rho_max": float(rho.max()), "rho_min": float(rho.min())}
    s.close()
    st = torch.cuda.Stream()
    s = solver(64, st.cuda_stream)
    s.set_state(U)
    s.run_steps(200, cfl)
    s.sync()
    s.set_state(U)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    s.run_steps(200, cfl)
    e1.record(st)
    torch.cuda.synchronize()
    s.sync()
    ms = e0.elapsed_time(e1) / 200
    s.set_option("profile", 1)
    s.step(cfl)
    prof, _ = s.profile()
    s.close()
    tot = sum(prof)
    out["f64_200_steps"] = {"ms_per_step": ms, "value": 3.0 * nx * ny / (ms * 1e-3), "unit": UNIT,
                            "profile_ms": {"stage1_with_dt": prof[0], "stage2": prof[1], "stage3": prof[2],
                                           "oe": prof[3]},
                            "oe_share": prof[3] / tot if tot > 0 else None,
                            "projected_complete_run_seconds": ms * 1e-3 * nst}
    return out


def configs_report_safe(a, torch):
    from paper_2609_26194_b300 import fam
    try:
        return configs_report(a, torch)
    except fam.FamError as e:
        return {"status": str(e)}


def adjoint_report(a, torch):
    """Gradient of dx dy sum(rho) over a 64x64 window after 200 steps (1024^2,
    FAM5, FP64, checkpoints every 20) against the plain forward run."""
    from paper_2609_26194_b300 import fam, inputs
    n, nsteps, cfl = a.adjoint_n, a.adjoint_steps, 0.55
    ck = min(20, max(1, nsteps // 2))
    U0 = inputs.euler2d_fourier(n, seed=5)
    G = np.zeros_like(U0)
    w0 = n // 2 - 32
    G[0, 0, w0:w0 + 64, w0:w0 + 64] = 1.0 / (n * n)
    s = fam.Solver(2, n, n, k=5, equation=fam.EULER, bc=fam.PERIODIC)
    s.set_state(U0)
    s.run_steps(2, cfl)
    s.sync()
    s.set_state(U0)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    s.run_steps(nsteps, cfl)
    s.sync()
    fwd_s = time.perf_counter() - t0
    torch.cuda.reset_peak_memory_stats()
    t0 = time.perf_counter()
    grad = s.adjoint(U0, G, nsteps, cfl, ckpt_every=ck)
    adj_s = time.perf_counter() - t0
    s.close()
    state_gb = U0.nbytes / 1e9
    return {"workload": f"2D Euler FAM5 periodic {n}x{n}, {nsteps} steps, CFL 0.55, J = dx dy sum rho over "
                        f"cells [{w0},{w0 + 64})^2, checkpoints every {ck}", "forward_seconds": fwd_s,
            "forward_plus_reverse_seconds": adj_s, "ratio_vs_plain_forward": adj_s / fwd_s,
            "forward_value": 3.0 * n * n * nsteps / fwd_s, "unit": UNIT,
            "device_memory_gb_estimate": round(state_gb * (1.05 * (nsteps // ck + 4 * ck + 3) + 12), 2),
            "grad_norm_inf": float(np.max(np.abs(grad)))}


def run_fam(a):
    import torch
    from paper_2609_26194_b300 import fam, inputs

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    def max_ranks(x: float) -> float:
        return max_over_ranks(x, dist, "cuda")

    n, k, prec = a.n, a.k, a.precision
    cfl = cfl_of(a)
    U = inputs.euler2d_smooth(n)
    if prec == 32:
        U = U.astype(np.float32)
    # a dedicated stream shared by the library's launches and the CUDA events
    # (torch's default stream is the legacy NULL stream, handle 0)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    s = fam.Solver(2, n, n, k=k, equation=fam.EULER, bc=fam.PERIODIC, precision=prec,
                   stream=stream.cuda_stream, pp_limiter=1 if a.pp else 0)
    dev = torch.from_numpy(U).cuda()
    s.set_state(dev)
    # the library's tile autotuner (a few probe steps per tile shape, untimed)
    # (and whether the final stage and the OE run split or as one fused launch)
    if a.tile == "auto":
        tile = fam.TILES_2D[s.tune(cfl, probe_steps=2)]
        fused = s.fused_oe
        s.set_state(dev)
    else:
        s.set_option("tile2d", int(a.tile))
        tile = fam.TILES_2D[int(a.tile)]
        fused = int(a.fused)
        s.set_option("fused_oe", fused)
    for _ in range(a.warmup):
        s.step(cfl)
    s.sync()
    s.set_option("profile", 1)
    clocks = ClockSampler(local) if rank == 0 else None
    if clocks:
        clocks.start()
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(a.steps):
        s.step(cfl)
    e1.record(stream)
    barrier()
    ms = e0.elapsed_time(e1)
    ck = clocks.stop() if clocks else None
    s.sync()
    kern_ms, prof_steps = s.profile()
    ms = max_ranks(ms)
    cells = n * n
    value = replica_value(world, cells, a.steps, ms)

    # end to end through the C ABI with host buffers: per step, H2D of the
    # state from pinned memory, one FAM step, D2H of the state
    host_in = torch.from_numpy(U).pin_memory()
    host_out = torch.empty_like(host_in).pin_memory()
    s.set_option("profile", 0)
    barrier()
    t0 = time.perf_counter()
    for _ in range(a.e2e_steps):
        s.set_state(host_in.numpy())
        s.step(cfl)
        s.get_state(host_out.numpy())
    barrier()
    e2e_s = max_ranks(time.perf_counter() - t0)
    state_bytes = U.nbytes
    e2e = {"value": world * 3.0 * cells * a.e2e_steps / e2e_s, "unit": UNIT,
           "h2d_bytes_per_step": state_bytes, "d2h_bytes_per_step": state_bytes}

    # roofline of the dominant kernel (the stage kernel; with the fused final
    # stage + OE, stages 1 and 2 are the plain stage kernel's launches)
    peak_flops = fam.alu_peak(prec)
    if fused:
        stage_ms = sum(kern_ms[:2]) / max(1, 2 * prof_steps)
        oe_ms = None
    else:
        stage_ms = sum(kern_ms[:3]) / max(1, 3 * prof_steps)
        oe_ms = kern_ms[3] / max(1, prof_steps)
    fpc = FLOP_PER_CELL_STAGE.get((k, prec))
    traffic = DRAM_BYTES_PER_CELL.get((k, prec))
    if fpc is not None:
        achieved = fpc * cells / (stage_ms * 1e-3)
        roof = {"bound": "alu", "achieved": achieved / 1e12, "peak": peak_flops / 1e12, "unit": "TFLOP/s",
                "frac": achieved / peak_flops, "traffic": (traffic * cells if traffic else None),
                "frac_is": "algorithmic FLOP of the method (products on the integer pipes included) / "
                           f"measured FP{prec} FMA peak",
                "peak_source": f"measured FP{prec} FMA loop on this GPU (fam_alu_peak), live in this run",
                "kernel": "stage2d", "kernel_ms": stage_ms}
        ipc = FP64_UNIT_INST_PER_CELL.get((k, prec))
        if ipc is not None:  # the FP64 unit's own occupancy: its instructions against half the FLOP peak
            roof["fp64_unit"] = {"instructions_per_cell": ipc,
                                 "frac": ipc * cells / (stage_ms * 1e-3) / (peak_flops / 2.0)}
    else:
        roof = {"bound": "alu", "achieved": None, "peak": peak_flops / 1e12, "unit": "TFLOP/s", "frac": None,
                "traffic": None, "kernel": "stage2d", "kernel_ms": stage_ms}
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        pass
    hbm = peaks.get("hbm_gbs", 6400.0)
    alg_bytes = 8.0 / 3.0 * 12 * (prec // 8)  # 8 state passes per step, per cell-stage
    hbm_roof = {"algorithmic_bytes_per_cell_stage": alg_bytes,
                "achieved_gbs": alg_bytes * value / world / 1e9, "peak_gbs": hbm,
                "frac": alg_bytes * value / world / 1e9 / hbm,
                "peak_source": "MEASURED_PEAKS.json hbm_gbs" if "hbm_gbs" in peaks else "fallback 6400 GB/s"}
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": ms / a.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64" if prec == 64 else "f32",
            "data": "synthetic (seeded analytic initial data, exact moments)",
            "config": {**workload_config(a), "tile": list(tile), "final_stage_and_oe": "fused" if fused else "split",
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
            "roofline": roof, "hbm_roofline": hbm_roof,
            "kernel_ms": ({"stage1": kern_ms[0] / max(1, prof_steps), "stage2": kern_ms[1] / max(1, prof_steps),
                           "stage3_oe_fused": kern_ms[2] / max(1, prof_steps)} if fused else
                          {"stage1": kern_ms[0] / max(1, prof_steps), "stage2": kern_ms[1] / max(1, prof_steps),
                           "stage3": kern_ms[2] / max(1, prof_steps), "oe": oe_ms}),
            "e2e": e2e, "gpu_launches": ((3 if fused else 4) + (3 if a.pp else 0)) * a.steps, "clocks": ck}
    if rank == 0 and world == 1 and not a.no_batched:
        line["batched"] = batched_report(a, torch)
        line["batched2d"] = batched2d_report(a, torch)
        line["batched2d_f32"] = batched2d_report(a, torch, 32)
    if rank == 0 and world == 1 and not a.no_adjoint:
        line["adjoint"] = adjoint_report(a, torch)
    if rank == 0 and world == 1 and not a.no_configs:
        line["configs"] = configs_report_safe(a, torch)
    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        cb, _ = oracle_rate(a, 15.0)
        cb["single_thread"] = oracle_single_thread(a, 6.0)
        line["cpu_baseline"] = cb
    if rank == 0:
        print(json.dumps(line), flush=True)
    s.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


def main():
    a = parse()
    if a.oracle_rate_only is not None:  # child of oracle_single_thread (runs no GPU code)
        r, _ = oracle_rate(a, a.oracle_rate_only)
        print(json.dumps(r), flush=True)
        return 0
    if a.impl == "reference":
        return run_reference(a)
    if a.adjoint_only:
        import torch
        print(json.dumps({"adjoint": adjoint_report(a, torch)}), flush=True)
        return 0
    return run_fam(a)


if __name__ == "__main__":
    sys.exit(main())
