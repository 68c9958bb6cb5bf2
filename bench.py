"""Benchmark of the 1D WCC half-step on GB300.

Headline: the FP32-mixed path (float-float cell averages); the FP64 path is
timed in the same run under "variants", and "l1_vs_oracle" gives both paths'
L1 error against the FP64 oracle on the same workload at N = 2^12.

Workload (one GPU): 1D Euler, gamma = 1.4, N = 2^22 cells on [0, 1], P = 3,
transmissive boundaries, seeded Riemann data (rho, p ~ U(0.1, 1),
u ~ U(-0.5, 0.5) on each side of x = 0.5), limiter on, CFL nu = 0.2 (half
step).  One bench "step" is one captured CUDA graph of 32 half-steps (each a
fused half-step kernel over the whole stage: CK, flux integral, cell
average, derivatives, point value, characteristic limiter, CFL reduction).
The state (hundreds of MB) is larger than L2, so no flush is needed.

Metric: cell-updates/s = cells of the stage x half-steps / time.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl wcc|reference]
                    [--precision fp64|mixed] [--log2n 22]
    python bench.py --sweep        # precision / convergence sweep (density wave)
    python bench.py --workloads    # the paper's 1D workloads of Sec. 5

Under torchrun each rank runs an independent replica (the path has no
exchange step here); value = cell-updates of all ranks / max time.
--impl reference times the CPU oracle on the host cores (rank 0 only).
"""
from __future__ import annotations

import argparse
import math
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

METRIC = "1D Euler P=3 cell-updates/s, FP32-mixed vs FP64 at equal L1 error; % roofline"
HALFSTEPS_PER_STEP = 32
CFL = 0.2
P = 3


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--e2e-in-flight", type=int, default=E2E_IN_FLIGHT,
                    help="problems in flight in the end-to-end leg (each on its own stream and host thread)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="wcc", choices=["wcc", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["fp64", "mixed"])
    ap.add_argument("--log2n", type=int, default=22)
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--batch", type=int, default=1, help="also time the 4096-instance batch (1/0)")
    ap.add_argument("--tb", type=int, default=1, help="also time two half-steps per launch (1/0)")
    ap.add_argument("--sweep", action="store_true", help="precision / convergence sweep (density wave) instead")
    ap.add_argument("--sweep-max-log2n", type=int, default=16)
    ap.add_argument("--workloads", action="store_true",
                    help="the paper's 1D workloads (composite wave, Sod, Shu-Osher) instead")
    ap.add_argument("--two-d", action="store_true",
                    help="the 2D Euler half-step (isentropic vortex, P = 3) instead")
    ap.add_argument("--n2d", type=int, default=2048, help="cells per axis of the 2D workload")
    ap.add_argument("--rows2d", type=int, default=0,
                    help="strip height of the 2D FP32-mixed line (0: picked by wcc2d_autotune)")
    ap.add_argument("--workloads2d", action="store_true",
                    help="the paper's 2D Riemann problems at 1200^2 to t_end instead")
    ap.add_argument("--advection", action="store_true",
                    help="the linear-advection workload (N = 200, P = 2, to t = 2): time and error")
    ap.add_argument("--burgers", action="store_true",
                    help="the Burgers workload: N = 2^10..2^20, P = 1..4, FP64 and FP32-mixed")
    ap.add_argument("--burgers-log2n", default="10,14,18,20", help="log2 N of the Burgers workload, comma-separated")
    ap.add_argument("--high-order", action="store_true",
                    help="FP64 Euler half-steps at P = 3..6 (seeded Riemann data) instead")
    return ap.parse_args()


# Problems kept in flight by the end-to-end measurement: each has its own
# solver handle, CUDA stream, pinned host buffers and host thread, so the
# copies of one overlap the half-steps of the others.
E2E_IN_FLIGHT = 3
E2E_STEPS = 10  # timed steps per in-flight problem of the end-to-end leg


def e2e_bench(wcc, pr, prec, cells_per_step, steps, dev, barrier, in_flight=E2E_IN_FLIGHT):
    """Whole-job throughput through the public API with host buffers.

    Every step of every in-flight problem is wcc_set_initial from pinned host
    memory (copy engine H2D, then the layout conversion on the device), one
    graph of 32 half-steps and wcc_get_dofs back into pinned host memory (the
    call synchronises).  in_flight problems run on their own host threads
    (the binding releases the GIL in every call); "serial_value" is the same
    loop with one problem."""
    import torch
    count = pr.q0.size
    jobs = []
    for _ in range(in_flight):
        st = torch.cuda.Stream()
        s = wcc.Solver(pr.system, pr.N, P, (pr.x_l, pr.x_r), pr.bc, precision=prec,
                       graph_chunk=HALFSTEPS_PER_STEP, stream=st.cuda_stream)
        h_in = torch.from_numpy(pr.q0.reshape(-1).copy()).pin_memory()
        h_out = torch.empty(count, dtype=torch.float64).pin_memory()
        jobs.append((s, h_in, h_out))

    def run(job, k):
        s, h_in, h_out = job
        for _ in range(k):
            s.set_initial_ptr(h_in.data_ptr(), count)
            s.step(HALFSTEPS_PER_STEP, CFL)
            s.get_dofs_ptr(h_out.data_ptr(), count)

    for job in jobs:  # warm-up: graphs captured, pages touched
        run(job, 2)
    barrier()
    t0 = time.perf_counter()
    run(jobs[0], steps)
    barrier()
    serial = job_throughput(cells_per_step * steps, time.perf_counter() - t0, dev)
    threads = [threading.Thread(target=run, args=(job, steps)) for job in jobs]
    barrier()
    t0 = time.perf_counter()
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    barrier()
    value = job_throughput(cells_per_step * steps * len(jobs), time.perf_counter() - t0, dev)
    for s, _, h_out in jobs:
        assert np.all(np.isfinite(h_out.numpy()))
        s.close()
    return {"value": value, "unit": "cell-updates/s",
            "h2d_bytes_per_step": int(count * 8), "d2h_bytes_per_step": int(count * 8),
            "steps": steps * len(jobs), "in_flight": len(jobs), "serial_value": serial,
            "route": "pinned host -> copy engine -> device staging -> layout kernel (and back)"}


def workload_name(log2n):
    return f"euler1d-riemann-N2^{log2n}-P{P}-transmissive-cfl{CFL}"


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


# FP64 operations the half-step kernel issues per cell-update (Euler, P = 3,
# limiter on), counted from the executed DADD / DMUL / DFMA instructions (ncu
# smsp__sass_thread_inst_executed_op_d{add,mul,fma}_pred_on.sum over one
# launch at N = 2^21, DFMA counted as 2) divided by the cells of the launch:
# (2 x 692675342 + 306816515 + 163894018) / 2097152.5.
FP64_FLOPS_PER_CELL_UPDATE = 885.04
# DRAM bytes (read + write) of one launch at the bench size (N = 2^22), from
# one ncu capture each (dram__bytes_read.sum + dram__bytes_write.sum, one
# launch after three warm-up launches of the same kernel, graphs of 32
# half-steps; profiles/halfstep_mixed_euler_p3.md).  The writes of the last
# tiles are still in L2 when the kernel ends, so the figure is a little below
# the algorithmic one read + one write of the state.
FP64_TRAFFIC_2_22 = 402869760 + 352474368
MIXED_TRAFFIC_2_22 = 251716864 + 200629504
# FP32 flops per cell-update of the same kernel, from one capture at
# N = 2^21 of its executed paired instructions (sm__sass_thread_inst_executed_
# op_f{add2,ffma2,fmul2}, thread instructions over the 2097152.5 cells):
# 135.0 FADD2, 143.6 FFMA2 and 82.3 FMUL2 per cell-update, plus 8.5 scalar
# FMUL.  A thread carries two cells and a paired instruction does one
# operation for each, so per cell-update that is 2 x 135.0 adds, 2 x 143.6
# FMAs (2 flops each), 2 x 82.3 multiplies and 8.5 multiplies.  Lane-wise
# min/max and compares are not counted.
MIXED_FP32_FLOPS_PER_CELL = 270.0 + 2 * 287.2 + 164.6 + 8.5
# FP64 pipe peak of the GB300 (dense, nominal): 1.25 TFLOP/s.
FP64_PEAK_TFLOPS = 1.25


def bytes_per_cell_update(precision):
    # one read and one write of the state: nv * (P + 1) values per cell
    nv, K = 3, P + 1
    if precision == "fp64":
        return 2 * nv * K * 8
    return 2 * nv * (8 + 4 * (K - 1))


# ------------------------------------------------------------ clocks


class ClockSampler:
    def __init__(self):
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", str(int(os.environ.get("LOCAL_RANK", "0")))],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    mx.append(float(parts[2]))
                except ValueError:
                    continue
                for n, v in zip(names, parts[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------ CPU oracle


def host_info():
    """The host the oracle ran on: logical cores, architecture and CPU model
    (from lscpu where it exists)."""
    import platform

    model = platform.processor() or platform.machine()
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.split(":")[0].strip() == "Model name":
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    return {"nproc": os.cpu_count() or 1, "machine": platform.machine(), "cpu": model}


def cpu_oracle_rate(log2n, seconds, threads=None):
    """Oracle cell-updates/s on the host cores (all of them unless `threads`
    is given) over a bounded sample of the workload: a contiguous window of
    the N = 2^log2n grid around the jump, advanced with the CFL rule until
    ~`seconds` of wall time are spent."""
    import oracle
    from paper_2104_04347_gb300 import inputs

    threads = threads or os.cpu_count() or 1
    oracle.set_threads(threads)
    N = 1 << log2n
    pr = inputs.euler_riemann_seeded(N, P)
    win = min(1 << 16, N)
    lo = N // 2 - win // 2
    q = pr.q0[lo:lo + win + 1].copy()
    law = oracle.make_law(oracle.EULER, P, limiter=True, bc=oracle.TRANSMISSIVE)
    s = oracle.Solver(law, q, pr.dx)
    cells = 0
    t0 = time.perf_counter()
    while time.perf_counter() - t0 < seconds:
        n = s.q.shape[0]
        s.step_cfl(1, CFL)
        cells += oracle.new_count(law, s.parity ^ 1, n)
    dt = time.perf_counter() - t0
    return cells / dt, threads, (f"{len(s.dts)} half-steps of a {win}-cell window of the "
                                 f"N=2^{log2n} grid around the jump, {dt:.1f} s")


def run_reference(args, rank, world):
    """The reference arm: the CPU oracle as it stands, on the host cores.  A
    step is HALFSTEPS_PER_STEP half-steps of a bounded sample of the
    workload (the 2^16-cell window of the N = 2^log2n grid around the jump);
    W untimed steps, then K timed ones."""
    if rank != 0:
        return
    import oracle
    from paper_2104_04347_gb300 import inputs

    cores = os.cpu_count() or 1
    oracle.set_threads(cores)
    N = 1 << args.log2n
    pr = inputs.euler_riemann_seeded(N, P)
    win = min(1 << 16, N)
    lo = N // 2 - win // 2
    law = oracle.make_law(oracle.EULER, P, limiter=True, bc=oracle.TRANSMISSIVE)
    s = oracle.Solver(law, pr.q0[lo:lo + win + 1].copy(), pr.dx)

    def one_step():
        cells = 0
        for _ in range(HALFSTEPS_PER_STEP):
            n = s.q.shape[0]
            s.step_cfl(1, CFL)
            cells += oracle.new_count(law, s.parity ^ 1, n)
        return cells

    for _ in range(args.warmup):
        one_step()
    cells = 0
    t0 = time.perf_counter()
    for _ in range(args.steps):
        cells += one_step()
    dt = time.perf_counter() - t0
    rate = cells / dt
    sample = (f"{args.steps} steps of {HALFSTEPS_PER_STEP} half-steps (after {args.warmup} untimed) of a "
              f"{win}-cell window of the N=2^{args.log2n} grid around the jump, {dt:.1f} s")
    line = {
        "impl": "reference", "metric": METRIC, "value": rate, "unit": "cell-updates/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dt * 1e3 / max(1, args.steps), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded Riemann initial data, splitmix64 seed 2104043471)",
        "config": {"workload": workload_name(args.log2n), "N": N, "P": P, "cells_integer_stage": N + 1,
                   "precision": "fp64", "halfsteps_per_step": HALFSTEPS_PER_STEP, "cfl": CFL,
                   "limiter": True, "parallelism": f"host cores x{cores}", "sample_cells": win + 1},
        "cpu_baseline": {"value": rate, "unit": "cell-updates/s", "cores": cores, "kind": "oracle",
                         "sample": sample, "host": host_info()},
        "e2e": {"value": rate, "unit": "cell-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "per_full_step": {"value": rate / 2, "unit": "cell-full-steps/s"},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------ GPU


def reduce_over_ranks(x, op, device):
    """All-reduce one number over the ranks of the default process group
    (op: "max" or "sum"); the number itself without a group."""
    import torch
    import torch.distributed as td

    if not (td.is_available() and td.is_initialized()):
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    td.all_reduce(t, op=td.ReduceOp.MAX if op == "max" else td.ReduceOp.SUM)
    return float(t.item())


def job_throughput(local_units, local_seconds, device):
    """Whole-job rate of independent replicas: the units all ranks processed
    divided by the slowest rank's time."""
    return reduce_over_ranks(local_units, "sum", device) / reduce_over_ranks(local_seconds, "max", device)


def riemann_l1_exact(pr, q, t, parity=0):
    """L1 distance (mean over the cells) of the centre density point values
    q[:, 0, 0] of a stage from the exact solution of the seeded Riemann
    problem (jump at 0.5) at time t."""
    from oracle import exact
    from paper_2104_04347_gb300 import inputs

    x = inputs.centres(pr.N, pr.x_l, pr.x_r, pr.bc, parity)
    rho, _, _ = exact.riemann_sample(*inputs.riemann_states(), (x - 0.5) / t)
    return float(np.mean(np.abs(q[:, 0, 0] - rho)))


def l1_check(log2n_small=12, halfsteps=2000):
    """L1 error (centre point values, scaled per variable) of both GPU
    precisions against the FP64 oracle on the bench workload at a small N,
    each replaying its own realised dt sequence; and the density's L1
    distance from the exact Riemann solution for both and for the oracle."""
    import oracle
    from paper_2104_04347_gb300 import inputs, wcc

    oracle.set_threads(os.cpu_count() or 1)
    pr = inputs.euler_riemann_seeded(1 << log2n_small, P)
    law = oracle.make_law(oracle.EULER, P, limiter=True, bc=oracle.TRANSMISSIVE)
    out = {"workload": f"euler1d-riemann-N2^{log2n_small}-P{P}, {halfsteps} half-steps, cfl {CFL}",
           "N": 1 << log2n_small, "halfsteps": halfsteps,
           "note": "the bench grid itself (N = 2^22, 128 half-steps) is checked on sampled windows by "
                   "tests/test_gpu_mixed.py::test_mixed_full_size_sampled_windows"}
    for name, prec in (("mixed", wcc.FP32_MIXED), ("fp64", wcc.FP64)):
        with wcc.Solver(pr.system, pr.N, P, (pr.x_l, pr.x_r), pr.bc, precision=prec) as s:
            s.set_initial(pr.q0)
            s.step(halfsteps, CFL)
            q = s.get_dofs()
            dts = s.dt_history()
        ref = oracle.Solver(law, pr.q0, pr.dx)
        ref.step_dt(dts)
        scale = np.max(np.abs(ref.q[:, :, 0]), axis=0)
        out[name] = float(np.max(np.mean(np.abs(q[:, :, 0] - ref.q[:, :, 0]), axis=0) / scale))
        t = float(np.sum(dts))
        out.setdefault("density_l1_vs_exact", {})
        out["density_l1_vs_exact"][f"t_{name}"] = t
        out["density_l1_vs_exact"][name] = riemann_l1_exact(pr, q, t, halfsteps % 2)
        out["density_l1_vs_exact"][f"oracle_on_{name}_dts"] = riemann_l1_exact(pr, ref.q, t, halfsteps % 2)
    return out


def time_solver(solver, stream, steps, warmup, barrier):
    import torch
    for _ in range(warmup):
        solver.step(HALFSTEPS_PER_STEP, CFL)
    solver.synchronize()
    launches0 = solver.launch_count()
    barrier()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
    with torch.cuda.stream(stream):
        ev[0].record(stream)
        for k in range(steps):
            solver.step(HALFSTEPS_PER_STEP, CFL)
            ev[k + 1].record(stream)
    barrier()
    solver.synchronize()
    total_ms = ev[0].elapsed_time(ev[-1])
    step_ms = [ev[k].elapsed_time(ev[k + 1]) for k in range(steps)]
    return total_ms, step_ms, solver.launch_count() - launches0


def batch_bench(stream, steps, warmup, p3_rate, barrier):
    """The batched workload: 4096 independent Euler problems (N log-uniform in
    [256, 65536], P in {2, 3}, Riemann or density-wave data), FP32-mixed,
    persistent launches in graphs of 32 half-steps, grid and pass depth (one
    or two half-steps per launch) picked by the autotuner; the untuned batch
    (one half-step per launch, all resident CTAs) is timed beside it.
    Returns the batch line and the single-grid comparison."""
    import torch

    from paper_2104_04347_gb300 import inputs, wcc

    probs = inputs.batch_workload()
    cells = {2: 0, 3: 0}
    per_step = 0
    for p in probs:
        c0 = inputs.num_cells(p.N, p.bc, 0)
        c1 = inputs.num_cells(p.N, p.bc, 1)
        cells[p.P] = cells.get(p.P, 0) + 0.5 * (c0 + c1)
        per_step += (HALFSTEPS_PER_STEP // 2) * (c0 + c1)
    with wcc.Batch(probs, graph_chunk=HALFSTEPS_PER_STEP, stream=stream.cuda_stream) as b:
        b.set_initial()
        ctas = b.autotune(CFL)
        _, depth = b.tuning()
        total_ms, step_ms, launches = time_solver(b, stream, steps, warmup, barrier)
        pairs, fallbacks = b.tb_stats()
    value = per_step * steps / (total_ms * 1e-3)
    with wcc.Batch(probs, graph_chunk=HALFSTEPS_PER_STEP, stream=stream.cuda_stream) as b1:
        b1.set_initial()
        t1, _, _ = time_solver(b1, stream, steps, warmup, barrier)
    value_one = per_step * steps / (t1 * 1e-3)
    # single-grid FP32-mixed rate at P = 2 on the same grid shape as the headline
    pr = inputs.euler_riemann_seeded(1 << 22, 2)
    with wcc.Solver(pr.system, pr.N, 2, (pr.x_l, pr.x_r), pr.bc, precision=wcc.FP32_MIXED,
                    graph_chunk=HALFSTEPS_PER_STEP, stream=stream.cuda_stream) as s2:
        s2.set_initial(pr.q0)
        t2, _, _ = time_solver(s2, stream, max(2, min(steps, 5)), warmup, barrier)
    p2_rate = (HALFSTEPS_PER_STEP // 2) * ((pr.N + 1) + pr.N) * max(2, min(steps, 5)) / (t2 * 1e-3)
    ctot = cells[2] + cells[3]
    single = 1.0 / ((cells[2] / ctot) / p2_rate + (cells[3] / ctot) / p3_rate)
    return {"workload": "euler1d-batch-4096-N256..65536-P2/3-riemann/density-wave", "value": value,
            "unit": "cell-updates/s", "ms_per_step": total_ms / steps, "steps": steps,
            "cells_per_halfstep": per_step / HALFSTEPS_PER_STEP, "persistent_ctas": ctas,
            "halfsteps_per_launch": depth, "pairs": pairs, "pair_fallbacks": fallbacks,
            "untuned_default_grid": value_one,
            "gpu_launches": launches, "single_grid_same_mix": single, "single_grid_p2": p2_rate,
            "single_grid_p3": p3_rate, "single_over_batch": single / value}


def tb_bench(pr, stream, steps, warmup, barrier, dev, cells_per_step, cells_per_launch, pk):
    """The headline workload with two half-steps per launch (tb_depth = 2):
    one read and one write of the state per pair, so 60 B per cell-update in
    FP32-mixed; same steps of 32 half-steps (16 launches), CUDA events."""
    from paper_2104_04347_gb300 import wcc

    with wcc.Solver(pr.system, pr.N, P, (pr.x_l, pr.x_r), pr.bc, precision=wcc.FP32_MIXED,
                    graph_chunk=HALFSTEPS_PER_STEP, stream=stream.cuda_stream, tb_depth=2) as s:
        s.set_initial(pr.q0)
        total_ms, step_ms, launches = time_solver(s, stream, steps, warmup, barrier)
        pairs, fallbacks, nu2 = s.tb_stats()
    value = job_throughput(cells_per_step * steps, total_ms * 1e-3, dev)
    kernel_ms = statistics.median(step_ms) / HALFSTEPS_PER_STEP
    bpc = bytes_per_cell_update("mixed") / 2
    gbs = bpc * cells_per_launch / (kernel_ms * 1e-3) / 1e9
    return {"value": value, "unit": "cell-updates/s", "ms_per_step": total_ms / steps, "steps": steps,
            "ms_per_halfstep": kernel_ms, "gpu_launches": launches, "bytes_per_cell_update": bpc,
            "hbm_gbs": gbs, "hbm_frac": gbs / pk["hbm_gbs"], "pairs": pairs, "fallbacks": fallbacks,
            "nu2_max": nu2, "cfl": CFL,
            "dt_rule": "one dt per pair from the first stage's bound; second half-step's CFL number checked"}


def tuned_bench(pr, stream, steps, warmup, barrier, dev, cells_per_step):
    """The headline workload with the launch configuration wcc_autotune picks
    on it (cells per CTA, one or two half-steps per launch)."""
    from paper_2104_04347_gb300 import wcc

    with wcc.Solver(pr.system, pr.N, P, (pr.x_l, pr.x_r), pr.bc, precision=wcc.FP32_MIXED,
                    graph_chunk=HALFSTEPS_PER_STEP, stream=stream.cuda_stream) as s:
        s.set_initial(pr.q0)
        t0 = time.perf_counter()
        cpb, tb = s.autotune(CFL)
        tune_s = time.perf_counter() - t0
        total_ms, step_ms, launches = time_solver(s, stream, steps, warmup, barrier)
    value = job_throughput(cells_per_step * steps, total_ms * 1e-3, dev)
    return {"value": value, "unit": "cell-updates/s", "cells_per_block": cpb, "tb_depth": tb,
            "ms_per_halfstep": statistics.median(step_ms) / HALFSTEPS_PER_STEP, "steps": steps,
            "gpu_launches": launches, "tuning_seconds": tune_s,
            "candidates": "cells_per_block 255 / 510 with one half-step per launch, two half-steps per launch"}


def run_wcc(args, rank, world):
    import torch

    from paper_2104_04347_gb300 import inputs, wcc

    dist = world > 1
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if dist:
        import torch.distributed as td
        td.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)

    def barrier():
        if dist:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    def max_over_ranks(x):
        return reduce_over_ranks(x, "max", dev)

    N = 1 << args.log2n
    pr = inputs.euler_riemann_seeded(N, P)
    cells_per_step = (HALFSTEPS_PER_STEP // 2) * ((N + 1) + N)
    cells_per_launch = 0.5 * ((N + 1) + N)
    pk, pk_kind = peaks()
    precisions = [args.precision] + [p for p in ("mixed", "fp64") if p != args.precision]

    clocks = ClockSampler()
    clocks.start()
    results = {}
    for name in precisions:
        prec = wcc.FP64 if name == "fp64" else wcc.FP32_MIXED
        solver = wcc.Solver(pr.system, N, P, (pr.x_l, pr.x_r), pr.bc, precision=prec,
                            graph_chunk=HALFSTEPS_PER_STEP, stream=stream.cuda_stream)
        solver.set_initial(pr.q0)
        steps = args.steps if name == args.precision else max(2, min(args.steps, 5))
        total_ms, step_ms, launches = time_solver(solver, stream, steps, args.warmup, barrier)
        value = job_throughput(cells_per_step * steps, total_ms * 1e-3, dev)
        total_ms = max_over_ranks(total_ms)
        kernel_ms = statistics.median(step_ms) / HALFSTEPS_PER_STEP
        bpc = bytes_per_cell_update(name)
        res = {"value": value, "ms_per_step": total_ms / steps,
               "steps": steps, "kernel_ms": kernel_ms, "gpu_launches": launches}
        gbs = bpc * cells_per_launch / (kernel_ms * 1e-3) / 1e9
        hbm = {"bound": "hbm", "achieved": gbs, "peak": pk["hbm_gbs"], "unit": "GB/s",
               "frac": gbs / pk["hbm_gbs"], "traffic": None,
               "peak_source": ("measured hbm_gbs (MEASURED_PEAKS.json)" if pk_kind == "measured"
                               else "fallback 6.8 TB/s"),
               "bytes_per_cell_update": bpc, "kernel_ms": kernel_ms}
        if name == "fp64":
            tf = FP64_FLOPS_PER_CELL_UPDATE * cells_per_launch / (kernel_ms * 1e-3) / 1e12
            res["roofline"] = {"bound": "alu", "achieved": tf, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                               "frac": tf / FP64_PEAK_TFLOPS,
                               "traffic": FP64_TRAFFIC_2_22 if args.log2n == 22 else None,
                               "peak_source": "nominal GB300 FP64 1.25 TFLOP/s (recipe)",
                               "flops_per_cell_update": FP64_FLOPS_PER_CELL_UPDATE, "kernel_ms": kernel_ms,
                               "hbm_frac": hbm["frac"]}
        else:
            if args.log2n == 22:
                hbm["traffic"] = MIXED_TRAFFIC_2_22
            res["roofline"] = hbm
        results[name] = res
        solver.close()
    if args.tb:
        results["mixed_tb2"] = tb_bench(pr, stream, max(2, min(args.steps, 10)), args.warmup, barrier, dev,
                                        cells_per_step, cells_per_launch, pk)
        results["mixed_tuned"] = tuned_bench(pr, stream, max(2, min(args.steps, 10)), args.warmup, barrier, dev,
                                             cells_per_step)
    if args.batch:
        results["batch"] = batch_bench(stream, max(2, min(args.steps, 5)), args.warmup,
                                       results["mixed"]["value"] / world, barrier)
    clk = clocks.stop()

    # ---- end to end through the public API with host buffers (headline precision)
    # 10 steps per in-flight problem whatever --steps is, so that filling and
    # draining the pipeline of problems is a small part of the timed region
    e2e = e2e_bench(wcc, pr, wcc.FP64 if args.precision == "fp64" else wcc.FP32_MIXED, cells_per_step,
                    E2E_STEPS, dev, barrier, args.e2e_in_flight)

    fp64_peak_meas = wcc.measure_fp_peak(wcc.FP64)
    fp32_peak_meas = wcc.measure_fp_peak(wcc.FP32_MIXED)
    head = results[args.precision]
    roof = dict(head["roofline"])
    roof["fp64_fma_peak_measured_tflops"] = fp64_peak_meas
    roof["fp32_fma_peak_measured_tflops"] = fp32_peak_meas
    if args.precision == "mixed" and fp32_peak_meas > 0:
        # the other side of the roofline: FP32 flops over the measured FP32 peak
        fl = MIXED_FP32_FLOPS_PER_CELL * cells_per_launch / (roof["kernel_ms"] * 1e-3) / 1e12
        roof["fp32_flops_per_cell_update"] = MIXED_FP32_FLOPS_PER_CELL
        roof["fp32_tflops"] = fl
        roof["fp32_frac"] = fl / fp32_peak_meas
    line = {
        "metric": METRIC, "value": head["value"], "unit": "cell-updates/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": head["ms_per_step"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if args.precision == "fp64" else "f32",
        "data": "synthetic (seeded Riemann initial data, splitmix64 seed 2104043471)",
        "config": {"workload": workload_name(args.log2n), "N": N, "P": P, "cells_integer_stage": N + 1,
                   "precision": args.precision, "halfsteps_per_step": HALFSTEPS_PER_STEP, "cfl": CFL,
                   "limiter": True, "l2": "state > L2 (252 / 403 MB per stage), no flush needed",
                   "parallelism": f"replicas x{world}"},
        "roofline": roof,
        "per_full_step": {"value": head["value"] / 2, "unit": "cell-full-steps/s"},
        "e2e": e2e,
        "gpu_launches": head["gpu_launches"],
        "clocks": clk,
        "variants": {k: v for k, v in results.items() if k != args.precision},
    }
    if rank == 0 and world == 1:
        line["l1_vs_oracle"] = l1_check()
        rate, cores, sample = cpu_oracle_rate(args.log2n, args.cpu_seconds)
        rate1, _, sample1 = cpu_oracle_rate(args.log2n, args.cpu_seconds / 4, threads=1)
        line["cpu_baseline"] = {"value": rate, "unit": "cell-updates/s", "cores": cores, "kind": "oracle",
                                "sample": sample, "host": host_info(),
                                "single_thread": {"value": rate1, "unit": "cell-updates/s", "sample": sample1}}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        torch.distributed.destroy_process_group()


def precision_sweep(max_log2n=16):
    """Smooth Euler density wave rho = 1 + 0.2 sin 2 pi x, u = 1, p = 1,
    periodic [0, 1], to t = 1, P = 1..4 at N = 2^8 .. 2^max_log2n and
    P = 5, 6 at N = 2^4 .. 2^11: every
    precision on the same half-step sizes; L1 of the density point values
    against the exact solution and against the FP64 path (and the oracle for
    N <= 2^10), and the measured order.  Prints one JSON line per case and a
    markdown table."""
    import math

    import oracle
    from paper_2104_04347_gb300 import inputs, wcc

    oracle.set_threads(os.cpu_count() or 1)
    nu = {1: 0.4, 2: 0.3, 3: 0.25, 4: 0.2, 5: 0.16, 6: 0.14}
    amax = 1.0 + math.sqrt(1.4 / 0.8)
    names = {wcc.FP64: "fp64", wcc.FP32_MIXED: "fp32-mixed", wcc.FP32: "fp32"}
    rows = []
    for P in (1, 2, 3, 4, 5, 6):
        prev = {}
        # P = 5, 6 reach the FP64 rounding floor by 2^10 cells; finer meshes
        # only take longer
        top = max_log2n if P <= 4 else min(max_log2n, 11)
        for log2n in range(8 if P <= 4 else 4, top + 1):
            N = 1 << log2n
            pr = inputs.euler_density_wave(N, P)
            dts = oracle.constant_speed_dts(1.0, nu[P] * pr.dx / amax)
            x = inputs.centres(N, 0.0, 1.0, inputs.PERIODIC)
            exact = 1.0 + 0.2 * np.sin(2 * math.pi * (x - 1.0))
            res = {}
            for prec in (wcc.FP64, wcc.FP32_MIXED, wcc.FP32):
                with wcc.Solver(pr.system, N, P, (0.0, 1.0), pr.bc, precision=prec, limiter=True) as s:
                    s.set_initial(pr.q0)
                    t0 = time.perf_counter()
                    s.step_dt(dts)
                    q = s.get_dofs()
                    res[prec] = (q, time.perf_counter() - t0)
            q64 = res[wcc.FP64][0]
            ref = None
            if log2n <= 10:
                sol = oracle.Solver(oracle.make_law(oracle.EULER, P, limiter=True), pr.q0, pr.dx)
                sol.step_dt(dts)
                ref = sol.q
            for prec, (q, secs) in res.items():
                e = float(np.mean(np.abs(q[:, 0, 0] - exact)))
                row = {"P": P, "N": N, "precision": names[prec], "halfsteps": len(dts),
                       "l1_exact": e, "l1_vs_fp64": float(np.mean(np.abs(q[:, 0, 0] - q64[:, 0, 0]))),
                       "l1_vs_oracle": None if ref is None else float(np.mean(np.abs(q[:, 0, 0] - ref[:, 0, 0]))),
                       "order": (math.log2(prev[prec] / e) if prec in prev and e > 0 else None), "seconds": secs}
                prev[prec] = e
                rows.append(row)
                print(json.dumps(row), flush=True)
    print("| P | N | precision | L1 vs exact | order | L1 vs FP64 | L1 vs oracle |")
    print("|---|---|---|---|---|---|---|")
    for r in rows:
        o = "" if r["order"] is None else f"{r['order']:.2f}"
        lo = "" if r["l1_vs_oracle"] is None else f"{r['l1_vs_oracle']:.2e}"
        print(f"| {r['P']} | {r['N']} | {r['precision']} | {r['l1_exact']:.3e} | {o} | {r['l1_vs_fp64']:.2e} | {lo} |")


def paper_workloads():
    """The 1D workloads of Sec. 5 at the paper's sizes, P = 1..3 with the
    Sec. 5 CFL numbers, run to t_end through wcc_step_until in every
    precision:
      * composite wave, periodic [-1, 1], 400 cells, t = 12 (six periods; the
        exact solution is the initial data);
      * Sod, [0, 2], 200 cells, t = 0.4 (exact Riemann solution);
      * modified Shu-Osher, [-5, 5], 2000 cells, t = 5 (no exact solution:
        the standard deviation of the density behind the shock, x in
        [0.5, 2.3], shows how much of the entropy wave survives).
    Per case: half-steps, time to solution (second pass on the same handle,
    host wall clock around the call, which returns synchronised), L1 of the
    density cell averages against the exact solution, and L1 against the
    oracle replaying the same half-step sizes (FP64 and FP32-mixed).  One JSON
    line per case and a markdown table."""
    import math

    import oracle
    from oracle import exact
    from paper_2104_04347_gb300 import inputs, wcc

    oracle.set_threads(os.cpu_count() or 1)
    nu = {1: 0.4, 2: 0.3, 3: 0.25}
    names = {wcc.FP64: "fp64", wcc.FP32_MIXED: "fp32-mixed", wcc.FP32: "fp32"}

    def avg(q):
        k = np.arange(q.shape[-1])
        w = np.where(k % 2 == 0, 1.0 / (np.array([math.factorial(i + 1) for i in k]) * 2.0 ** k), 0.0)
        return q @ w

    def sod_exact(pr, t):
        x = inputs.centres(pr.N, pr.x_l, pr.x_r, pr.bc)
        pts = x[:, None] + pr.dx * ((np.arange(64) + 0.5) / 64 - 0.5)[None, :]
        rho, _, _ = exact.riemann_sample((1.0, 0.0, 1.0), (0.125, 0.0, 0.1), (pts - 1.0) / t)
        return rho.mean(axis=1)

    cases = (("composite-wave", lambda P: inputs.advection_composite(400, P), 12.0),
             ("sod", lambda P: inputs.sod(200, P), 0.4),
             ("shu-osher", lambda P: inputs.shu_osher(2000, P), 5.0))
    rows = []
    for name, make, t_end in cases:
        for P in (1, 2, 3):
            pr = make(P)
            length = pr.x_r - pr.x_l
            ref_exact = avg(pr.q0)[:, 0] if name == "composite-wave" else (
                sod_exact(pr, t_end) if name == "sod" else None)
            x = inputs.centres(pr.N, pr.x_l, pr.x_r, pr.bc)
            band = (x > 0.5) & (x < 2.3)
            for prec in (wcc.FP64, wcc.FP32_MIXED, wcc.FP32):
                with wcc.Solver(pr.system, pr.N, P, (pr.x_l, pr.x_r), pr.bc, precision=prec) as s:
                    s.set_initial(pr.q0)
                    s.step_until(t_end, nu[P])  # first pass: graph capture, history growth
                    s.set_initial(pr.q0)
                    t0 = time.perf_counter()
                    n = s.step_until(t_end, nu[P])
                    secs = time.perf_counter() - t0
                    q = s.get_dofs()
                    dts = s.dt_history()
                rho = avg(q)[:, 0]
                row = {"workload": name, "P": P, "N": pr.N, "precision": names[prec], "t_end": t_end,
                       "halfsteps": n, "seconds": secs, "us_per_halfstep": 1e6 * secs / n,
                       "l1_exact": None if ref_exact is None else float(length * np.mean(np.abs(rho - ref_exact))),
                       "wave_std": float(np.std(rho[band])) if name == "shu-osher" else None,
                       "l1_vs_oracle": None}
                if prec != wcc.FP32:
                    sol = oracle.Solver(oracle.make_law(pr.system, P, limiter=True, bc=pr.bc), pr.q0, pr.dx)
                    t1 = time.perf_counter()
                    sol.step_dt(dts)
                    row["oracle_seconds"] = time.perf_counter() - t1
                    row["oracle_cores"] = oracle.get_threads()
                    row["l1_vs_oracle"] = float(length * np.mean(np.abs(rho - avg(sol.q)[:, 0])))
                rows.append(row)
                print(json.dumps(row), flush=True)
    print("| workload | P | precision | half-steps | time to t_end | µs / half-step | L1 vs exact | "
          "entropy-wave std | L1 vs oracle | oracle time (same half-steps) |")
    print("|---|---|---|---|---|---|---|---|---|---|")
    for r in rows:
        le = "" if r["l1_exact"] is None else f"{r['l1_exact']:.3e}"
        ws = "" if r["wave_std"] is None else f"{r['wave_std']:.4f}"
        lo = "" if r["l1_vs_oracle"] is None else f"{r['l1_vs_oracle']:.1e}"
        ot = "" if "oracle_seconds" not in r else f"{r['oracle_seconds']:.2f} s ({r['oracle_cores']} cores)"
        print(f"| {r['workload']} | {r['P']} | {r['precision']} | {r['halfsteps']} | {1e3 * r['seconds']:.1f} ms | "
              f"{r['us_per_halfstep']:.2f} | {le} | {ws} | {lo} | {ot} |")


# 2D path (Sec. 3, Sec. 4): the isentropic vortex of Sec. 5.3 on n x n cells,
# P = 3 (WCCS-4), limiter on, CFL 0.25 (Sec. 5), one bench step = 8 half-steps.
HALFSTEPS_2D = 8
CFL_2D = 0.25
# Algorithmic DRAM bytes per cell-update: the 4 x 10 DOFs read and written
# once (FP32: 4 B each, FP64: 8 B; FP32-mixed: 4 more floats, the low parts
# of the cell averages).
BYTES_2D_PER_CELL = {"fp32_mixed": 2 * 44 * 4, "fp32": 2 * 40 * 4, "fp64": 2 * 40 * 8}
# Arithmetic per cell-update of halfstep2d<EULER, 3>, from ncu's executed
# FADD/FMUL/FFMA (FP32 kernel, 128-thread strips) and DADD/DMUL/DFMA (FP64
# kernel, 64-thread strips) thread instructions of one launch at n = 1024
# divided by the 1024^2 cells (FMA = 2 flops; min/max, compares and
# conversions not counted; a paired FADD2 counts 2, a paired FFMA2 4).
# FP32-mixed: its current kernel (96-thread strips, 19 rows per strip).
# FP32: none, not recounted since its projections went to paired FP32.
FLOPS_2D_PER_CELL = {"fp32_mixed": (1403120218 + 2 * 1618423496 + 264650802 + 2 * 12582912 + 4 * 155189248) / 1048576.0,
                     "fp32": None,
                     "fp64": (412078081 + 2 * 2396458776 + 341564899) / 1048576.0}
# DRAM bytes (read + write) of one launch per cell, same captures; scaled by
# cells to the bench size.  The writes undercount the stored DOFs: part of
# the output is still in L2 when the kernel ends.  FP32-mixed: one launch at
# the bench size itself, 2048^2, per strip height (a strip re-reads one parent
# row, so the bytes depend slightly on it); heights not captured report none.
TRAFFIC_2D_MIXED_BY_ROWS = {19: (780613888 + 691828736) / 4194304.0}
TRAFFIC_2D_PER_CELL = {"fp32_mixed": None, "fp32": None,
                       "fp64": (358728448 + 294830336) / 1048576.0}


def two_d_bench(args):
    """FP32 and FP64 2D Euler half-steps on the isentropic vortex: cell-updates/s
    with inputs resident in HBM, the kernel's share of the HBM and arithmetic
    rooflines, and the CPU oracle on a small sample of the same workload."""
    import torch

    import oracle
    from paper_2104_04347_gb300 import inputs, wcc

    n, P = args.n2d, 3
    pr = inputs.isentropic_vortex(n, P)
    stream = torch.cuda.Stream()
    pk, pk_src = peaks()
    fp32_peak = wcc.measure_fp_peak(wcc.FP32_MIXED)  # the FP32 FMA probe
    clocks = ClockSampler()
    clocks.start()
    results = {}
    # the headline FP32-mixed line with the strip height picked by
    # wcc2d_autotune; the default height (16) and the other precisions beside it
    for prec, name, steps, tune in ((wcc.FP32_MIXED, "fp32_mixed", args.steps, True),
                                    (wcc.FP32_MIXED, "fp32_mixed_rows16", args.steps, False),
                                    (wcc.FP32, "fp32", args.steps, False),
                                    (wcc.FP64, "fp64", max(2, min(args.steps, 3)), False)):
        rows = args.rows2d if tune and args.rows2d else 16
        with wcc.Solver2D(pr.system, n, n, P, (pr.x_l, pr.x_r, pr.y_l, pr.y_r), pr.bc, precision=prec,
                          rows_per_cta=rows, stream=stream.cuda_stream) as s:
            s.set_initial(pr.q0)
            if tune and not args.rows2d:
                rows = s.autotune(CFL_2D)
            for _ in range(args.warmup):
                s.step(HALFSTEPS_2D, CFL_2D)
            s.synchronize()
            l0 = s.launch_count()
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
            with torch.cuda.stream(stream):
                ev[0].record(stream)
                for k in range(steps):
                    s.step(HALFSTEPS_2D, CFL_2D)
                    ev[k + 1].record(stream)
            s.synchronize()
            total_ms = ev[0].elapsed_time(ev[-1])
            launches = s.launch_count() - l0
        per_launch_s = total_ms / 1e3 / (steps * HALFSTEPS_2D)
        cells = n * n
        r = {"value": cells / per_launch_s, "ms_per_halfstep": per_launch_s * 1e3, "steps": steps,
             "gpu_launches": launches, "rows_per_cta": rows}
        kind = name if name in BYTES_2D_PER_CELL else "fp32_mixed"
        gbs = BYTES_2D_PER_CELL[kind] * cells / per_launch_s / 1e9
        r["hbm"] = {"achieved_gbs": gbs, "peak_gbs": pk["hbm_gbs"], "frac": gbs / pk["hbm_gbs"],
                    "bytes_per_cell": BYTES_2D_PER_CELL[kind],
                    "traffic": None}
        per_cell = TRAFFIC_2D_MIXED_BY_ROWS.get(rows) if kind == "fp32_mixed" else TRAFFIC_2D_PER_CELL[kind]
        if per_cell:
            r["hbm"]["traffic"] = per_cell * cells
        if FLOPS_2D_PER_CELL[kind]:
            tf = FLOPS_2D_PER_CELL[kind] * cells / per_launch_s / 1e12
            peak = FP64_PEAK_TFLOPS if name == "fp64" else fp32_peak
            r["arith"] = {"achieved_tflops": tf, "peak_tflops": peak, "frac": tf / peak,
                          "flops_per_cell": FLOPS_2D_PER_CELL[kind]}
        results[name] = r
    clk = clocks.stop()
    # CPU oracle on a bounded sample: the same vortex at 64 x 64, FP64, a few half-steps
    m = 64
    prs = inputs.isentropic_vortex(m, P)
    sol = oracle.Solver2D(oracle.make_law2d(oracle.EULER, P), prs.q0, prs.dx, prs.dy)
    t0 = time.perf_counter()
    k = 0
    while time.perf_counter() - t0 < args.cpu_seconds / 4 or k < 2:
        sol.step_cfl(1, CFL_2D)
        k += 1
    cpu_rate = m * m * k / (time.perf_counter() - t0)
    # the headline is FP32-mixed, as in 1D: float arithmetic with float-float
    # cell averages (plain FP32 reaches its rounding floor on fine meshes)
    head = results["fp32_mixed"]
    bound = "hbm" if head["hbm"]["frac"] >= head.get("arith", {"frac": 0})["frac"] else "fp32"
    line = {
        "metric": "2D Euler P=3 cell-updates/s (isentropic vortex, WCCS-4)", "value": head["value"],
        "unit": "cell-updates/s", "n_gpus": 1, "steps": head["steps"], "warmup": args.warmup,
        "ms_per_step": head["ms_per_halfstep"] * HALFSTEPS_2D, "higher_is_better": True, "dtype": "f32 (float-float averages)",
        "data": "synthetic", "config": {"workload": f"2D Euler isentropic vortex {n}x{n}, P=3, limiter on, CFL 0.25, "
                                                    f"{HALFSTEPS_2D} half-steps per step; state larger than L2"},
        "roofline": {"bound": bound, "achieved": head["hbm"]["achieved_gbs"], "peak": pk["hbm_gbs"],
                     "unit": "GB/s", "frac": head["hbm"]["frac"], "traffic": head["hbm"]["traffic"],
                     "fp32_tflops": head.get("arith", {}).get("achieved_tflops"),
                     "fp32_frac": head.get("arith", {}).get("frac"), "peak_source": pk_src,
                     "fp32_peak_tflops": fp32_peak},
        "variants": results,
        "cpu_baseline": {"value": cpu_rate, "unit": "cell-updates/s", "cores": oracle.get_threads(), "kind": "oracle",
                         "sample": f"FP64 oracle, same vortex at {m}x{m}, {k} half-steps"},
        "clocks": clk,
        "gpu_launches": head["gpu_launches"],
    }
    print(json.dumps(line), flush=True)


# Degrees above the paper's tables: CFL 0.8 of the von Neumann limit of the
# linear scheme (0.2116 at P = 5, 0.1851 at P = 6; Sec. 2.3), the bench's 0.2
# below that.
CFL_HIGH = {3: 0.2, 4: 0.2, 5: 0.16, 6: 0.14}
# FP64 flops per cell-update of halfstep_fp64<EULER, P> (ncu DADD + DMUL +
# 2 DFMA thread instructions of one launch over the launch's cells); P = 3 is
# FP64_FLOPS_PER_CELL_UPDATE, P = 4..6 from one launch each at N = 2^20
# (e.g. P = 6: (132561538 + 271580931 + 2 x 1108567950) / 1048576.5).
FP64_FLOPS_HIGH = {3: None,
                   4: (101969794 + 187162371 + 2 * 522598030) / 1048576.5,
                   5: (120968962 + 232542339 + 2 * 766449806) / 1048576.5,
                   6: (132561538 + 271580931 + 2 * 1108567950) / 1048576.5}


def high_order_bench(args):
    """FP64 Euler half-steps at P = 3..6 on the bench's seeded Riemann data:
    cell-updates/s (CUDA events, graphs of 32 half-steps, inputs resident)
    and the share of the FP64 peak where the flop count is known."""
    import torch

    from paper_2104_04347_gb300 import inputs, wcc

    FP64_FLOPS_HIGH[3] = FP64_FLOPS_PER_CELL_UPDATE
    stream = torch.cuda.Stream()
    clocks = ClockSampler()
    clocks.start()
    rows = []
    for P in (3, 4, 5, 6):
        pr = inputs.euler_riemann_seeded(1 << args.log2n, P)
        with wcc.Solver(pr.system, pr.N, P, (pr.x_l, pr.x_r), pr.bc, precision=wcc.FP64,
                        stream=stream.cuda_stream) as s:
            s.set_initial(pr.q0)
            for _ in range(args.warmup):
                s.step(HALFSTEPS_PER_STEP, CFL_HIGH[P])
            s.synchronize()
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
            with torch.cuda.stream(stream):
                ev[0].record(stream)
                for k in range(args.steps):
                    s.step(HALFSTEPS_PER_STEP, CFL_HIGH[P])
                    ev[k + 1].record(stream)
            s.synchronize()
            ms = ev[0].elapsed_time(ev[-1]) / (args.steps * HALFSTEPS_PER_STEP)
            cells = s.num_cells()
        row = {"P": P, "N": pr.N, "cfl": CFL_HIGH[P], "ms_per_halfstep": ms, "cell_updates_per_s": cells / (ms / 1e3)}
        # the oracle on a bounded sample of the same workload: a 2^14-cell
        # window around the jump, CFL half-steps for about cpu_seconds / 8
        import oracle
        win = inputs.euler_riemann_seeded(1 << 14, P)
        sol = oracle.Solver(oracle.make_law(oracle.EULER, P, limiter=True, bc=oracle.TRANSMISSIVE), win.q0, win.dx)
        t0 = time.perf_counter()
        k = 0
        while k < 2 or time.perf_counter() - t0 < args.cpu_seconds / 8:
            sol.step_cfl(1, CFL_HIGH[P])
            k += 1
        row["oracle_cell_updates_per_s"] = sol.q.shape[0] * k / (time.perf_counter() - t0)
        row["oracle_cores"] = oracle.get_threads()
        if FP64_FLOPS_HIGH[P]:
            tf = FP64_FLOPS_HIGH[P] * cells / (ms / 1e3) / 1e12
            row.update({"fp64_flops_per_cell": FP64_FLOPS_HIGH[P], "fp64_tflops": tf, "fp64_frac": tf / FP64_PEAK_TFLOPS})
        rows.append(row)
        print(json.dumps(row), flush=True)
    print(json.dumps({"clocks": clocks.stop()}), flush=True)
    print("| P | CFL | ms / half-step | cell-updates/s | FP64 flops / cell | of the FP64 peak | oracle (2^14-cell window) |")
    print("|---|---|---|---|---|---|---|")
    for r in rows:
        fl = "" if "fp64_flops_per_cell" not in r else f"{r['fp64_flops_per_cell']:.0f}"
        fr = "" if "fp64_frac" not in r else f"{r['fp64_frac']:.3f}"
        print(f"| {r['P']} | {r['cfl']} | {r['ms_per_halfstep']:.3f} | {r['cell_updates_per_s'] / 1e9:.3f} G | {fl} | {fr} | "
              f"{r['oracle_cell_updates_per_s'] / 1e6:.2f} M ({r['oracle_cores']} cores) |")


# Floating-point operations per cell-update of the oracle's half-step as the
# oracle writes it (derivative form, binomial Leibniz sums, divisions by
# constants, each parent's Cauchy-Kovalewski table counted once), limiter on:
# the output of `python oracle/count_flops.py 1 P 1` (Burgers) and `2 P 1`
# (Euler).  Reported beside the kernels' own counts, not used as a roofline.
ORACLE_FLOPS = {(1, 1): 93.0, (1, 2): 191.0, (1, 3): 314.0, (1, 4): 502.0,
                (2, 1): 517.0, (2, 2): 847.0, (2, 3): 1252.0, (2, 4): 1852.0, (2, 5): 2725.0, (2, 6): 3934.0}
# FP64 operations per cell-update the Burgers FP64 kernel executes
# (halfstep_fp64<BURGERS, P>, limiter on): DADD + DMUL + 2 DFMA thread
# instructions of one launch at N = 2^20 (ncu, profiles/burgers_halfstep.md)
# over the launch's cells, e.g. P = 3: (24167170 + 41019267 + 2 x 60018446) / 2^20.
BURGERS_FP64_FLOPS = {1: 67.17, 2: 127.37, 3: 176.64, 4: 252.11}
BURGERS_CFL = {1: 0.4, 2: 0.3, 3: 0.25, 4: 0.2}


def burgers_bench(args):
    """The Burgers workload (u_t + (u^2/2)_x = 0, periodic [0, 2 pi], seeded
    u0 = 0.5 + 8 Fourier modes, limiter on) at N = 2^10, 2^14, 2^18, 2^20
    (--burgers-log2n), P = 1..4 (CFL 0.4 / 0.3 / 0.25 / 0.2), FP64,
    FP32-mixed, and FP32-mixed with two half-steps per launch.  Per case:
    cell-updates/s over graphs of 32 half-steps with CUDA events (inputs
    resident; from the initial data: the kernels' work does not depend on
    the state), the HBM fraction at the algorithmic bytes (one read and one
    write of the state per launch: 16 (P + 1) B in FP64, 2 (8 + 4 P) B in
    FP32-mixed, half of that per cell-update with two half-steps per launch)
    and, for FP64, the fraction of the FP64 peak at the kernel's executed
    FP64 operations (BURGERS_FP64_FLOPS);
    time to 2 t_s (past the shock) for N <= 2^18; and the oracle on the host
    cores on a bounded sample (N = 2^14, CFL half-steps for about
    cpu_seconds / 8 per degree)."""
    import torch

    from paper_2104_04347_gb300 import inputs, wcc

    pk, pk_kind = peaks()
    stream = torch.cuda.Stream()
    clocks = ClockSampler()
    clocks.start()
    rows = []
    sizes = [int(x) for x in args.burgers_log2n.split(",")]
    for P in (1, 2, 3, 4):
        cfl = BURGERS_CFL[P]
        for log2n in sizes:
            N = 1 << log2n
            pr = inputs.burgers_fourier(N, P)
            t_s = inputs.shock_time(inputs.burgers_fourier_data())
            for prec, name, tb in ((wcc.FP64, "fp64", 1), (wcc.FP32_MIXED, "fp32-mixed", 1),
                                   (wcc.FP32_MIXED, "fp32-mixed-tb2", 2)):
                with wcc.Solver(pr.system, N, P, (pr.x_l, pr.x_r), pr.bc, precision=prec,
                                stream=stream.cuda_stream, tb_depth=tb) as s:
                    s.set_initial(pr.q0)
                    for _ in range(args.warmup):
                        s.step(HALFSTEPS_PER_STEP, cfl)
                    s.synchronize()
                    reps = max(args.steps, 4 if log2n >= 18 else 40)
                    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
                    with torch.cuda.stream(stream):
                        ev[0].record(stream)
                        for _ in range(reps):
                            s.step(HALFSTEPS_PER_STEP, cfl)
                        ev[1].record(stream)
                    s.synchronize()
                    ms = ev[0].elapsed_time(ev[1]) / (reps * HALFSTEPS_PER_STEP)
                    tts = None
                    if log2n <= 18:
                        s.set_initial(pr.q0)
                        t0 = time.perf_counter()
                        k = s.step_until(2.0 * t_s, cfl)
                        tts = {"t_end": 2.0 * t_s, "halfsteps": k, "seconds": time.perf_counter() - t0}
                rate = N / (ms * 1e-3)
                bpc = 16 * (P + 1) if prec == wcc.FP64 else 2 * (8 + 4 * P) / tb
                row = {"workload": f"burgers1d-fourier8-N2^{log2n}-P{P}-periodic-cfl{cfl}", "N": N, "P": P,
                       "precision": name, "ms_per_halfstep": ms, "cell_updates_per_s": rate,
                       "bytes_per_cell_update": bpc, "hbm_gbs": bpc * rate / 1e9,
                       "hbm_frac": bpc * rate / 1e9 / pk["hbm_gbs"], "time_to_2ts": tts}
                if prec == wcc.FP64:
                    tf = BURGERS_FP64_FLOPS[P] * rate / 1e12
                    row.update({"fp64_flops_per_cell_update": BURGERS_FP64_FLOPS[P],
                                "oracle_flops_per_cell_update": ORACLE_FLOPS[(1, P)], "fp64_tflops": tf,
                                "fp64_frac": tf / FP64_PEAK_TFLOPS})
                rows.append(row)
                print(json.dumps(row), flush=True)
    clk = clocks.stop()
    # the oracle on the host cores (bounded sample)
    import oracle
    oracle.set_threads(os.cpu_count() or 1)
    cpu = {}
    for P in (1, 2, 3, 4):
        win = inputs.burgers_fourier(1 << 14, P)
        sol = oracle.Solver(oracle.make_law(oracle.BURGERS, P, limiter=True), win.q0, win.dx)
        t0 = time.perf_counter()
        k = 0
        while k < 2 or time.perf_counter() - t0 < args.cpu_seconds / 8:
            sol.step_cfl(1, BURGERS_CFL[P])
            k += 1
        cpu[P] = win.N * k / (time.perf_counter() - t0)
    print(json.dumps({"clocks": clk, "peak_hbm_gbs": pk["hbm_gbs"], "peak_source": pk_kind,
                      "oracle_cell_updates_per_s": cpu, "oracle_cores": oracle.get_threads(),
                      "oracle_sample": "N = 2^14, CFL half-steps from the initial data"}), flush=True)
    print("| P | N | precision | ms / half-step | cell-updates/s | of HBM | of FP64 peak (kernel flops) | "
          "time to 2 t_s | oracle (host) |")
    print("|---|---|---|---|---|---|---|---|---|")
    for r in rows:
        fr = f"{r['fp64_frac']:.3f}" if "fp64_frac" in r else ""
        tt = "" if r["time_to_2ts"] is None else f"{r['time_to_2ts']['seconds']:.3f} s ({r['time_to_2ts']['halfsteps']})"
        print(f"| {r['P']} | 2^{int(math.log2(r['N']))} | {r['precision']} | {r['ms_per_halfstep']:.4f} | "
              f"{r['cell_updates_per_s'] / 1e9:.2f} G | {r['hbm_frac']:.3f} | {fr} | {tt} | "
              f"{cpu[r['P']] / 1e6:.2f} M |")


def advection_config(args):
    """The linear-advection workload: u0 = sin(pi x) on periodic [0, 2],
    N = 200, P = 2, limiter off, to t = 2 (one period; the exact solution is
    the initial data) at nu = 0.25 (the half-step reading of CFL 0.5), FP64.
    Reports the time to solution through wcc_step_dt (host clock around the
    synchronous run, second pass), L1 of the point values against the exact
    translate, and the oracle's time and L1 on the host cores."""
    import oracle
    from paper_2104_04347_gb300 import inputs, wcc

    pr = inputs.advection_sine(200, 2, 0.0, 2.0)
    dts = oracle.constant_speed_dts(2.0, 0.25 * pr.dx)
    x = inputs.centres(200, 0.0, 2.0, inputs.PERIODIC)
    exact = np.sin(np.pi * x)
    with wcc.Solver(pr.system, 200, 2, (0.0, 2.0), pr.bc, limiter=False) as s:
        for _ in range(2):
            s.set_initial(pr.q0)
            t0 = time.perf_counter()
            s.step_dt(dts)
            q = s.get_dofs()
            secs = time.perf_counter() - t0
    oracle.set_threads(1)
    sol = oracle.Solver(oracle.make_law(oracle.ADVECTION, 2, limiter=False), pr.q0, pr.dx)
    t0 = time.perf_counter()
    sol.step_dt(dts)
    osecs = time.perf_counter() - t0
    row = {"workload": "advection1d-sine-N200-P2-periodic-nu0.25-t2", "halfsteps": len(dts),
           "gpu_seconds": secs, "gpu_cell_updates_per_s": 200 * len(dts) / secs,
           "l1_vs_exact": float(np.mean(np.abs(q[:, 0, 0] - exact))),
           "max_vs_oracle": float(np.max(np.abs(q - sol.q))),
           "oracle_seconds": osecs, "oracle_cell_updates_per_s": 200 * len(dts) / osecs, "oracle_cores": 1,
           "note": "200 cells: the GPU run is bound by launch latency, one launch per half-step"}
    print(json.dumps(row), flush=True)


def paper_workloads_2d(n=1200):
    """The 2D Riemann problems of Sec. 5.3 at the paper's resolution (n x n
    cells on [-1, 1]^2, transmissive): configuration 1 (four shocks) to
    t = 1.1 and configuration 2 (four contacts) to t = 1, P = 1..3 with the
    Sec. 5 CFL numbers, limiter on, through wcc2d_step_until.  Reports the
    half-steps, the time to solution (second pass on the handle, host clock
    around the synchronous call) and the density range.  FP32-mixed and FP32
    at every P; FP64 at P = 1."""
    from paper_2104_04347_gb300 import inputs, wcc

    nu = {1: 0.4, 2: 0.3, 3: 0.25}
    rows = []
    for cfg, t_end in ((1, 1.1), (2, 1.0)):
        for P in (1, 2, 3):
            pr = inputs.riemann2d(n, P, cfg)
            precs = ((wcc.FP32_MIXED, "fp32-mixed"), (wcc.FP32, "fp32"))
            if P == 1:
                precs += ((wcc.FP64, "fp64"),)
            for prec, name in precs:
                with wcc.Solver2D(pr.system, n, n, P, (pr.x_l, pr.x_r, pr.y_l, pr.y_r), pr.bc, precision=prec,
                                  rows_per_cta=16) as s:
                    s.set_initial(pr.q0)
                    s.step_until(t_end, nu[P])  # first pass: history growth, warm caches
                    s.set_initial(pr.q0)
                    t0 = time.perf_counter()
                    k = s.step_until(t_end, nu[P])
                    secs = time.perf_counter() - t0
                    q = s.get_dofs()
                    launches = s.launch_count()
                rho = q[:, :, 0, 0]
                row = {"workload": f"riemann2d-{cfg}", "n": n, "P": P, "precision": name, "t_end": t_end,
                       "halfsteps": k, "seconds": secs, "ms_per_halfstep": 1e3 * secs / k,
                       "cell_updates_per_s": n * n * k / secs, "rho_min": float(rho.min()), "rho_max": float(rho.max())}
                rows.append(row)
                print(json.dumps(row), flush=True)
    print("| problem | P | precision | half-steps | time to t_end | ms / half-step | cell-updates/s | density range |")
    print("|---|---|---|---|---|---|---|---|")
    for r in rows:
        print(f"| {r['workload']} (t = {r['t_end']}) | {r['P']} | {r['precision']} | {r['halfsteps']} | {r['seconds']:.2f} s | "
              f"{r['ms_per_halfstep']:.3f} | {r['cell_updates_per_s'] / 1e9:.2f} G | {r['rho_min']:.3f} .. {r['rho_max']:.3f} |")


def main():
    args = parse()
    if args.workloads2d:
        paper_workloads_2d()
        return
    if args.high_order:
        high_order_bench(args)
        return
    if args.burgers:
        burgers_bench(args)
        return
    if args.advection:
        advection_config(args)
        return
    if args.two_d:
        two_d_bench(args)
        return
    if args.sweep:
        precision_sweep(args.sweep_max_log2n)
        return
    if args.workloads:
        paper_workloads()
        return
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_wcc(args, rank, world)


if __name__ == "__main__":
    main()
