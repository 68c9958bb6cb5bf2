"""Benchmark of the 1D WCC half-step on GB300.

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

Under torchrun each rank runs an independent replica (the path has no
exchange step here); value = cell-updates of all ranks / max time.
--impl reference times the CPU oracle on the host cores (rank 0 only).
"""
from __future__ import annotations

import argparse
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
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="wcc", choices=["wcc", "reference"])
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"])
    ap.add_argument("--log2n", type=int, default=22)
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    return ap.parse_args()


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
# (2 x 1053618000 + 207934209 + 378169546) / 2097152.5.
FP64_FLOPS_PER_CELL_UPDATE = 1284.3
# DRAM bytes (read + write) of one FP64 launch, from the same capture
# (201536256 + 149675008 at N = 2^21), scaled by cells to N = 2^22.
FP64_TRAFFIC_PER_CELL = (201536256 + 149675008) / 2097152.5
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


def cpu_oracle_rate(log2n, seconds):
    """Oracle cell-updates/s on the host cores over a bounded sample of the
    workload: a contiguous window of the N = 2^log2n grid around the jump,
    advanced with the CFL rule until ~`seconds` of CPU time are spent."""
    import oracle
    from paper_2104_04347_gb300 import inputs

    threads = os.cpu_count() or 1
    oracle.set_threads(threads)
    N = 1 << log2n
    pr = inputs.euler_riemann_seeded(N, P)
    win = 1 << 16
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
    if rank != 0:
        return
    rate, cores, sample = cpu_oracle_rate(args.log2n, max(1.0, args.cpu_seconds))
    line = {
        "impl": "reference", "metric": METRIC, "value": rate, "unit": "cell-updates/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": None, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_name(args.log2n), "N": 1 << args.log2n, "P": P,
                   "precision": "fp64", "halfsteps_per_step": HALFSTEPS_PER_STEP},
        "cpu_baseline": {"value": rate, "unit": "cell-updates/s", "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": rate, "unit": "cell-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------ GPU


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
    prec = wcc.FP64 if args.precision == "fp64" else wcc.FP32_MIXED

    N = 1 << args.log2n
    pr = inputs.euler_riemann_seeded(N, P)
    solver = wcc.Solver(pr.system, N, P, (pr.x_l, pr.x_r), pr.bc, precision=prec,
                        graph_chunk=HALFSTEPS_PER_STEP, stream=stream.cuda_stream)
    solver.set_initial(pr.q0)
    ncells = solver.num_cells()           # integer stage: N + 1; half stage: N
    cells_per_step = (HALFSTEPS_PER_STEP // 2) * ((N + 1) + N)

    def barrier():
        if dist:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        solver.step(HALFSTEPS_PER_STEP, CFL)
    solver.synchronize()

    # ---- device-resident timing
    launches0 = solver.launch_count()
    clocks = ClockSampler()
    clocks.start()
    barrier()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    with torch.cuda.stream(stream):
        ev[0].record(stream)
        for k in range(args.steps):
            solver.step(HALFSTEPS_PER_STEP, CFL)
            ev[k + 1].record(stream)
    barrier()
    clk = clocks.stop()
    solver.synchronize()
    launches = solver.launch_count() - launches0
    total_ms = ev[0].elapsed_time(ev[-1])
    step_ms = [ev[k].elapsed_time(ev[k + 1]) for k in range(args.steps)]
    if dist:
        t = torch.tensor([total_ms], device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        total_ms = float(t.item())
    value = world * cells_per_step * args.steps / (total_ms * 1e-3)
    kernel_ms = statistics.median(step_ms) / HALFSTEPS_PER_STEP

    # ---- end to end through the public API with host buffers
    count = pr.q0.size
    h_in = torch.from_numpy(pr.q0.reshape(-1).copy()).pin_memory()
    h_out = torch.empty(count, dtype=torch.float64).pin_memory()
    e2e_steps = max(2, min(args.steps, 5))
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        solver.set_initial_ptr(h_in.data_ptr(), count)
        solver.step(HALFSTEPS_PER_STEP, CFL)
        solver.get_dofs_ptr(h_out.data_ptr(), count)
    barrier()
    e2e_s = time.perf_counter() - t0
    if dist:
        t = torch.tensor([e2e_s], device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        e2e_s = float(t.item())
    e2e_value = world * cells_per_step * e2e_steps / e2e_s
    assert np.all(np.isfinite(h_out.numpy()))

    fp64_peak_meas = wcc.measure_fp_peak(wcc.FP64)
    fp32_peak_meas = wcc.measure_fp_peak(wcc.FP32_MIXED)
    pk, pk_kind = peaks()
    bpc = bytes_per_cell_update(args.precision)
    cells_per_launch = 0.5 * ((N + 1) + N)
    if args.precision == "fp64" and FP64_FLOPS_PER_CELL_UPDATE:
        achieved = FP64_FLOPS_PER_CELL_UPDATE * cells_per_launch / (kernel_ms * 1e-3) / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": achieved / FP64_PEAK_TFLOPS,
                "traffic": FP64_TRAFFIC_PER_CELL * cells_per_launch if args.log2n == 22 else None,
                "peak_source": "nominal GB300 FP64 1.25 TFLOP/s (recipe); FMA-chain measurement alongside",
                "flops_per_cell_update": FP64_FLOPS_PER_CELL_UPDATE}
    else:
        achieved = bpc * cells_per_launch / (kernel_ms * 1e-3) / 1e9
        roof = {"bound": "hbm", "achieved": achieved, "peak": pk["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / pk["hbm_gbs"], "traffic": None,
                "peak_source": f"{pk_kind} hbm_gbs (MEASURED_PEAKS.json)" if pk_kind == "measured"
                else "fallback 6.8 TB/s"}
    roof["kernel_ms"] = kernel_ms
    roof["fp64_fma_peak_measured_tflops"] = fp64_peak_meas
    roof["fp32_fma_peak_measured_tflops"] = fp32_peak_meas
    roof["bytes_per_cell_update"] = bpc

    line = {
        "metric": METRIC, "value": value, "unit": "cell-updates/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if args.precision == "fp64" else "f32+f64",
        "data": "synthetic (seeded Riemann initial data, splitmix64 seed 2104043471)",
        "config": {"workload": workload_name(args.log2n), "N": N, "P": P, "cells_integer_stage": N + 1,
                   "precision": args.precision, "halfsteps_per_step": HALFSTEPS_PER_STEP, "cfl": CFL,
                   "limiter": True, "l2": "state > L2 (no flush needed)",
                   "parallelism": f"replicas x{world}"},
        "roofline": roof,
        "e2e": {"value": e2e_value, "unit": "cell-updates/s",
                "h2d_bytes_per_step": int(count * 8), "d2h_bytes_per_step": int(count * 8),
                "steps": e2e_steps},
        "gpu_launches": launches,
        "clocks": clk,
    }
    if rank == 0 and world == 1:
        rate, cores, sample = cpu_oracle_rate(args.log2n, args.cpu_seconds)
        line["cpu_baseline"] = {"value": rate, "unit": "cell-updates/s", "cores": cores, "kind": "oracle",
                                "sample": sample}
    solver.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        torch.distributed.destroy_process_group()


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_wcc(args, rank, world)


if __name__ == "__main__":
    main()
