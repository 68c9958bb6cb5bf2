"""The reference arm of bench.py (the CPU oracle, no GPU needed) prints one
JSON line with the keys the benchmark contract asks for."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "2",
                          "--warmup", "1", "--log2n", "12"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["value"] > 0 and d["ms_per_step"] > 0 and d["higher_is_better"] is True
    assert d["steps"] == 2 and d["warmup"] == 1
    assert d["config"]["workload"].startswith("euler1d-riemann-N2^12-P3")
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert cb["host"]["nproc"] >= 1 and cb["host"]["machine"] and cb["host"]["cpu"]
    assert d["per_full_step"]["value"] == d["value"] / 2
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_oracle_rate_on_one_thread():
    import oracle
    sys.path.insert(0, ROOT)
    import bench
    before = oracle.get_threads()
    try:
        rate, threads, sample = bench.cpu_oracle_rate(12, 0.5, threads=1)
    finally:
        oracle.set_threads(before)
    assert threads == 1 and rate > 0 and "half-steps" in sample


def test_riemann_l1_exact_of_the_oracle():
    # the oracle's density on the bench workload (N = 2^10) approaches the
    # exact Riemann solution: first order in L1 at the discontinuities
    import numpy as np
    import oracle
    from paper_2104_04347_gb300 import inputs
    sys.path.insert(0, ROOT)
    import bench
    errs = []
    for N in (256, 1024):
        pr = inputs.euler_riemann_seeded(N, 3)
        law = oracle.make_law(oracle.EULER, 3, limiter=True, bc=oracle.TRANSMISSIVE)
        s = oracle.Solver(law, pr.q0, pr.dx)
        dts = oracle.constant_speed_dts(0.05, 0.2 * pr.dx / oracle.max_speed(law, pr.q0))
        s.step_dt(dts)
        errs.append(bench.riemann_l1_exact(pr, s.q, float(np.sum(dts)), len(dts) % 2))
    assert errs[1] < 0.6 * errs[0] and errs[1] < 5e-3, errs
    # the initial data itself is the exact solution at t -> 0
    pr = inputs.euler_riemann_seeded(1000, 3)
    assert bench.riemann_l1_exact(pr, pr.q0, 1e-12) < 2e-3
