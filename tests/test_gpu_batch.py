"""Batched solving (wcc_batch_*): many independent Euler problems in one
persistent launch per half-step, FP32-mixed.

Each instance must evolve like the same problem run alone through the
single-grid FP32-mixed path: the batch runs the same tile code with the same
per-instance dt rule.  The compiler may contract multiply-adds differently
when that code is inlined into another kernel, so the two agree to FP32
rounding (L1 <= 1e-6 of the variable's scale, the mixed-precision bound),
not bit for bit: per cell within max(2e-6 x scale, 50 x the oracle's own
spread under FP32-level input perturbations) -- the limiter's conditioning
(tests/gpu_common.py) applies to FP32 rounding too.  Runs of one batch kernel are bitwise reproducible: any
persistent grid size, and the autotuner, give identical results.  Sampled
instances are also checked against the FP64 oracle."""
import numpy as np
import pytest

from paper_2104_04347_gb300 import inputs, wcc
from tests.gpu_common import fp32_pair_violation, oracle_run, scales

pytestmark = pytest.mark.gpu

CFL = 0.2


def _small_batch(count=40, seed=7):
    return inputs.batch_workload(count, n_min=8, n_max=900, seed=seed)


def _l1(q, ref):
    sc = scales(ref)
    return float(np.max(np.mean(np.abs(q[:, :, 0] - ref[:, :, 0]), axis=0) / sc))


def _alone(pr, nsteps):
    with wcc.Solver(pr.system, pr.N, pr.P, (pr.x_l, pr.x_r), pr.bc, precision=wcc.FP32_MIXED) as s:
        s.set_initial(pr.q0)
        s.step(nsteps, CFL)
        return s.get_dofs(), s.dt_history(), s.state()[0]


def test_batch_matches_instances_run_alone():
    probs = _small_batch()
    nsteps = 60
    with wcc.Batch(probs) as b:
        b.set_initial()
        b.step(nsteps, CFL)
        qs = b.get_dofs()
        times = b.times()
        hists = [b.dt_history(i) for i in range(len(probs))]
    for i, pr in enumerate(probs):
        q, dts, t = _alone(pr, nsteps)
        assert len(hists[i]) == nsteps
        np.testing.assert_allclose(hists[i], dts, rtol=1e-5)
        assert abs(times[i] - hists[i].sum()) <= 1e-12 * times[i]
        assert fp32_pair_violation(pr, qs[i], q, hists[i]) <= 1.0, i


def test_batch_odd_steps_and_layout():
    probs = _small_batch(12, seed=3)
    with wcc.Batch(probs) as b:
        b.set_initial()
        b.step(7, CFL)
        assert b.state() == (7, 1)
        qs = b.get_dofs()
    for i, pr in enumerate(probs):
        q, _, _ = _alone(pr, 7)
        assert q.shape[0] == inputs.num_cells(pr.N, pr.bc, 1) == qs[i].shape[0]
        assert np.max(np.abs(qs[i] - q)) <= 1e-5 * np.max(np.abs(q))


def test_batch_against_oracle_sampled():
    probs = _small_batch(24, seed=11)
    with wcc.Batch(probs) as b:
        b.set_initial()
        b.step(100, CFL)
        qs = b.get_dofs()
        hists = [b.dt_history(i) for i in range(len(probs))]
    for i in (0, 5, 11, 17, 23):
        ref, _, _ = oracle_run(probs[i], hists[i])
        sc = scales(ref)
        l1 = np.max(np.mean(np.abs(qs[i][:, :, 0] - ref[:, :, 0]), axis=0) / sc)
        assert l1 <= 1e-6, (i, l1)


def test_autotune_keeps_the_state():
    # the autotuner times candidate launches on the batch itself and puts
    # the stages, times, step counts and dt histories back
    probs = _small_batch(30, seed=5)
    with wcc.Batch(probs) as a, wcc.Batch(probs) as b:
        a.set_initial()
        b.set_initial()
        a.step(5, CFL)
        b.step(5, CFL)
        ctas = a.autotune(CFL)
        assert ctas > 0 and a.tuning()[0] == ctas
        for qa, qb in zip(a.get_dofs(), b.get_dofs()):
            assert np.array_equal(qa, qb)
        assert a.state() == b.state() == (5, 1)
        assert np.array_equal(a.times(), b.times())
        for i in range(len(probs)):
            assert np.array_equal(a.dt_history(i), b.dt_history(i))
        a.step(40, CFL)
        assert a.state() == (45, 1)


def _run_batch(probs, nsteps, grid=None):
    with wcc.Batch(probs) as a:
        a.set_initial()
        if grid is not None:
            a.set_grid(grid)
        a.step(nsteps, CFL)
        return a.get_dofs()


@pytest.mark.parametrize("grid", [1, 7, 152, 100000])
def test_any_persistent_grid_gives_the_same_result(grid):
    probs = _small_batch(16, seed=9)
    ref = _run_batch(probs, 20)
    got = _run_batch(probs, 20, grid)
    for a, b in zip(ref, got):
        assert np.array_equal(a, b)


def test_batch_errors():
    probs = _small_batch(6, seed=1)
    probs[2].P = 4
    probs[3].P = 1
    with pytest.raises(wcc.WCCError):
        wcc.Batch(probs)  # more than two degrees
    probs = _small_batch(6, seed=1)
    bad = [p.q0.copy() for p in probs]
    bad[4][0, 0, 0] = -1.0
    with wcc.Batch(probs) as b:
        with pytest.raises(wcc.WCCError) as ei:
            b.set_initial(bad)
        assert ei.value.code == -6
        with pytest.raises(wcc.WCCError) as ei:
            b.step(2, CFL)
        assert ei.value.code == -2
        b.set_initial()
        b.step(4, CFL)
        b.synchronize()


def test_full_batch_workload_sampled():
    # The batched benchmark workload: 4096 instances, N log-uniform in
    # [256, 65536], P in {2, 3}; sampled instances against their own runs.
    probs = inputs.batch_workload()
    nsteps = 64
    with wcc.Batch(probs) as b:
        b.set_initial()
        b.step(nsteps, CFL)
        qs = b.get_dofs()
        rng = np.random.default_rng(2)
        picks = list(rng.integers(0, len(probs), 6))
        hists = {i: b.dt_history(i) for i in picks}
    for i in picks:
        q, dts, _ = _alone(probs[i], nsteps)
        np.testing.assert_allclose(hists[i], dts, rtol=1e-5)
        assert fp32_pair_violation(probs[i], qs[i], q, hists[i]) <= 1.0
