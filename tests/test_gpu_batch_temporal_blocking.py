"""Batches with two half-steps per launch (tb_depth = 2), FP32-mixed.

One launch advances every instance of the batch by two half-steps with one
dt per instance and pair (the CFL step of the pair's first stage).  The
second half-step's CFL number is checked on the device for every instance;
when any instance exceeds its bound the launch leaves the whole batch
untouched and the host re-does the pair as two single half-steps.  Checks:
  * each instance against the FP64 oracle replaying its realised dt list
    (L1 <= 1e-6 of the variable's scale, the FP32-mixed bound);
  * each instance against the same problem run alone with single half-steps
    on the same dt list (the FP32 rounding envelope of
    tests/gpu_common.fp32_pair_violation);
  * the bookkeeping: equal dts within a pair, times, half-step counts and
    parity, odd counts ending with one single half-step;
  * refused pairs (tb_cfl_growth = -1 refuses every pair) give bit for bit
    the single-half-step batch;
  * the autotuner's choice of grid and pass depth keeps the state and
    reproduces a batch created with that configuration;
  * degree mixes {2}, {3}, {2, 3} and the benchmark batch on sampled
    instances."""
import numpy as np
import pytest

from paper_2104_04347_gb300 import inputs, wcc
from tests.gpu_common import fp32_pair_violation, oracle_run, scales

pytestmark = pytest.mark.gpu

CFL = 0.2
L1_TOL = 1e-6


def _l1(q, ref):
    return float(np.max(np.mean(np.abs(q[:, :, 0] - ref[:, :, 0]), axis=0) / scales(ref)))


def _batch(count, seed, degrees=(2, 3), n_max=900):
    return inputs.batch_workload(count, n_min=8, n_max=n_max, seed=seed, degrees=degrees)


def _run(probs, nsteps, *, tb_depth=2, growth=0.1, grid=None, graph_chunk=32):
    with wcc.Batch(probs, tb_depth=tb_depth, tb_cfl_growth=growth, graph_chunk=graph_chunk) as b:
        b.set_initial()
        if grid is not None:
            b.set_grid(grid)
        b.step(nsteps, CFL)
        qs = b.get_dofs()
        hists = [b.dt_history(i) for i in range(len(probs))]
        stats = b.tb_stats()
        state = b.state()
        times = b.times()
    return qs, hists, stats, state, times


def _alone_on(pr, dts):
    with wcc.Solver(pr.system, pr.N, pr.P, (pr.x_l, pr.x_r), pr.bc, precision=wcc.FP32_MIXED) as s:
        s.set_initial(pr.q0)
        s.step_dt(dts)
        return s.get_dofs()


@pytest.mark.parametrize("degrees", [(2, 3), (3,), (2,)], ids=["P23", "P3", "P2"])
def test_pairs_match_single_halfsteps_alone(degrees):
    probs = _batch(30, 7, degrees)
    nsteps = 60
    qs, hists, (pairs, fb), state, times = _run(probs, nsteps)
    assert state == (nsteps, 0)
    assert pairs + fb == nsteps // 2
    for i, pr in enumerate(probs):
        h = hists[i]
        assert len(h) == nsteps
        if fb == 0:
            assert np.array_equal(h[0::2], h[1::2])
        assert abs(times[i] - h.sum()) <= 1e-12 * times[i]
        assert fp32_pair_violation(pr, qs[i], _alone_on(pr, h), h) <= 1.0, i


def test_pairs_against_oracle_sampled():
    probs = _batch(24, 11)
    qs, hists, (pairs, fb), _, _ = _run(probs, 100)
    assert pairs > 0
    for i in (0, 5, 11, 17, 23):
        ref, _, _ = oracle_run(probs[i], hists[i])
        assert _l1(qs[i], ref) <= L1_TOL, i


@pytest.mark.parametrize("nsteps", [1, 2, 7, 34])
def test_bookkeeping_and_odd_counts(nsteps):
    probs = _batch(12, 3)
    qs, hists, (pairs, fb), state, _ = _run(probs, nsteps, growth=10.0)
    assert state == (nsteps, nsteps % 2)
    assert pairs == nsteps // 2 and fb == 0   # growth 10: capped at the stability limit only
    for i, pr in enumerate(probs):
        h = hists[i]
        assert len(h) == nsteps
        assert np.array_equal(h[0:2 * pairs:2], h[1:2 * pairs:2])
        assert qs[i].shape[0] == inputs.num_cells(pr.N, pr.bc, nsteps % 2)
    ref, _, _ = oracle_run(probs[4], hists[4])
    assert _l1(qs[4], ref) <= L1_TOL


def test_refused_pairs_equal_single_halfstep_batch():
    probs = _batch(16, 9)
    q2, h2, (pairs, fb), s2, _ = _run(probs, 30, growth=-1.0)
    q1, h1, _, s1, _ = _run(probs, 30, tb_depth=1)
    assert pairs == 0 and fb == 15 and s1 == s2
    for a, b in zip(h2, h1):
        assert np.array_equal(a, b)
    for a, b in zip(q2, q1):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("grid", [1, 152, 100000])
def test_any_persistent_grid_gives_the_same_result(grid):
    probs = _batch(16, 5)
    ref, _, _, _, _ = _run(probs, 20, growth=10.0)
    got, _, _, _, _ = _run(probs, 20, growth=10.0, grid=grid)
    for a, b in zip(ref, got):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("growth", [0.1, -1.0])
def test_direct_launches_equal_graphs(growth):
    # graph_chunk 0 launches every pair directly; 6 pairs per graph leaves a
    # direct tail; refusals (growth -1) go through the same recovery
    probs = _batch(12, 17)
    ref = _run(probs, 38, growth=growth)
    for chunk in (0, 12):
        got = _run(probs, 38, growth=growth, graph_chunk=chunk)
        assert got[2] == ref[2] and got[3] == ref[3]
        for a, b in zip(got[1], ref[1]):
            assert np.array_equal(a, b)
        for a, b in zip(got[0], ref[0]):
            assert np.array_equal(a, b)


def test_autotune_chooses_depth_and_keeps_the_state():
    # tuned right after loading, then stepped: as a fresh batch created with
    # the chosen pass depth (the grid does not change results)
    probs = _batch(30, 13)
    with wcc.Batch(probs) as a, wcc.Batch(probs) as fresh:
        a.set_initial()
        fresh.set_initial()
        ctas = a.autotune(CFL)
        grid, depth = a.tuning()
        assert ctas == grid > 0 and depth in (1, 2)
        assert a.state() == (0, 0) and not np.any(a.times())
        for x, y in zip(a.get_dofs(), fresh.get_dofs()):
            assert np.array_equal(x, y)
        a.step(46, CFL)
        qa = a.get_dofs()
        ha = [a.dt_history(i) for i in range(len(probs))]
        assert a.state() == (46, 0)
    with wcc.Batch(probs, tb_depth=depth) as b:
        b.set_initial()
        b.step(46, CFL)
        qb = b.get_dofs()
        hb = [b.dt_history(i) for i in range(len(probs))]
    for x, y in zip(ha, hb):
        assert np.array_equal(x, y)
    for x, y in zip(qa, qb):
        assert np.array_equal(x, y)


def test_depth_two_needs_degrees_two_and_three():
    probs = _batch(6, 1, degrees=(3, 4))
    with pytest.raises(wcc.WCCError):
        wcc.Batch(probs, tb_depth=2)
    with wcc.Batch(probs) as b:       # the autotuner then times one depth only
        b.set_initial()
        b.autotune(CFL)
        assert b.tuning()[1] == 1


def test_full_batch_workload_sampled():
    # the batched benchmark workload (4096 instances, N log-uniform in
    # [256, 65536], P in {2, 3}) in pairs; sampled instances against their
    # own single half-steps on the same dts and against the oracle
    probs = inputs.batch_workload()
    nsteps = 64
    with wcc.Batch(probs, tb_depth=2) as b:
        b.set_initial()
        b.step(nsteps, CFL)
        qs = b.get_dofs()
        pairs, fb = b.tb_stats()
        rng = np.random.default_rng(2)
        picks = [int(i) for i in rng.integers(0, len(probs), 5)]
        hists = {i: b.dt_history(i) for i in picks}
    assert pairs + fb == nsteps // 2 and pairs > 0
    for i in picks:
        assert fp32_pair_violation(probs[i], qs[i], _alone_on(probs[i], hists[i]), hists[i]) <= 1.0
    ref, _, _ = oracle_run(probs[picks[0]], hists[picks[0]])
    assert _l1(qs[picks[0]], ref) <= L1_TOL
