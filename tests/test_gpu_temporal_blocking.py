"""Two half-steps per launch (tb_depth = 2, temporal blocking) in the FP32
variants, through the C ABI.

A pair shares one dt, the CFL step of its first stage; the second
half-step's own CFL number is checked on the device and a refused pair is
re-done as two single half-steps.  Checks:
  * against the FP64 oracle replaying the realised dt list (the FP32-mixed
    rules: L1 <= 1e-6 of scale, per entry the FP32 rounding envelope of
    tests/gpu_common.fp32_pair_violation);
  * against single half-steps taking the same dt list;
  * the bookkeeping: dt comes in equal pairs, t is their sum, parity and
    half-step counts, an odd count ends with one single half-step;
  * refused pairs (tb_cfl_growth = -1 refuses every pair): the result is bit
    for bit that of single half-steps;
  * tile edges, tiny meshes, both boundaries, P = 1..4, and the benchmark
    grid (N = 2^22) on sampled windows."""
import numpy as np
import pytest

import oracle
from paper_2104_04347_gb300 import inputs, wcc
from tests.gpu_common import SCATTER_FACTOR, fp32_pair_violation, law_of, oracle_l1_spread, oracle_run, scales
from tests.test_gpu_parity import CFL, _problem

pytestmark = pytest.mark.gpu

TILE_TB = 254  # final cells per CTA of the two-half-step kernel
L1_TOL = 1e-6


def l1_rel(q, ref):
    return float(np.max(np.mean(np.abs(q[:, :, 0] - ref[:, :, 0]), axis=0) / scales(ref)))


def run(pr, nsteps, cfl, *, tb_depth=2, growth=0.1, precision=wcc.FP32_MIXED, graph_chunk=32, dts=None):
    with wcc.Solver(pr.system, pr.N, pr.P, (pr.x_l, pr.x_r), pr.bc, precision=precision, graph_chunk=graph_chunk,
                    tb_depth=tb_depth, tb_cfl_growth=growth) as s:
        s.set_initial(pr.q0)
        if dts is None:
            s.step(nsteps, cfl)
        else:
            s.step_dt(dts)
        q = s.get_dofs()
        t, k, parity = s.state()
        hist = s.dt_history()
        stats = s.tb_stats() if tb_depth == 2 else None
    return q, hist, t, k, parity, stats


CASES = [(inputs.EULER, 3, inputs.TRANSMISSIVE), (inputs.EULER, 3, inputs.PERIODIC),
         (inputs.EULER, 2, inputs.TRANSMISSIVE), (inputs.EULER, 1, inputs.PERIODIC),
         (inputs.EULER, 4, inputs.TRANSMISSIVE), (inputs.BURGERS, 3, inputs.PERIODIC),
         (inputs.BURGERS, 2, inputs.TRANSMISSIVE), (inputs.ADVECTION, 2, inputs.PERIODIC),
         (inputs.ADVECTION, 4, inputs.TRANSMISSIVE)]


def _id(c):
    return f"{['adv', 'burgers', 'euler'][c[0]]}-P{c[1]}-{['periodic', 'transmissive'][c[2]]}"


@pytest.mark.parametrize("case", CASES, ids=_id)
def test_pairs_against_oracle(case):
    system, P, bc = case
    pr = _problem(system, P, 5 * TILE_TB + 37, bc)
    q, dts, t, k, parity, (pairs, fallbacks, nu2) = run(pr, 100, CFL[P])
    assert k == 100 and parity == 0 and len(dts) == 100
    assert np.array_equal(dts[0::2], dts[1::2])          # one dt per pair
    assert fallbacks == 0 and pairs == 50
    assert 0.0 < nu2 <= CFL[P] * 1.1
    ref, tref, _ = oracle_run(pr, dts)
    assert abs(t - tref) <= 1e-14 * tref
    assert l1_rel(q, ref) <= L1_TOL


@pytest.mark.parametrize("case", CASES[:6], ids=_id)
def test_pairs_match_single_halfsteps(case):
    # the same dt list taken one half-step per launch: the same arithmetic,
    # equal to FP32 rounding (the kernels may contract multiply-adds
    # differently)
    system, P, bc = case
    pr = _problem(system, P, 3 * TILE_TB + 11, bc)
    q2, dts, _, _, _, _ = run(pr, 64, CFL[P])
    q1, d1, _, _, _, _ = run(pr, None, None, tb_depth=1, dts=dts)
    assert np.array_equal(d1, dts)
    assert fp32_pair_violation(pr, q2, q1, dts) <= 1.0


@pytest.mark.parametrize("nsteps", [1, 2, 7, 33, 64])
def test_bookkeeping_and_odd_counts(nsteps):
    pr = inputs.euler_riemann_seeded(1000, 3)
    q, dts, t, k, parity, (pairs, fb, _) = run(pr, nsteps, 0.2)
    assert k == nsteps and len(dts) == nsteps and parity == nsteps % 2
    assert pairs == nsteps // 2 and fb == 0
    assert q.shape[0] == inputs.num_cells(pr.N, pr.bc, parity)
    assert np.array_equal(dts[0:2 * pairs:2], dts[1:2 * pairs:2])
    assert t == pytest.approx(float(np.sum(dts)), rel=1e-15)
    ref, _, _ = oracle_run(pr, dts)
    assert l1_rel(q, ref) <= L1_TOL


@pytest.mark.parametrize("bc", [inputs.PERIODIC, inputs.TRANSMISSIVE])
def test_refused_pairs_equal_single_halfsteps(bc):
    # growth -1 makes the bound 0: every pair is refused and re-done singly
    pr = _problem(inputs.EULER, 3, 2 * TILE_TB + 5, bc)
    q2, d2, _, k, _, (pairs, fb, _) = run(pr, 40, 0.2, growth=-1.0)
    q1, d1, _, _, _, _ = run(pr, 40, 0.2, tb_depth=1)
    assert k == 40 and pairs == 0 and fb == 20
    assert np.array_equal(d2, d1)
    assert np.array_equal(q2, q1)


def test_partly_refused_pairs():
    # growth 0: a pair is taken only when the bound does not grow over its
    # first half-step; the rest are re-done singly.  Riemann data (its bound
    # moves every half-step) against the oracle replaying the realised dts.
    pr = inputs.euler_riemann_seeded(3000, 3)
    q, dts, _, k, _, (pairs, fb, nu2) = run(pr, 120, 0.2, growth=0.0)
    assert k == 120 and 2 * pairs + 2 * fb == 120
    assert pairs > 0 and fb > 0
    assert nu2 <= 0.2 * (1 + 1e-15)
    ref, _, _ = oracle_run(pr, dts)
    assert l1_rel(q, ref) <= L1_TOL


@pytest.mark.parametrize("N", [4, 5, TILE_TB - 1, TILE_TB, TILE_TB + 1, 2 * TILE_TB, 2 * TILE_TB + 2])
@pytest.mark.parametrize("bc", [inputs.PERIODIC, inputs.TRANSMISSIVE])
def test_tile_edges_and_tiny_meshes(N, bc):
    # L1 within 1e-6, or within 50 x the oracle's own L1 spread when its
    # input is perturbed at FP32 rounding level: on the 5-cell Riemann mesh
    # the limiter amplifies 1e-7 input noise a hundredfold (spread ~1e-5)
    pr = _problem(inputs.EULER, 3, N, bc)
    q, dts, _, _, _, (pairs, fb, _) = run(pr, 24, 0.2)
    assert pairs == 12 and fb == 0
    ref, spread = oracle_l1_spread(pr, dts, 1e-7)
    assert l1_rel(q, ref) <= max(L1_TOL, SCATTER_FACTOR * spread)


def test_direct_launches_equal_graphs():
    pr = inputs.euler_riemann_seeded(2000, 3)
    qa, da, _, _, _, _ = run(pr, 70, 0.2, graph_chunk=32)
    qb, db, _, _, _, _ = run(pr, 70, 0.2, graph_chunk=0)
    assert np.array_equal(da, db) and np.array_equal(qa, qb)


def test_step_until_with_pairs():
    pr = inputs.euler_density_wave(512, 3)
    with wcc.Solver(pr.system, pr.N, 3, (pr.x_l, pr.x_r), pr.bc, precision=wcc.FP32_MIXED, tb_depth=2) as s:
        s.set_initial(pr.q0)
        n = s.step_until(0.25, 0.25)
        t, k, parity = s.state()
        q = s.get_dofs()
        dts = s.dt_history()
    assert parity == 0 and k == n and abs(t - 0.25) < 1e-13
    ref, _, _ = oracle_run(pr, dts)
    assert l1_rel(q, ref) <= L1_TOL


def test_full_size_sampled_windows():
    # the benchmark grid, N = 2^22, P = 3, Riemann data, nu = 0.2, 64
    # half-steps in pairs (graphs of 16 pairs); the oracle recomputes windows
    # (a cell depends on the initial data within k/2 + 1 cells)
    N, P, k = 1 << 22, 3, 64
    pr = inputs.euler_riemann_seeded(N, P)
    q, dts, _, _, parity, (pairs, fb, _) = run(pr, k, 0.2)
    assert parity == 0 and pairs == k // 2 and fb == 0
    rng = np.random.default_rng(11)
    centres = [N // 2, 3, N - 3] + list(rng.integers(200, N - 200, 3))
    half = k // 2 + 8
    law = law_of(pr)
    got, want = [], []
    for c in centres:
        lo, hi = max(0, c - 2 * half), min(N + 1, c + 2 * half)
        s = oracle.Solver(law, pr.q0[lo:hi], pr.dx)
        s.step_dt(dts)
        a = lo if lo == 0 else lo + half
        b = hi if hi == N + 1 else hi - half
        got.append(q[a:b])
        want.append(s.q[a - lo:b - lo])
    got, want = np.concatenate(got), np.concatenate(want)
    sc = np.max(np.abs(pr.q0[:, :, 0]), axis=0)
    assert float(np.max(np.mean(np.abs(got[:, :, 0] - want[:, :, 0]), axis=0) / sc)) <= L1_TOL
