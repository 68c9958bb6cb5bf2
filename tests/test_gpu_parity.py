"""GPU parity: the FP64 CUDA path (through the C ABI) against the CPU oracle,
element by element, on the same seeded inputs with the same half-step sizes.

Bound (see tests/gpu_common.py): per cell max(1e-11 x scale, 50 x the
oracle's own spread under few-ulp input perturbations); where the scheme is
well conditioned this is the plain 1e-11 bound, asserted separately for the
limiter-off runs.  Every comparison also caps the share of entries the
spread term excuses and the largest plain difference (the *_CAPS below)."""
import math

import numpy as np
import pytest

import oracle
from paper_2104_04347_gb300 import inputs, wcc
from tests.gpu_common import (TOL64, assert_parity, gpu_run, gpu_solver, law_of, merge, oracle_run, oracle_spread,
                              parity_report, scaled_error, trajectory_check)

pytestmark = pytest.mark.gpu

TILE = 127  # new cells per CTA
CFL = {1: 0.4, 2: 0.3, 3: 0.25, 4: 0.2}

# Caps on what the spread term of the bound may excuse (gpu_common.Parity):
# the share of entries beyond 1e-11 x scale and the largest plain relative
# difference, about 2-3 x the values measured on GB300.  Trajectories not
# listed are well conditioned and held to the plain 1e-11 bound (nothing
# excused); the listed ones carry the limiter's conditioning near shocks,
# jumps and (P = 2) smooth extrema.  Per half-step the spread term excuses
# at most 0.02 % of the entries, none by more than 1.2e-11.
PLAIN = dict(excused_max=0.0, raw_max=TOL64)
TRAJECTORY_CAPS = {
    (inputs.BURGERS, 2, inputs.PERIODIC): dict(excused_max=0.02, raw_max=1e-9),
    (inputs.BURGERS, 2, inputs.TRANSMISSIVE): dict(excused_max=0.03, raw_max=1e-9),
    (inputs.BURGERS, 3, inputs.PERIODIC): dict(excused_max=0.02, raw_max=1e-9),
    (inputs.BURGERS, 3, inputs.TRANSMISSIVE): dict(excused_max=0.02, raw_max=1e-9),
    (inputs.BURGERS, 4, inputs.TRANSMISSIVE): dict(excused_max=0.002, raw_max=1e-10),
    (inputs.EULER, 2, inputs.TRANSMISSIVE): dict(excused_max=0.10, raw_max=3e-4),
    (inputs.EULER, 3, inputs.TRANSMISSIVE): dict(excused_max=0.06, raw_max=1e-7),
    (inputs.EULER, 4, inputs.TRANSMISSIVE): dict(excused_max=0.05, raw_max=2e-8),
}
STEP_CAPS = dict(excused_max=0.002, raw_max=5e-11)
EDGE_CAPS = dict(excused_max=0.06, raw_max=1e-10)
FULL_SIZE_CAPS = dict(excused_max=0.02, raw_max=1e-9)


def _problem(system, P, N, bc):
    if system == inputs.ADVECTION:
        if bc == inputs.PERIODIC:
            return inputs.advection_sine(N, P)
        return inputs.advection_polynomial(N, P, [0.2, -0.5, 0.7, 0.1, -0.3][: P + 1])
    if system == inputs.BURGERS:
        pr = inputs.burgers_fourier(N, P)
        if bc == inputs.TRANSMISSIVE:
            pr = inputs.Problem(pr.system, N, P, pr.x_l, pr.x_r, bc, np.concatenate([pr.q0, pr.q0[:1]]))
        return pr
    if bc == inputs.TRANSMISSIVE:
        return inputs.euler_riemann_seeded(N, P)
    return inputs.euler_density_wave(N, P)


ALL = [(s, P, bc) for s in (inputs.ADVECTION, inputs.BURGERS, inputs.EULER) for P in (1, 2, 3, 4)
       for bc in (inputs.PERIODIC, inputs.TRANSMISSIVE)]


def _id(c):
    return f"{['adv', 'burgers', 'euler'][c[0]]}-P{c[1]}-{['periodic', 'transmissive'][c[2]]}"


@pytest.mark.parametrize("case", ALL, ids=_id)
def test_trajectory_100_halfsteps(case):
    system, P, bc = case
    N = 5 * TILE + 38          # several tiles and a ragged tail
    pr = _problem(system, P, N, bc)
    q, dts, t, parity = gpu_run(pr, 100, CFL[P])
    assert len(dts) == 100 and parity == 0
    ref, tref, _ = oracle_run(pr, dts)
    assert abs(t - tref) <= 1e-14 * tref and q.shape == ref.shape
    rep = trajectory_check(pr, q, dts)
    assert_parity(rep, **TRAJECTORY_CAPS.get(case, PLAIN))


@pytest.mark.parametrize("case", ALL, ids=_id)
def test_every_halfstep_from_gpu_state(case):
    # Teacher-forced: each GPU half-step against one oracle half-step from the
    # GPU's own previous state (exported through the ABI).
    system, P, bc = case
    N = 3 * TILE + 17
    pr = _problem(system, P, N, bc)
    law = law_of(pr)
    reps = []
    with gpu_solver(pr) as s:
        s.set_initial(pr.q0)
        prev = s.get_dofs()
        for n in range(60):
            parity = s.state()[2]
            s.step(1, CFL[P])
            cur = s.get_dofs()
            lam = s.dt_history()[-1] / pr.dx

            def run(q):
                return oracle.halfstep(law, parity, q, lam)

            ref = run(prev)
            spread = oracle_spread(run, prev, ref, seed=n)
            reps.append(parity_report(cur, ref, spread))
            prev = cur
    assert_parity(merge(reps), **STEP_CAPS)


@pytest.mark.parametrize("system", [inputs.ADVECTION, inputs.BURGERS, inputs.EULER])
@pytest.mark.parametrize("P", [1, 2, 3, 4])
def test_limiter_off_plain_bound(system, P):
    # Without the limiter the scheme is well conditioned: plain 1e-11 bound.
    N = 4 * TILE + 5
    pr = _problem(system, P, N, inputs.PERIODIC)
    q, dts, _, _ = gpu_run(pr, 100, CFL[P], limiter=False)
    ref, _, _ = oracle_run(pr, dts, limiter=False)
    assert scaled_error(q, ref) <= TOL64


@pytest.mark.parametrize("P", [3, 4])
def test_smooth_euler_limiter_on_plain_bound(P):
    # (P = 2 is left to the conditioning-aware trajectory test: its limiter
    # reacts to rounding-level slopes at the extrema of the wave.)
    pr = inputs.euler_density_wave(600, P)
    q, dts, _, _ = gpu_run(pr, 100, CFL[P])
    ref, _, _ = oracle_run(pr, dts)
    assert scaled_error(q, ref) <= TOL64


def test_config1_advection_exact_translate():
    # Advection of sin(pi x) on periodic [0, 2], N = 200, P = 2, limiter off,
    # to t = 2 (one period) with nu = 0.25.
    pr = inputs.advection_sine(200, 2, 0.0, 2.0)
    dts = oracle.constant_speed_dts(2.0, 0.25 * pr.dx)
    q, _, t, parity = gpu_run(pr, None, None, limiter=False, dts=dts)
    ref, _, _ = oracle_run(pr, dts, limiter=False)
    assert parity == 0 and abs(t - 2.0) < 1e-12
    assert scaled_error(q, ref) <= TOL64
    x = inputs.centres(200, 0.0, 2.0, inputs.PERIODIC)
    l1 = np.mean(np.abs(q[:, 0, 0] - np.sin(math.pi * x)))
    l1_ref = np.mean(np.abs(ref[:, 0, 0] - np.sin(math.pi * x)))
    assert abs(l1 - l1_ref) < 1e-12 and l1 < 1e-6


@pytest.mark.parametrize("N", [4, 5, TILE - 1, TILE, TILE + 1, 2 * TILE])
@pytest.mark.parametrize("bc", [inputs.PERIODIC, inputs.TRANSMISSIVE])
def test_small_and_tile_edge_sizes(N, bc):
    pr = _problem(inputs.EULER, 3, N, bc)
    q, dts, _, _ = gpu_run(pr, 24, 0.2)
    assert_parity(trajectory_check(pr, q, dts), **EDGE_CAPS)


@pytest.mark.parametrize("bc", [inputs.PERIODIC, inputs.TRANSMISSIVE])
def test_odd_number_of_halfsteps_ends_on_half_stage(bc):
    pr = _problem(inputs.BURGERS, 3, 300, bc)
    dts = np.full(7, 0.2 * pr.dx / 1.5)
    q, _, t, parity = gpu_run(pr, None, None, dts=dts)
    ref, _, rparity = oracle_run(pr, dts)
    assert parity == 1 == rparity
    assert q.shape[0] == inputs.num_cells(300, bc, 1)
    assert scaled_error(q, ref) <= TOL64


def test_graph_and_direct_launches_identical():
    pr = _problem(inputs.EULER, 3, 3000, inputs.TRANSMISSIVE)
    q1, d1, _, _ = gpu_run(pr, 70, 0.2, graph_chunk=32)
    q2, d2, _, _ = gpu_run(pr, 70, 0.2, graph_chunk=0)
    assert np.array_equal(d1, d2)
    assert np.array_equal(q1, q2)


def test_checkpoint_resume_bitwise():
    # P = 2: the exported u_kx = k! e_k round-trips exactly (k! in {1, 1, 2}).
    pr = _problem(inputs.BURGERS, 2, 1000, inputs.PERIODIC)
    q_full, dts, _, _ = gpu_run(pr, 40, 0.3)
    q_half, d_half, _, _ = gpu_run(pr, 20, 0.3)
    pr2 = inputs.Problem(pr.system, pr.N, pr.P, pr.x_l, pr.x_r, pr.bc, q_half)
    q_res, d_res, _, _ = gpu_run(pr2, 20, 0.3)
    assert np.array_equal(np.concatenate([d_half, d_res]), dts)
    assert np.array_equal(q_res, q_full)


def test_conservation_on_gpu():
    pr = _problem(inputs.EULER, 3, 4096, inputs.PERIODIC)
    q, _, _, _ = gpu_run(pr, 200, 0.25)
    w = np.array([1.0, 0.0, 1.0 / 24.0, 0.0])       # cell average of the P = 3 polynomial
    tot0 = (pr.q0 @ w).sum(axis=0)
    tot = (q @ w).sum(axis=0)
    np.testing.assert_allclose(tot, tot0, rtol=1e-12)


def test_error_paths():
    pr = inputs.euler_riemann_seeded(256, 2)
    bad = pr.q0.copy()
    bad[10, 0, 0] = -1.0
    s = wcc.Solver(pr.system, pr.N, pr.P, (0.0, 1.0), pr.bc)
    with pytest.raises(wcc.WCCError) as ei:
        s.step(1, 0.2)
    assert ei.value.code == -2                           # before set_initial
    with pytest.raises(wcc.WCCError) as ei:
        s.set_initial(bad)
    assert ei.value.code == -6                           # positivity
    bad[10, 0, 0] = float("nan")
    with pytest.raises(wcc.WCCError) as ei:
        s.set_initial(bad)
    assert ei.value.code in (-5, -6)
    with pytest.raises(wcc.WCCError) as ei:
        s.set_initial(pr.q0[:-1])
    assert ei.value.code == -1                           # wrong count
    with pytest.raises(wcc.WCCError) as ei:
        s.step(1, -0.5)
    assert ei.value.code in (-1, -2)
    s.set_initial(pr.q0)                                  # recovers
    s.step(4, 0.2)
    s.synchronize()
    s.close()


def test_full_size_euler_sampled_windows():
    # The bench workload: Euler, N = 2^22 on [0, 1], P = 3, transmissive,
    # seeded Riemann data, CFL 0.2, in the bench's launch configuration
    # (graph chunks of 32).  After k half-steps a cell depends only on the
    # initial data within k/2 + 1 cells, so the oracle recomputes windows of
    # the grid one by one.
    N, P, k = 1 << 22, 3, 64
    pr = inputs.euler_riemann_seeded(N, P)
    q, dts, _, parity = gpu_run(pr, k, 0.2)
    assert parity == 0 and len(dts) == k
    rng = np.random.default_rng(5)
    centres = [N // 2, N // 2 - 40, N // 2 + 40, 3, N - 3] + list(rng.integers(100, N - 100, 3))
    half = k // 2 + 8
    law = law_of(pr)
    reps = []
    for c in centres:
        lo, hi = max(0, c - 2 * half), min(N + 1, c + 2 * half)

        def run(q0):
            s = oracle.Solver(law, q0, pr.dx)
            s.step_dt(dts)
            return s.q

        ref = run(pr.q0[lo:hi])
        spread = oracle_spread(run, pr.q0[lo:hi], ref)
        # compare cells at least `half` away from an artificial window edge
        a = lo if lo == 0 else lo + half
        b = hi if hi == N + 1 else hi - half
        reps.append(parity_report(q[a:b], ref[a - lo:b - lo], spread[a - lo:b - lo]))
        assert reps[-1].violation <= 1.0, (c, reps[-1])
    assert_parity(merge(reps), **FULL_SIZE_CAPS)
