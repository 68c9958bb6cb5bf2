"""GPU parity of the 2D path on discontinuous data: the two 2D Riemann
problems of Sec. 5.3 (four shocks; four contacts) on [-1, 1]^2 with
transmissive boundaries, P = 1..3, limiter on, where the rotated
characteristic limiter is active.

* FP64, every half-step: the GPU's CFL half-step from its own state against
  the oracle's half-step from the same state, per entry within
  max(1e-11 x scale, 50 x the oracle's own spread under 4e-16 input noise)
  (the limiter's weights are ill-conditioned at a discontinuity, as in 1D);
  the GPU's dt is the oracle's CFL step of that state.
* FP32 and FP32-mixed: the trajectory's L1 against the oracle replaying the
  same half-step sizes, within max(1e-5, 50 x the oracle's L1 spread under
  1e-7 noise).
"""
import numpy as np
import pytest

import oracle
from paper_2104_04347_gb300 import inputs, wcc

pytestmark = pytest.mark.gpu

CFL = {1: 0.4, 2: 0.3, 3: 0.25}
N, STEPS = 48, 16


def _solver(pr, precision=wcc.FP64):
    return wcc.Solver2D(pr.system, pr.nx, pr.ny, pr.P, (pr.x_l, pr.x_r, pr.y_l, pr.y_r), pr.bc, precision=precision)


def _law(P):
    return oracle.make_law2d(oracle.EULER, P, limiter=True, bc=oracle.TRANSMISSIVE)


def _scale(q):
    return np.maximum(np.max(np.abs(q[:, :, :, 0]), axis=(0, 1)), 1e-300)[None, None, :, None]


@pytest.mark.parametrize("P", [1, 2, 3])
@pytest.mark.parametrize("config", [1, 2])
def test_every_halfstep_fp64(config, P):
    pr = inputs.riemann2d(N, P, config)
    law = _law(P)
    rng = np.random.default_rng(config * 10 + P)
    worst = 0.0
    with _solver(pr) as s:
        s.set_initial(pr.q0)
        prev = pr.q0
        for k in range(STEPS):
            s.step(1, CFL[P])
            got = s.get_dofs()
            dt = s.dt_history()[-1]
            assert abs(dt - oracle.cfl_dt2d(law, prev, pr.dx, pr.dy, CFL[P])) <= 1e-12 * dt
            lx, ly = dt / pr.dx, dt / pr.dy
            want = oracle.halfstep2d(law, k % 2, prev, lx, ly)
            spread = np.zeros_like(want)
            for _ in range(3):
                pert = prev * (1.0 + 4e-16 * rng.standard_normal(prev.shape))
                spread = np.maximum(spread, np.abs(oracle.halfstep2d(law, k % 2, pert, lx, ly) - want))
            bound = np.maximum(1e-11 * _scale(want), 50.0 * spread)
            worst = max(worst, float(np.max(np.abs(got - want) / bound)))
            prev = got
    assert worst <= 1.0, worst


@pytest.mark.parametrize("precision", [wcc.FP32, wcc.FP32_MIXED])
@pytest.mark.parametrize("P", [1, 2, 3])
@pytest.mark.parametrize("config", [1, 2])
def test_trajectory_fp32(config, P, precision):
    pr = inputs.riemann2d(N, P, config)
    law = _law(P)
    with _solver(pr, precision) as s:
        s.set_initial(pr.q0)
        s.step(STEPS, CFL[P])
        got = s.get_dofs()
        dts = s.dt_history()
    ref = oracle.Solver2D(law, pr.q0, pr.dx, pr.dy)
    ref.step_dt(dts)
    sc = _scale(ref.q)[0, 0, :, 0]

    def l1(a):
        return float(np.max(np.mean(np.abs(a[:, :, :, 0] - ref.q[:, :, :, 0]), axis=(0, 1)) / sc))

    rng = np.random.default_rng(P)
    spread = 0.0
    for _ in range(3):
        r2 = oracle.Solver2D(law, pr.q0 * (1.0 + 1e-7 * rng.standard_normal(pr.q0.shape)), pr.dx, pr.dy)
        r2.step_dt(dts)
        spread = max(spread, l1(r2.q))
    assert l1(got) <= max(1e-5, 50.0 * spread), (l1(got), spread)
