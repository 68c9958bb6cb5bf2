"""GPU parity of the FP64 path at P = 5 and 6 (the oracle pins these degrees in
tests/test_oracle_high_order.py).

* One half-step from the same state, both parities, every system, both
  boundaries, limiter on and off: within 1e-11 of each variable's scale, on
  meshes of several 127-cell tiles and a ragged tail.
* The Euler density wave to t = 1 at the CFL numbers of the stability scan
  (0.16, 0.14): the GPU's errors against the exact solution equal the
  oracle's on the same half-step sizes, and converge at order P + 1.
* FP32-mixed at P = 5, 6 (and two half-steps per launch): L1 within 1e-6
  of the oracle replaying the same half-step sizes, on smooth data and on
  Riemann data, both boundaries; the summed cell averages conserved; on the
  density wave the error follows the oracle's down to the FP32 floor.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2104_04347_gb300 import inputs, wcc
from tests.gpu_common import gpu_solver, scales

pytestmark = pytest.mark.gpu

CFL = {5: 0.16, 6: 0.14}  # 0.8 of the von Neumann limits (tests/golden/stability_limits.txt)


def _problem(system, N, P, bc):
    if system == inputs.EULER:
        if bc == inputs.PERIODIC:
            return inputs.euler_density_wave(N, P)
        return inputs.euler_riemann_seeded(N, P)
    if system == inputs.BURGERS:
        pr = inputs.burgers_fourier(N, P)
    else:
        pr = inputs.advection_sine(N, P)
    if bc == inputs.TRANSMISSIVE:
        pr = inputs.Problem(pr.system, N, P, pr.x_l, pr.x_r, inputs.TRANSMISSIVE,
                            np.concatenate([pr.q0, pr.q0[:1]], axis=0), pr.name)
    return pr


@pytest.mark.parametrize("bc", [inputs.PERIODIC, inputs.TRANSMISSIVE])
@pytest.mark.parametrize("system", [inputs.ADVECTION, inputs.BURGERS, inputs.EULER])
@pytest.mark.parametrize("P", [5, 6])
def test_one_halfstep_each_parity(P, system, bc):
    pr = _problem(system, 300, P, bc)
    for limiter in (False, True):
        law = oracle.make_law(pr.system, P, limiter=limiter, bc=pr.bc)
        with gpu_solver(pr, limiter=limiter) as s:
            s.set_initial(pr.q0)
            q = pr.q0
            for parity in (0, 1):
                dt = 0.7 * CFL[P] * pr.dx / oracle.max_speed(law, q)
                s.step_dt([dt])
                got = s.get_dofs()
                want = oracle.halfstep(law, parity, q, dt / pr.dx)
                sc = scales(want)
                err = float(np.max(np.abs(got - want) / sc[None, :, None]))
                assert err <= 1e-11, (P, system, bc, limiter, parity, err)
                q = want


@pytest.mark.parametrize("P", [5, 6])
def test_density_wave_converges_like_the_oracle(P):
    amax = 1.0 + math.sqrt(1.4 / 0.8)
    Ns = (16, 24, 32)
    gpu_err, ora_err = [], []
    for N in Ns:
        pr = inputs.euler_density_wave(N, P)
        dts = oracle.constant_speed_dts(1.0, CFL[P] * pr.dx / amax)
        with gpu_solver(pr) as s:
            s.set_initial(pr.q0)
            s.step_dt(dts)
            q = s.get_dofs()
        ref = oracle.Solver(oracle.make_law(oracle.EULER, P), pr.q0, pr.dx)
        ref.step_dt(dts)
        x = inputs.centres(N, 0.0, 1.0, inputs.PERIODIC)
        exact = 1.0 + 0.2 * np.sin(2 * math.pi * (x - 1.0))
        gpu_err.append(float(np.mean(np.abs(q[:, 0, 0] - exact))))
        ora_err.append(float(np.mean(np.abs(ref.q[:, 0, 0] - exact))))
    for g, o in zip(gpu_err, ora_err):
        assert abs(g - o) <= 1e-3 * o + 1e-13, (gpu_err, ora_err)
    order = math.log(gpu_err[-2] / gpu_err[-1]) / math.log(Ns[-1] / Ns[-2])
    assert P + 1 - 0.2 < order < P + 1 + 0.9, (gpu_err, order)


def test_cfl_steps_run_at_p6():
    pr = inputs.euler_riemann_seeded(4096, 6)
    with gpu_solver(pr) as s:
        s.set_initial(pr.q0)
        s.step(64, CFL[6])
        t, steps, parity = s.state()
        dts = s.dt_history()
    law = oracle.make_law(oracle.EULER, 6, limiter=True, bc=oracle.TRANSMISSIVE)
    assert steps == 64 and parity == 0 and abs(dts[0] - CFL[6] * pr.dx / oracle.max_speed(law, pr.q0)) <= 1e-12


def _l1(q, ref):
    return float(np.max(np.mean(np.abs(q[:, :, 0] - ref[:, :, 0]), axis=0) / scales(ref)))


@pytest.mark.parametrize("tb", [1, 2])
@pytest.mark.parametrize("bc", [inputs.PERIODIC, inputs.TRANSMISSIVE])
@pytest.mark.parametrize("system", [inputs.BURGERS, inputs.EULER])
@pytest.mark.parametrize("P", [5, 6])
def test_fp32_mixed_against_the_oracle(P, system, bc, tb):
    pr = _problem(system, 3 * 255 + 41, P, bc)
    with wcc.Solver(pr.system, pr.N, P, (pr.x_l, pr.x_r), pr.bc, precision=wcc.FP32_MIXED, tb_depth=tb) as s:
        s.set_initial(pr.q0)
        s.step(64, CFL[P])
        q = s.get_dofs()
        dts = s.dt_history()
    ref = oracle.Solver(oracle.make_law(pr.system, P, bc=pr.bc), pr.q0, pr.dx)
    ref.step_dt(dts)
    assert np.all(np.isfinite(q))
    assert _l1(q, ref.q) <= 1e-6, (P, system, bc, tb, _l1(q, ref.q))


@pytest.mark.parametrize("P", [5, 6])
def test_fp32_mixed_conserves(P):
    pr = inputs.euler_density_wave(1024, P)
    with wcc.Solver(pr.system, pr.N, P, (pr.x_l, pr.x_r), pr.bc, precision=wcc.FP32_MIXED) as s:
        s.set_initial(pr.q0)
        s.step(200, CFL[P])
        q = s.get_dofs()
    w = np.array([(1 + (-1) ** k) / (math.factorial(k + 1) * 2.0 ** (k + 1)) for k in range(P + 1)])
    tot0, tot = (pr.q0 @ w).sum(axis=0), (q @ w).sum(axis=0)
    assert np.all(np.abs(tot - tot0) <= 1e-12 * np.maximum(np.abs(tot0), 1.0))


@pytest.mark.parametrize("P", [5, 6])
def test_fp32_mixed_density_wave_follows_the_oracle(P):
    # coarse meshes, where the scheme's error is far above FP32 rounding: the
    # same errors as the oracle on the same half-step sizes, to 1 % plus
    # 3e-8, the accumulated rounding floor of FP32-stored derivatives (the
    # FP32-mixed L1 distance to FP64 over a unit-time run is 1e-9 .. 3e-8 for
    # P = 2..6 on meshes of 16..2048 cells)
    amax = 1.0 + math.sqrt(1.4 / 0.8)
    for N in (8, 12, 16):
        pr = inputs.euler_density_wave(N, P)
        dts = oracle.constant_speed_dts(1.0, CFL[P] * pr.dx / amax)
        with wcc.Solver(pr.system, N, P, (0.0, 1.0), pr.bc, precision=wcc.FP32_MIXED) as s:
            s.set_initial(pr.q0)
            s.step_dt(dts)
            q = s.get_dofs()
        ref = oracle.Solver(oracle.make_law(oracle.EULER, P), pr.q0, pr.dx)
        ref.step_dt(dts)
        x = inputs.centres(N, 0.0, 1.0, inputs.PERIODIC)
        exact = 1.0 + 0.2 * np.sin(2 * math.pi * (x - 1.0))
        e, eo = float(np.mean(np.abs(q[:, 0, 0] - exact))), float(np.mean(np.abs(ref.q[:, 0, 0] - exact)))
        assert abs(e - eo) <= 1e-2 * eo + 3e-8, (N, e, eo)
