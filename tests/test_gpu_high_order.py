"""GPU parity of the FP64 path at P = 5 and 6 (the oracle pins these degrees in
tests/test_oracle_high_order.py).

* One half-step from the same state, both parities, every system, both
  boundaries, limiter on and off: within 1e-11 of each variable's scale, on
  meshes of several 127-cell tiles and a ragged tail.
* The Euler density wave to t = 1 at the CFL numbers of the stability scan
  (0.16, 0.14): the GPU's errors against the exact solution equal the
  oracle's on the same half-step sizes, and converge at order P + 1.
* The FP32 variants stop at P = 4.
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


@pytest.mark.parametrize("precision", [wcc.FP32_MIXED, wcc.FP32])
def test_fp32_variants_stop_at_p4(precision):
    with pytest.raises(wcc.WCCError) as ei:
        wcc.Solver(inputs.EULER, 256, 5, (0.0, 1.0), inputs.TRANSMISSIVE, precision=precision)
    assert ei.value.code == -1
