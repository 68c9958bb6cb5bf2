"""Pins for the oracle on Burgers' equation against the exact solution by
characteristics before the shock, and bounds after it."""
import math

import numpy as np
import pytest

import oracle
from oracle import exact
from paper_2104_04347_gb300 import inputs


@pytest.mark.parametrize("P", [1, 2, 3, 4])
def test_preshock_order(P):
    # the linear scheme (limiter off) converges at order P + 1 before the shock
    data = inputs.burgers_fourier_data()
    ts = inputs.shock_time(data)
    t_end = 0.5 * ts
    errs = []
    for N in (128, 256, 512):
        pr = inputs.burgers_fourier(N, P)
        law = oracle.make_law(oracle.BURGERS, P, limiter=False)
        s = oracle.Solver(law, pr.q0, pr.dx)
        amax = 0.5 + float(np.abs(data.amps).sum())          # bound on |u|
        s.step_dt(oracle.constant_speed_dts(t_end, 0.2 * pr.dx / amax))
        x = inputs.centres(N, 0.0, 2 * math.pi, inputs.PERIODIC)
        ue = exact.burgers_characteristics(lambda z: data.derivative(z, 0),
                                           lambda z: data.derivative(z, 1), x, s.t)
        errs.append(np.mean(np.abs(s.q[:, 0, 0] - ue)))
    order = math.log2(errs[1] / errs[2])
    assert order > P + 1 - 0.35, (errs, order)


@pytest.mark.parametrize("P", [1, 2, 3, 4])
def test_postshock_bounded(P):
    data = inputs.burgers_fourier_data()
    ts = inputs.shock_time(data)
    pr = inputs.burgers_fourier(256, P)
    law = oracle.make_law(oracle.BURGERS, P, limiter=True)
    s = oracle.Solver(law, pr.q0, pr.dx)
    while s.t < 2 * ts:
        s.step_cfl(2, {1: 0.4, 2: 0.3, 3: 0.25, 4: 0.2}[P])
    u0 = pr.q0[:, 0, 0]
    u = s.q[:, 0, 0]
    assert np.all(np.isfinite(u))
    span = u0.max() - u0.min()
    assert u.min() > u0.min() - 0.1 * span and u.max() < u0.max() + 0.1 * span
