"""Pins of the oracle's CFL bound (1D ``max_speed``, 2D ``max_speeds2d``)
against characteristic speeds written out by hand.

The paper uses a_max through the CFL number nu = a_max dt / dx (Table 1
caption; the CFL numbers of Sec. 5) but does not say where a_max is taken.
The reading here: the largest spectral radius of the flux Jacobian over the
cells of the stage being advanced, evaluated at each cell's centre point
value u_0x (the k = 0 DOF), not at its cell average.  The speeds are |a|
(advection), |u| (Burgers) and |u| + c with c = sqrt(gamma p / rho) (Euler);
in 2D |u| + c along x, |v| + c along y, and the step rate s_x/dx + s_y/dy.

Every state below carries second derivatives, so that the cell average
differs from the centre value and a bound taken from averages fails; the
Euler states are chosen so that max(|u|, c) and |u| + c pick different
values."""
import math

import numpy as np
import pytest

import oracle

GAMMA = 1.4


def euler_point(rho, u, p, P, u2=(0.0, 0.0, 0.0)):
    """One cell of 1D Euler DOFs [var][k] whose centre point values are the
    conserved form of (rho, u, p); u2 adds second derivatives u_2x."""
    q = np.zeros((3, P + 1))
    q[0, 0] = rho
    q[1, 0] = rho * u
    q[2, 0] = p / (GAMMA - 1.0) + 0.5 * rho * u * u
    if P >= 2:
        q[:, 2] = u2
    return q


def speed(rho, u, p):
    return abs(u) + math.sqrt(GAMMA * p / rho)


@pytest.mark.parametrize("P", [1, 3])
def test_advection_speed_is_abs_a(P):
    law = oracle.make_law(oracle.ADVECTION, P, a=-1.7)
    q = np.zeros((5, 1, P + 1))
    q[:, 0, 0] = [3.0, -4.0, 0.5, 0.0, 9.0]  # the data does not enter
    assert oracle.max_speed(law, q) == 1.7


def test_burgers_speed_is_abs_centre_value():
    P = 3
    law = oracle.make_law(oracle.BURGERS, P)
    q = np.zeros((3, 1, P + 1))
    q[:, 0, 0] = [0.3, -0.9, 0.5]
    q[:, 0, 1] = [2.0, 0.05, -1.0]
    # cell averages u_0x + u_2x / 24: 0.3 + 0.1, -0.9 + 0.2, 0.5 + 0.5 -> max 1.0
    q[:, 0, 2] = [2.4, 4.8, 12.0]
    assert oracle.max_speed(law, q) == pytest.approx(0.9, rel=0, abs=0)


@pytest.mark.parametrize("P", [2, 3])
def test_euler_speed_is_abs_u_plus_c_at_centre(P):
    law = oracle.make_law(oracle.EULER, P, gamma=GAMMA)
    states = [(1.25, -0.8, 0.6), (0.5, 0.3, 1.0), (2.0, 1.1, 0.2)]
    q = np.stack([euler_point(*s, P, u2=(0.5, -0.4, 3.0)) for s in states])
    want = max(speed(*s) for s in states)
    got = oracle.max_speed(law, q)
    assert got == pytest.approx(want, rel=1e-14)
    # the second state wins: |u| + c = 0.3 + sqrt(2.8); max(|u|, c) would give
    # sqrt(2.8) (state 2) and a speed from the cell averages another value
    assert got == pytest.approx(0.3 + math.sqrt(2.8), rel=1e-14)
    avg = q[:, :, 0] + q[:, :, 2] / 24.0
    rho, m, E = avg[:, 0], avg[:, 1], avg[:, 2]
    u = m / rho
    p = (GAMMA - 1.0) * (E - 0.5 * rho * u * u)
    assert abs(np.max(np.abs(u) + np.sqrt(GAMMA * p / rho)) - got) > 1e-3


def test_euler_speed_nan_wins():
    law = oracle.make_law(oracle.EULER, 1, gamma=GAMMA)
    q = np.stack([euler_point(1.0, 0.0, 1.0, 1), euler_point(1.0, 0.0, -1.0, 1)])
    assert math.isnan(oracle.max_speed(law, q))  # negative pressure: c is NaN


def _cell2d(nv, P, c00):
    nq = oracle.nq2d(P)
    c = np.zeros((nv, nq))
    c[:, 0] = c00
    return c


def test_2d_euler_speeds_and_rate():
    P = 2
    nq = oracle.nq2d(P)
    law = oracle.make_law2d(oracle.EULER, P, gamma=GAMMA)
    prim = [(1.0, 0.9, -0.1, 0.5), (0.8, -0.2, 0.7, 1.2), (1.5, 0.1, 0.1, 0.3)]
    q = np.zeros((1, 3, 4, nq))
    for j, (rho, u, v, p) in enumerate(prim):
        E = p / (GAMMA - 1.0) + 0.5 * rho * (u * u + v * v)
        q[0, j] = _cell2d(4, P, [rho, rho * u, rho * v, E])
        q[0, j, :, oracle.idx2d(2, 0)] = [0.3, -0.2, 0.1, 2.0]  # u_2x: averages differ
        q[0, j, :, oracle.idx2d(0, 2)] = [-0.1, 0.4, 0.2, -1.5]
    dx, dy = 0.01, 0.04
    sx = [abs(u) + math.sqrt(GAMMA * p / r) for r, u, v, p in prim]
    sy = [abs(v) + math.sqrt(GAMMA * p / r) for r, u, v, p in prim]
    rate = [a / dx + b / dy for a, b in zip(sx, sy)]
    got = oracle.max_speeds2d(law, q, dx, dy)
    assert got[0] == pytest.approx(max(sx), rel=1e-14)
    assert got[1] == pytest.approx(max(sy), rel=1e-14)
    assert got[2] == pytest.approx(max(rate), rel=1e-14)
    # the rate is a maximum over cells of the sum, not the sum of the maxima
    assert max(rate) < max(sx) / dx + max(sy) / dy - 1.0
    assert oracle.cfl_dt2d(law, q, dx, dy, 0.3) == pytest.approx(0.3 / max(rate), rel=1e-14)


def test_2d_scalar_speeds():
    P = 1
    nq = oracle.nq2d(P)
    q = np.zeros((2, 2, 1, nq))
    q[:, :, 0, 0] = [[0.2, -1.3], [0.4, 0.9]]
    q[:, :, 0, oracle.idx2d(1, 0)] = 5.0
    lb = oracle.make_law2d(oracle.BURGERS, P)
    got = oracle.max_speeds2d(lb, q, 0.1, 0.2)
    assert got[0] == got[1] == pytest.approx(1.3, rel=0, abs=0)
    assert got[2] == pytest.approx(1.3 / 0.1 + 1.3 / 0.2, rel=1e-15)
    la = oracle.make_law2d(oracle.ADVECTION, P, ax=-0.5, ay=2.0)
    got = oracle.max_speeds2d(la, q, 0.1, 0.2)
    assert got[:2] == (0.5, 2.0)
    assert got[2] == pytest.approx(0.5 / 0.1 + 2.0 / 0.2, rel=1e-15)
