"""Round trip of the host layout through the FP32-mixed device storage.

wcc_set_initial turns the host's FP64 DOFs q_k = u_kx ([cell][var][k]) into
the device form -- the cell average (Eq. SubEq:1DCellAVG) as a float-float
pair and e_k = q_k / k! in FP32 -- with integer and FP32 arithmetic only;
wcc_get_dofs turns them back.  With no half-step in between, the result must
differ from the input only by that storage:
  * k >= 1: q_k comes back as fl32(q_k / k!) k!, so within about one FP32 ulp
    of q_k;
  * k = 0: the point value is rebuilt as ubar - sum_k e_k / ((k+1) 2^k), so
    it carries the float-float error of ubar plus the FP32 rounding of the
    stored e_k in the correction terms (plain FP32 keeps ubar rounded to
    FP32).
Inputs span many magnitudes, signs and zeros, including values the integer
conversions hand to the hardware path (|q| < 2^-74).
"""
import math

import numpy as np
import pytest

from paper_2104_04347_gb300 import inputs, wcc

pytestmark = pytest.mark.gpu

EPS32 = 2.0 ** -24


def _weights(P):
    """1 / ((k+1)! 2^k) for even k >= 2 (the weight of q_k in the average), else 0."""
    return np.array([1.0 / (math.factorial(k + 1) * 2.0 ** k) if (k >= 2 and k % 2 == 0) else 0.0
                     for k in range(P + 1)])


def _check(q, back, precision):
    P = q.shape[-1] - 1
    fact = np.array([math.factorial(k) for k in range(P + 1)], dtype=np.float64)
    w = _weights(P)
    corr = np.abs(q) @ w  # size of the correction terms, per (cell, var)
    # coefficients k >= 1: one FP32 rounding of q_k / k!, times k! exactly
    err_k = np.abs(back[..., 1:] - q[..., 1:])
    tol_k = 2.0 * EPS32 * np.abs(q[..., 1:]) + 1e-37 * fact[1:]
    assert np.all(err_k <= tol_k), float(np.max(err_k / tol_k))
    # point value: the average's storage error plus the FP32 rounding of e_k
    ubar_scale = np.abs(q[..., 0]) + corr
    avg_eps = 2.0 ** -44 if precision == wcc.FP32_MIXED else 2.0 * EPS32
    tol_0 = avg_eps * ubar_scale + 2.0 * EPS32 * corr + 1e-37
    err_0 = np.abs(back[..., 0] - q[..., 0])
    assert np.all(err_0 <= tol_0), float(np.max(err_0 / tol_0))


def _scalar_dofs(ncells, P, seed):
    rng = np.random.default_rng(seed)
    mag = 10.0 ** rng.uniform(-30.0, 30.0, size=(ncells, 1, P + 1))
    q = mag * rng.choice([-1.0, 1.0], size=mag.shape)
    q[rng.random(q.shape) < 0.1] = 0.0                       # zeros (exact)
    q[rng.random(q.shape) < 0.02] = 1e-300                   # hardware path of the split
    q[rng.random(q.shape) < 0.02] = 0.5                      # exactly representable
    return q


@pytest.mark.parametrize("precision", [wcc.FP32_MIXED, wcc.FP32])
@pytest.mark.parametrize("P", [1, 2, 3, 4])
@pytest.mark.parametrize("system,bc", [(inputs.ADVECTION, inputs.PERIODIC), (inputs.BURGERS, inputs.TRANSMISSIVE)])
def test_scalar_round_trip(system, bc, P, precision):
    N = 1000  # several tiles and a ragged tail
    ncells = inputs.num_cells(N, bc, 0)
    q = _scalar_dofs(ncells, P, seed=100 * P + system)
    with wcc.Solver(system, N, P, (0.0, 1.0), bc, precision=precision) as s:
        s.set_initial(q)
        back = s.get_dofs()
    _check(q, back, precision)
    # zeros come back exactly; so does 0.5 where k! is a power of two (k <= 2;
    # q_k / k! is then exact in FP32) and, for the point value, where every
    # correction term is zero
    k = np.arange(P + 1)
    exact = (q == 0.0) | ((q == 0.5) & (k <= 2))
    exact[..., 0] &= np.all(q[..., 1:] == 0.0, axis=-1)
    assert np.array_equal(back[exact], q[exact])


@pytest.mark.parametrize("precision", [wcc.FP32_MIXED, wcc.FP32])
@pytest.mark.parametrize("P", [1, 2, 3, 4])
def test_euler_round_trip(P, precision):
    N = 777
    ncells = inputs.num_cells(N, inputs.TRANSMISSIVE, 0)
    rng = np.random.default_rng(7 + P)
    rho = rng.uniform(0.1, 1.0, ncells)
    u = rng.uniform(-0.5, 0.5, ncells)
    p = rng.uniform(0.1, 1.0, ncells)
    q = np.zeros((ncells, 3, P + 1))
    q[:, :, 0] = inputs.primitive_to_conserved(rho, u, p)
    q[:, :, 1:] = 1e-2 * rng.standard_normal((ncells, 3, P)) * q[:, :, :1]
    with wcc.Solver(inputs.EULER, N, P, (0.0, 1.0), inputs.TRANSMISSIVE, precision=precision) as s:
        s.set_initial(q)
        back = s.get_dofs()
    _check(q, back, precision)


def test_round_trip_twice_is_stable():
    # a second pass through the storage changes nothing more than the first
    pr = inputs.euler_riemann_seeded(4096, 3)
    with wcc.Solver(pr.system, pr.N, pr.P, (pr.x_l, pr.x_r), pr.bc, precision=wcc.FP32_MIXED) as s:
        s.set_initial(pr.q0)
        once = s.get_dofs()
        s.set_initial(once)
        twice = s.get_dofs()
    assert np.max(np.abs(twice - once)) <= 4.0 * EPS32 * np.max(np.abs(once))
