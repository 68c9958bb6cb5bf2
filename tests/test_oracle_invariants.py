"""Invariant pins for the oracle: conservation (Sec. 2.1 remark, Sec. 2.2),
exactness on polynomial data, reduction to the staggered Lax-Friedrichs
scheme at P = 0, limiter properties (Eq. 1DLimitedPolynomial) and mirror
symmetry."""
import math

import numpy as np
import pytest

import oracle
from paper_2104_04347_gb300 import inputs


def cell_average(q):
    """Cell average of the polynomial of Eq. 1DPolynomial_Space, q [..., P+1]."""
    P = q.shape[-1] - 1
    w = np.array([(1 + (-1) ** k) / (math.factorial(k + 1) * 2 ** (k + 1)) for k in range(P + 1)])
    return q @ w


@pytest.mark.parametrize("P", [0, 1, 2, 3, 4])
@pytest.mark.parametrize("limiter", [False, True])
def test_conservation_periodic_burgers(P, limiter):
    pr = inputs.burgers_fourier(128, P)
    law = oracle.make_law(oracle.BURGERS, P, limiter=limiter)
    s = oracle.Solver(law, pr.q0, pr.dx)
    total0 = cell_average(s.q[:, 0, :]).sum()
    ts = inputs.shock_time(inputs.burgers_fourier_data())
    while s.t < 2 * ts:           # well past the shock
        s.step_cfl(2, 0.2)
        total = cell_average(s.q[:, 0, :]).sum()
        assert abs(total - total0) < 1e-12 * abs(total0) * 10
    assert np.all(np.isfinite(s.q))


@pytest.mark.parametrize("P", [1, 2, 3])
def test_conservation_periodic_euler(P):
    pr = inputs.euler_density_wave(64, P)
    law = oracle.make_law(oracle.EULER, P, limiter=True)
    s = oracle.Solver(law, pr.q0, pr.dx)
    tot0 = cell_average(s.q).sum(axis=0)
    s.step_cfl(40, 0.2)
    tot = cell_average(s.q).sum(axis=0)
    np.testing.assert_allclose(tot, tot0, rtol=1e-13)


@pytest.mark.parametrize("P", [1, 2, 3, 4])
def test_polynomial_data_advected_exactly(P):
    # u0 of degree P is translated exactly by the linear scheme (CK and the
    # time / space Taylor series are exact); check interior cells.
    rng = np.random.default_rng(P)
    coeffs = rng.uniform(-1, 1, P + 1)
    N = 40
    a = 0.8
    pr = inputs.advection_polynomial(N, P, coeffs)
    law = oracle.make_law(oracle.ADVECTION, P, limiter=False, bc=oracle.TRANSMISSIVE, a=a)
    s = oracle.Solver(law, pr.q0, pr.dx)
    nsteps = 6
    s.step_cfl(nsteps, 0.25)
    assert s.parity == 0
    poly = np.polynomial.Polynomial(coeffs)
    x = inputs.centres(N, 0.0, 1.0, inputs.TRANSMISSIVE)
    for k in range(P + 1):
        exact = poly.deriv(k)(x - a * s.t) * pr.dx ** k if k <= P else 0
        np.testing.assert_allclose(s.q[nsteps:-nsteps, 0, k], exact[nsteps:-nsteps],
                                   rtol=0, atol=1e-12)


def test_p0_is_staggered_lax_friedrichs():
    rng = np.random.default_rng(3)
    u = rng.uniform(-1, 1, size=(50, 1, 1))
    lam = 0.37
    law = oracle.make_law(oracle.BURGERS, 0, limiter=False)
    new = oracle.halfstep(law, 0, u, lam)
    uL, uR = u[:, 0, 0], np.roll(u[:, 0, 0], -1)
    np.testing.assert_allclose(new[:, 0, 0], 0.5 * (uL + uR) + lam * (0.5 * uL ** 2 - 0.5 * uR ** 2),
                               rtol=0, atol=1e-15)
    new1 = oracle.halfstep(law, 1, u, lam)
    uL, uR = np.roll(u[:, 0, 0], 1), u[:, 0, 0]
    np.testing.assert_allclose(new1[:, 0, 0], 0.5 * (uL + uR) + lam * (0.5 * uL ** 2 - 0.5 * uR ** 2),
                               rtol=0, atol=1e-15)


@pytest.mark.parametrize("system", [oracle.BURGERS, oracle.EULER])
@pytest.mark.parametrize("P", [1, 2, 3, 4])
def test_limiter_weights_and_mean(system, P):
    law = oracle.make_law(system, P, limiter=True)
    nv = oracle.nvars(system)
    rng = np.random.default_rng(7 * P + system)
    for trial in range(30):
        if system == oracle.EULER:
            def state():
                base = np.array([rng.uniform(0.5, 1.5), rng.uniform(-0.5, 0.5), rng.uniform(2.0, 4.0)])
                q = np.zeros((3, P + 1))
                q[:, 0] = base
                q[:, 1:] = rng.uniform(-0.3, 0.3, size=(3, P)) * (trial % 3)
                return q
            qL, qR = state(), state()
        else:
            qL = rng.uniform(-1, 1, size=(1, P + 1))
            qR = rng.uniform(-1, 1, size=(1, P + 1))
        out, cand, w, ub = oracle.new_cell(law, qL, qR, 0.15, diagnostics=True)
        np.testing.assert_allclose(w.sum(axis=1), 1.0, rtol=0, atol=1e-15)
        assert np.all(w >= 0)
        # the limited polynomial keeps the cell average (Sec. 2.2)
        np.testing.assert_allclose(cell_average(out), ub, rtol=1e-14, atol=1e-14)
        # the unlimited polynomial u_0 also has cell average ubar (Eq. 1DCalU)
        np.testing.assert_allclose(cell_average(cand[0]), ub, rtol=1e-14, atol=1e-14)


@pytest.mark.parametrize("P", [1, 2, 3, 4])
def test_flat_data_unchanged(P):
    for system, q in ((oracle.BURGERS, np.array([[0.7] + [0.0] * P])),
                      (oracle.EULER, np.array([[1.2] + [0.0] * P, [0.3] + [0.0] * P, [2.5] + [0.0] * P]))):
        law = oracle.make_law(system, P, limiter=True)
        out, _, w, _ = oracle.new_cell(law, q, q, 0.2, diagnostics=True)
        # a uniform state is a steady solution
        np.testing.assert_allclose(out, q, rtol=1e-15, atol=1e-15)
        if P >= 2:
            assert np.all(w[:, 0] == 1.0)


def test_limiter_inactive_on_smooth_data_p3():
    pr = inputs.advection_sine(200, 3)
    law = oracle.make_law(oracle.ADVECTION, 3, limiter=True)
    _, w = oracle.halfstep(law, 0, pr.q0, 0.25, weights=True)
    assert np.max(w[:, 0, 1] + w[:, 0, 2]) < 1e-20


def test_limiter_active_at_jump():
    q = np.zeros((40, 1, 4))
    q[20:, 0, 0] = 1.0
    law = oracle.make_law(oracle.ADVECTION, 3, limiter=True, bc=oracle.TRANSMISSIVE)
    s = oracle.Solver(law, q, 0.025)
    s.step_cfl(4, 0.25)
    _, w = oracle.halfstep(law, s.parity, s.q, 0.25, weights=True)
    assert np.max(w[:, 0, 1] + w[:, 0, 2]) > 0.5


def _mirror(q, sign_vars):
    """Mirror x -> -x: reverse the cells, flip odd derivatives, and apply the
    symmetry's sign to each variable."""
    P = q.shape[-1] - 1
    kflip = np.array([(-1.0) ** k for k in range(P + 1)])
    return q[::-1] * kflip[None, None, :] * np.asarray(sign_vars)[None, :, None]


@pytest.mark.parametrize("P", [1, 2, 3, 4])
@pytest.mark.parametrize("system", [oracle.BURGERS, oracle.EULER])
def test_mirror_symmetry(P, system):
    # Burgers: u(x,t) -> -u(-x,t); Euler: (rho, m, E)(x,t) -> (rho, -m, E)(-x,t).
    # On a transmissive grid the integer stage (N+1 cells) maps to itself
    # reversed, and so does the half stage.
    if system == oracle.BURGERS:
        pr = inputs.burgers_fourier(64, P)
        q = np.concatenate([pr.q0, pr.q0[:1]])     # 65 cells, transmissive grid
        signs = [-1.0]
    else:
        pr = inputs.euler_riemann(64, P, (1.0, 0.2, 1.0), (0.3, -0.4, 0.2))
        q = pr.q0
        signs = [1.0, -1.0, 1.0]
    law = oracle.make_law(system, P, limiter=True, bc=oracle.TRANSMISSIVE)
    a = oracle.Solver(law, q, 1.0 / 64)
    b = oracle.Solver(law, _mirror(q, signs), 1.0 / 64)
    for _ in range(5):
        a.step_cfl(1, 0.2)
        b.step_dt([a.dts[-1]])
        np.testing.assert_allclose(_mirror(a.q, signs), b.q, rtol=1e-11, atol=1e-12)
