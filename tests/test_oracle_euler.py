"""Pins for the oracle's Euler path (Sec. 4, Sec. 5.2): eigenvector
identities, the exact Riemann solver used as a reference, and the oracle's
WCC solution against exact solutions."""
import math

import numpy as np
import pytest

import oracle
from oracle import exact
from paper_2104_04347_gb300 import inputs

G = 1.4


def euler_flux(U, gamma=G):
    rho, m, E = U
    u = m / rho
    p = (gamma - 1) * (E - 0.5 * m * u)
    return np.array([m, m * u + p, (E + p) * u])


def jacobian_complex_step(U, gamma=G, h=1e-30):
    J = np.zeros((3, 3))
    for j in range(3):
        Uc = np.array(U, dtype=complex)
        Uc[j] += 1j * h
        J[:, j] = np.imag(euler_flux(Uc, gamma)) / h
    return J


def test_eigenvectors_diagonalise_jacobian():
    rng = np.random.default_rng(0)
    for _ in range(50):
        rho, u, p = rng.uniform(0.1, 2), rng.uniform(-2, 2), rng.uniform(0.1, 2)
        U = inputs.primitive_to_conserved(rho, u, p)
        R, L = oracle.euler_eigenvectors(G, U)
        np.testing.assert_allclose(L @ R, np.eye(3), atol=1e-13)
        A = jacobian_complex_step(U)
        c = math.sqrt(G * p / rho)
        np.testing.assert_allclose(L @ A @ R, np.diag([u - c, u, u + c]), atol=1e-12 * (1 + abs(u) + c) ** 3)


def test_riemann_sod_star_state():
    # Star state of Sod's problem from the textbook (Toro, Table 4.3 test 1).
    p, u = exact.riemann_star((1.0, 0.0, 1.0), (0.125, 0.0, 0.1))
    assert abs(p - 0.30313) < 5e-6 and abs(u - 0.92745) < 5e-6


def _integral_check(left, right, t=0.2):
    # Conservation of the exact solution: int (U(x,t) - U(x,0)) dx = t (F(W_L) - F(W_R))
    x = np.linspace(-1.0, 1.0, 400001)
    xm = 0.5 * (x[1:] + x[:-1])
    rho, u, p = exact.riemann_sample(left, right, xm / t)
    U = inputs.primitive_to_conserved(rho, u, p)
    U0 = np.where((xm < 0)[:, None], inputs.primitive_to_conserved(*left)[None, :],
                  inputs.primitive_to_conserved(*right)[None, :])
    lhs = ((U - U0) * (x[1] - x[0])).sum(axis=0)
    rhs = t * (euler_flux(inputs.primitive_to_conserved(*left))
               - euler_flux(inputs.primitive_to_conserved(*right)))
    np.testing.assert_allclose(lhs, rhs, atol=2e-5)


def test_riemann_conservation_sod_and_seeded():
    _integral_check((1.0, 0.0, 1.0), (0.125, 0.0, 0.1))
    _integral_check(*inputs.riemann_states(2104043471))
    _integral_check((0.2, -0.4, 0.15), (0.9, 0.45, 0.8))     # two rarefactions
    _integral_check((0.9, 0.5, 0.8), (0.2, -0.5, 0.1))      # two shocks


def test_riemann_rankine_hugoniot():
    left, right = (1.0, 0.0, 1.0), (0.125, 0.0, 0.1)
    ps, us = exact.riemann_star(left, right)
    # right shock speed from mass conservation, then momentum / energy must match
    rr, ur, pr = right
    g1 = (G - 1) / (G + 1)
    rs = rr * (ps / pr + g1) / (g1 * ps / pr + 1)
    S = (rs * us - rr * ur) / (rs - rr)
    Ua = inputs.primitive_to_conserved(rs, us, ps)
    Ub = inputs.primitive_to_conserved(rr, ur, pr)
    np.testing.assert_allclose(euler_flux(Ua) - euler_flux(Ub), S * (Ua - Ub), atol=1e-12)


def _density_l1(s, N, x_l, x_r, left, right, x0):
    x = inputs.centres(N, x_l, x_r, inputs.TRANSMISSIVE, s.parity)
    rho, _, _ = exact.riemann_sample(left, right, (x - x0) / s.t)
    return np.mean(np.abs(s.q[:, 0, 0] - rho))


@pytest.mark.parametrize("P", [1, 2, 3])
def test_sod_converges_to_exact(P):
    errs = []
    for N in (100, 200, 400):
        pr = inputs.sod(N, P)
        law = oracle.make_law(oracle.EULER, P, limiter=True, bc=oracle.TRANSMISSIVE)
        s = oracle.Solver(law, pr.q0, pr.dx)
        while s.t < 0.4 - 1e-12 or s.parity:
            s.step_cfl(1, 0.2)
        assert np.all(np.isfinite(s.q))
        errs.append(_density_l1(s, N, 0.0, 2.0, (1.0, 0.0, 1.0), (0.125, 0.0, 0.1), 1.0))
    assert errs[0] < 0.03
    assert errs[1] < errs[0] and errs[2] < errs[1]
    assert math.log2(errs[0] / errs[2]) / 2 > 0.5     # ~first order at discontinuities


def test_seeded_riemann_converges_to_exact():
    left, right = inputs.riemann_states(2104043471)
    errs = []
    for N in (128, 512):
        pr = inputs.euler_riemann_seeded(N, 3)
        law = oracle.make_law(oracle.EULER, 3, limiter=True, bc=oracle.TRANSMISSIVE)
        s = oracle.Solver(law, pr.q0, pr.dx)
        while s.t < 0.15 or s.parity:
            s.step_cfl(1, 0.2)
        errs.append(_density_l1(s, N, 0.0, 1.0, left, right, 0.5))
    assert errs[1] < 0.5 * errs[0]


def _density_wave_error(P, N, limiter):
    nu = {1: 0.4, 2: 0.3, 3: 0.25, 4: 0.2}[P]
    amax = 1.0 + math.sqrt(G / 0.8)
    pr = inputs.euler_density_wave(N, P)
    law = oracle.make_law(oracle.EULER, P, limiter=limiter)
    s = oracle.Solver(law, pr.q0, pr.dx)
    s.step_dt(oracle.constant_speed_dts(0.5, nu * pr.dx / amax))
    x = inputs.centres(N, 0.0, 1.0, inputs.PERIODIC)
    return np.mean(np.abs(s.q[:, 0, 0] - (1 + 0.2 * np.sin(2 * math.pi * (x - s.t)))))


@pytest.mark.parametrize("P", [1, 2, 3, 4])
def test_density_wave_order(P):
    # Smooth Euler flow rho = 1 + 0.2 sin(2 pi (x - t)), u = 1, p = 1; the
    # linear scheme (limiter off) converges at order P + 1.
    sizes = (16, 32, 64) if P >= 3 else (32, 64, 128)
    errs = [_density_wave_error(P, N, False) for N in sizes]
    order = math.log2(errs[-2] / errs[-1])
    assert abs(order - (P + 1)) < 0.3, (errs, order)


def test_density_wave_limiter_harmless_p3():
    # At P = 3 the limiter leaves the smooth solution alone once the wave is
    # resolved (Sec. 2.2: w_1, w_2 vanish at a high rate in smooth regions).
    for N in (64, 128):
        on, off = _density_wave_error(3, N, True), _density_wave_error(3, N, False)
        assert abs(on - off) < 1e-3 * off
