"""Pins for the oracle's Cauchy-Kovalewski procedure (Eq. 1DCauchy_Kovalewski;
Sec. 4 for the Euler system).

* Burgers closed forms in scaled variables (dx^a dt^b d_x^a d_t^b u):
  U_01 = -lam U U_x, U_11 = -lam (U_x^2 + U U_2x), U_02 = lam^2 (2 U U_x^2 + U^2 U_2x).
* Euler density wave (u = 1, p = 1 constant): the exact solution is a
  translation, so rho_{a,b} = (-lam)^b rho_{a+b}.
* Brute force: an independent symbolic derivation (sympy) that builds the
  time derivatives by differentiating F(U(x, t)) of the truncated time series
  directly, for random polynomial data, P = 1..4."""
import math

import numpy as np
import pytest

import oracle


def test_burgers_closed_forms():
    law = oracle.make_law(oracle.BURGERS, 3)
    rng = np.random.default_rng(1)
    for _ in range(20):
        q = rng.uniform(-1, 1, size=(1, 4))
        lam = rng.uniform(0.05, 0.5)
        U, F = oracle.ck_table(law, q, lam)
        u, ux, uxx = q[0, 0], q[0, 1], q[0, 2]
        assert math.isclose(U[0, 0, 1], -lam * u * ux, rel_tol=1e-14, abs_tol=1e-15)
        assert math.isclose(U[0, 1, 1], -lam * (ux * ux + u * uxx), rel_tol=1e-13, abs_tol=1e-15)
        assert math.isclose(U[0, 0, 2], lam ** 2 * (2 * u * ux * ux + u * u * uxx),
                            rel_tol=1e-13, abs_tol=1e-15)
        # flux table: F = U^2 / 2
        assert math.isclose(F[0, 0, 0], 0.5 * u * u, rel_tol=1e-15)


def test_advection_ck_is_translation():
    law = oracle.make_law(oracle.ADVECTION, 4, a=-0.7)
    q = np.array([[0.3, -1.2, 0.5, 2.0, -0.4]])
    lam = 0.31
    U, _ = oracle.ck_table(law, q, lam)
    for a in range(5):
        for b in range(5 - a):
            assert math.isclose(U[0, a, b], (-(-0.7) * lam) ** b * q[0, a + b], rel_tol=1e-14)


@pytest.mark.parametrize("P", [1, 2, 3, 4])
def test_euler_density_wave_translation(P):
    law = oracle.make_law(oracle.EULER, P)
    rng = np.random.default_rng(P)
    rho = np.concatenate([[1.0], rng.uniform(-0.2, 0.2, size=P)])
    q = np.stack([rho, rho, 0.5 * rho + np.eye(P + 1)[0] / 0.4])   # u = 1, p = 1
    lam = 0.23
    U, _ = oracle.ck_table(law, q, lam)
    for a in range(P + 1):
        for b in range(P + 1 - a):
            exp = (-lam) ** b * rho[a + b]
            assert abs(U[0, a, b] - exp) < 1e-14, (a, b)
            assert abs(U[1, a, b] - exp) < 1e-14, (a, b)
            assert abs(U[2, a, b] - 0.5 * exp - (1 / 0.4 if a == b == 0 else 0.0)) < 1e-13


def _symbolic_ck(system, P, coeffs, lam, gamma=1.4):
    """U[v][a][b] with dx = 1, dt = lam, from sympy differentiation."""
    sp = pytest.importorskip("sympy")
    x, t = sp.symbols("x t")
    nv = len(coeffs)
    D = [[sum(sp.Rational(c) * x ** k / math.factorial(k) for k, c in enumerate(coeffs[v]))]
         for v in range(nv)]

    def flux(Us):
        if system == oracle.BURGERS:
            return [Us[0] ** 2 / 2]
        rho, m, E = Us
        u = m / rho
        p = (sp.Rational(gamma).limit_denominator(1000) - 1) * (E - m * u / 2)
        return [m, m * u + p, (E + p) * u]

    for b in range(P):
        Ut = [sum(D[v][j] * t ** j / math.factorial(j) for j in range(b + 1)) for v in range(nv)]
        Fb = [sp.diff(f, t, b).subs(t, 0) for f in flux(Ut)]
        for v in range(nv):
            D[v].append(-sp.diff(Fb[v], x))
    out = np.zeros((nv, P + 1, P + 1))
    for v in range(nv):
        for b in range(P + 1):
            for a in range(P + 1 - b):
                out[v, a, b] = float(sp.diff(D[v][b], x, a).subs(x, 0)) * lam ** b
    return out


@pytest.mark.parametrize("P", [1, 2, 3, 4])
def test_burgers_ck_brute_force(P):
    from fractions import Fraction
    rng = np.random.default_rng(10 + P)
    coeffs = [[str(Fraction(int(rng.integers(-9, 10)), 7)) for _ in range(P + 1)]]
    lam = 0.375
    ref = _symbolic_ck(oracle.BURGERS, P, coeffs, lam)
    q = np.array([[float(Fraction(c)) for c in coeffs[0]]])
    U, _ = oracle.ck_table(oracle.make_law(oracle.BURGERS, P), q, lam)
    np.testing.assert_allclose(U, ref, rtol=1e-12, atol=1e-13)


@pytest.mark.parametrize("P", [1, 2, 3])
def test_euler_ck_brute_force(P):
    from fractions import Fraction
    rng = np.random.default_rng(20 + P)
    base = [Fraction(5, 4), Fraction(1, 3), Fraction(3, 1)]   # rho, m, E at the centre
    coeffs = []
    for v in range(3):
        row = [base[v]] + [Fraction(int(rng.integers(-5, 6)), 11) for _ in range(P)]
        coeffs.append([str(c) for c in row])
    lam = 0.25
    ref = _symbolic_ck(oracle.EULER, P, coeffs, lam, gamma=1.4)
    q = np.array([[float(Fraction(c)) for c in row] for row in coeffs])
    U, _ = oracle.ck_table(oracle.make_law(oracle.EULER, P, gamma=1.4), q, lam)
    np.testing.assert_allclose(U, ref, rtol=1e-11, atol=1e-12)
