"""Pins of the 2D oracle (Sec. 3, Sec. 4, Appendix B) against things fixed
outside it:
  * Table 3 (isentropic vortex, Sec. 5.3) for LCCS and WCCS at P = 1..3;
  * the exact time derivatives of exact solutions (the translating vortex,
    linear advection, 2D Burgers with linear data): the Cauchy-Kovalewski
    tables must reproduce them;
  * Gauss-Legendre quadrature of the exact space-time polynomial for the
    quarter averages, edge fluxes and vertex values of Appendix B;
  * exactness for polynomial data of degree <= P, limiter on or off;
  * reduction of the linear scheme to the 1D oracle on y-independent data;
  * x <-> y transpose symmetry, x and y mirror symmetry (Burgers: point
    reflection with u -> -u) of the limited half-step on discontinuous data,
    conservation, and the rotated eigenvectors against a complex-step
    Jacobian;
  * the smoothness indicator of Eq. 2DSmoothIndicator against quadrature;
  * order P + 1 against exact solutions (advection; Burgers before its
    shock), and Sod's tube along x against the exact Riemann solution with
    the rotated limiter on (first-order L1 rate, rows kept identical);
  * the limited advection half-step commutes with adding a constant (the
    limiter sees differences only), on rough data where it is active."""
import math
import os

import numpy as np
import pytest

import oracle
from oracle import exact
from paper_2104_04347_gb300 import inputs

CFL = {1: 0.4, 2: 0.3, 3: 0.25}


def _table3(golden_dir):
    rows = []
    with open(os.path.join(golden_dir, "table3_vortex.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                s, P, inv, l1, linf = line.split()
                rows.append((s, int(P), int(inv), float(l1), float(linf)))
    return rows


def _vortex_errors(scheme, P, n):
    pr = inputs.isentropic_vortex(n, P)
    s = oracle.Solver2D(oracle.make_law2d(oracle.EULER, P, limiter=scheme == "WCCS"), pr.q0, pr.dx, pr.dy)
    s.step_until(2.0, CFL[P])
    assert s.parity == 0 and abs(s.t - 2.0) < 1e-12
    X, Y = inputs._grid2d(n, n, -5.0, 5.0, -5.0, 5.0, inputs.PERIODIC)
    err = np.abs(s.q[:, :, 0, 0] - inputs.vortex_exact(X, Y, s.t)[0])
    return err.mean(), err.max()


def test_table3_meshes_1_5_and_1_10(golden_dir):
    # Readings fixed here (none is stated in the paper): the half step obeys
    # dt = nu / max over cells of ((|u| + c)/dx + (|v| + c)/dy), with the 1D
    # CFL numbers; the errors are the mean / max of the density point values
    # at the cell centres; the rotated direction is the central-difference
    # gradient of rho e.  The finer rows cost minutes on the CPU and are
    # recorded in the design notes instead.
    rows = [r for r in _table3(golden_dir) if r[2] in (5, 10)]
    assert len(rows) == 12
    for scheme, P, inv, l1, linf in rows:
        g1, ginf = _vortex_errors(scheme, P, 10 * inv)
        assert abs(g1 / l1 - 1) < 0.05, (scheme, P, inv, g1, l1)
        assert abs(ginf / linf - 1) < 0.05, (scheme, P, inv, ginf, linf)


def _expected_translation(D, P, cx, cy):
    """Scaled U[k][l][m] of u(x - cx t, y - cy t) from the scaled spatial
    derivatives D (cx, cy already multiplied by lamx, lamy):
    dt^m d_t^m = (-cx dx d_x - cy dy d_y)^m."""
    E = np.zeros((P + 1, P + 1, P + 1))
    for k in range(P + 1):
        for l in range(P + 1 - k):
            for m in range(P + 1 - k - l):
                s = 0.0
                for j in range(m + 1):
                    s += math.comb(m, j) * cx ** j * cy ** (m - j) * D[inputs.idx2d(k + j, l + m - j)]
                E[k, l, m] = (-1) ** m * s
    return E


@pytest.mark.parametrize("P", [1, 2, 3, 4])
def test_ck_reproduces_the_translating_vortex(P):
    pr = inputs.isentropic_vortex(20, P)
    law = oracle.make_law2d(oracle.EULER, P)
    lamx = lamy = 0.29  # the DOFs are scaled with dx = dy
    for (j, i) in [(9, 11), (12, 7), (3, 15), (10, 10)]:
        U, _, _ = oracle.ck_table2d(law, pr.q0[j, i], lamx, lamy)
        for v in range(4):
            exp = _expected_translation(pr.q0[j, i, v], P, lamx, lamy)
            scale = np.max(np.abs(pr.q0[j, i, v])) + 1e-300
            assert np.max(np.abs(U[v] - exp)) <= 1e-12 * scale, (P, j, i, v)


@pytest.mark.parametrize("P", [1, 2, 3, 4])
def test_ck_advection_and_burgers_closed_forms(P):
    rng = np.random.default_rng(100 + P)
    lamx, lamy = 0.23, 0.41
    # advection: u(x - ax t, y - ay t)
    ax, ay = 0.7, -1.3
    law = oracle.make_law2d(oracle.ADVECTION, P, ax=ax, ay=ay)
    D = rng.standard_normal(inputs.nq2d(P))
    U, F, G = oracle.ck_table2d(law, D, lamx, lamy)
    assert np.allclose(U[0], _expected_translation(D, P, ax * lamx, ay * lamy), rtol=0, atol=1e-13)
    assert np.allclose(F[0], ax * U[0], rtol=0, atol=1e-15) and np.allclose(G[0], ay * U[0], rtol=0, atol=1e-15)
    # Burgers f = g = u^2/2 with linear data u0 = a + b x + c y:
    # u = u0 / (1 + s t), s = b + c, so d_t^m u = (-s)^m m! u0 / (1 + s t)^(m+1)
    law = oracle.make_law2d(oracle.BURGERS, P)
    dx, dy, dt = 0.05, 0.08, 0.01
    a, b, c = 0.4, 0.9, -0.3
    D = np.zeros(inputs.nq2d(P))
    D[0], D[inputs.idx2d(1, 0)], D[inputs.idx2d(0, 1)] = a, b * dx, c * dy
    U, _, _ = oracle.ck_table2d(law, D, dt / dx, dt / dy)
    s = b + c
    for m in range(P + 1):
        f = (-s * dt) ** m * math.factorial(m)
        assert abs(U[0, 0, 0, m] - f * a) <= 1e-14
        if m <= P - 1:
            assert abs(U[0, 1, 0, m] - f * b * dx) <= 1e-14 and abs(U[0, 0, 1, m] - f * c * dy) <= 1e-14
        for k in range(P + 1):
            for l in range(P + 1 - k - m):
                if k + l >= 2:
                    assert abs(U[0, k, l, m]) <= 1e-14


def _poly_eval(D, P, xi, eta):
    return sum(D[inputs.idx2d(k, l)] * xi ** k * eta ** l / (math.factorial(k) * math.factorial(l))
               for k in range(P + 1) for l in range(P + 1 - k))


def _poly_deriv(D, P, k0, l0, xi, eta):
    """d^k0_xi d^l0_eta of the polynomial with scaled derivatives D."""
    s = 0.0
    for k in range(k0, P + 1):
        for l in range(l0, P + 1 - k):
            s += D[inputs.idx2d(k, l)] * xi ** (k - k0) * eta ** (l - l0) / (math.factorial(k - k0) * math.factorial(l - l0))
    return s


@pytest.mark.parametrize("P", [1, 2, 3, 4])
def test_appendix_b_terms_against_quadrature(P):
    # linear advection of a random degree-P polynomial: the space-time
    # solution u(xi - cx tau, eta - cy tau) is itself a polynomial, so every
    # term of Appendix B is an exact integral that Gauss-Legendre reproduces
    rng = np.random.default_rng(7 + P)
    ax, ay, lamx, lamy = 0.8, -0.6, 0.3, 0.2
    cx, cy = ax * lamx, ay * lamy
    law = oracle.make_law2d(oracle.ADVECTION, P, ax=ax, ay=ay)
    D = rng.standard_normal(inputs.nq2d(P))
    qa, fl, V = oracle.parent_terms2d(law, D, lamx, lamy)
    g, w = np.polynomial.legendre.leggauss(8)

    def mean_over(lo, hi, fn):  # mean of fn over [lo, hi] (vectorised)
        x = 0.5 * (hi - lo) * g + 0.5 * (hi + lo)
        return float(np.sum(0.5 * w * fn(x)))

    for idx, (sx, sy) in enumerate([(1, 1), (1, -1), (-1, 1), (-1, -1)]):  # RU, RD, LU, LD
        xlo, xhi = (0.0, 0.5) if sx > 0 else (-0.5, 0.0)
        ylo, yhi = (0.0, 0.5) if sy > 0 else (-0.5, 0.0)
        ref = mean_over(ylo, yhi, lambda y: np.array([mean_over(xlo, xhi, lambda x: _poly_eval(D, P, x, yy)) for yy in y]))
        assert abs(qa[0, idx] - ref) <= 1e-13 * (1 + abs(ref))
    # f on x = x_i over eta in [0, 1/2] (U) or [-1/2, 0] (D), tau in [0, 1]
    for idx, (lo, hi) in enumerate([(0.0, 0.5), (-0.5, 0.0)]):
        ref = ax * mean_over(0.0, 1.0, lambda tau: np.array(
            [mean_over(lo, hi, lambda eta: _poly_eval(D, P, -cx * t, eta - cy * t)) for t in tau]))
        assert abs(fl[0, idx] - ref) <= 1e-13 * (1 + abs(ref)), ("f", idx)
    # g on y = y_j over xi in [0, 1/2] (R) or [-1/2, 0] (L)
    for idx, (lo, hi) in enumerate([(0.0, 0.5), (-0.5, 0.0)]):
        ref = ay * mean_over(0.0, 1.0, lambda tau: np.array(
            [mean_over(lo, hi, lambda xi: _poly_eval(D, P, xi - cx * t, -cy * t)) for t in tau]))
        assert abs(fl[0, 2 + idx] - ref) <= 1e-13 * (1 + abs(ref)), ("g", idx)
    # vertex values at t^{n+1/2}: the translated polynomial's derivatives
    for k in range(P + 1):
        for l in range(P + 1 - k):
            ref = _poly_deriv(D, P, k, l, -cx, -cy)
            assert abs(V[0, inputs.idx2d(k, l)] - ref) <= 1e-13 * (1 + abs(ref))


@pytest.mark.parametrize("limiter", [False, True])
@pytest.mark.parametrize("P", [1, 2, 3, 4])
def test_exact_for_polynomials(P, limiter):
    # the new cell centred at (0, 0) has parents at (+-1/2, +-1/2) (cell
    # units); data of degree <= P advected exactly: the new DOFs are the
    # translate's derivatives at the new centre, and sigma = 0 keeps w_0 = 1
    rng = np.random.default_rng(31 + P)
    ax, ay, lamx, lamy = 1.1, 0.7, 0.21, 0.17
    cx, cy = ax * lamx, ay * lamy
    law = oracle.make_law2d(oracle.ADVECTION, P, ax=ax, ay=ay, limiter=limiter)
    Dc = rng.standard_normal(inputs.nq2d(P))  # the data around the new centre

    def dofs_at(xi, eta, shift=0.0):
        out = np.zeros(inputs.nq2d(P))
        for k in range(P + 1):
            for l in range(P + 1 - k):
                out[inputs.idx2d(k, l)] = _poly_deriv(Dc, P, k, l, xi - cx * shift, eta - cy * shift)
        return out

    parents = [dofs_at(-0.5, -0.5), dofs_at(0.5, -0.5), dofs_at(0.5, 0.5), dofs_at(-0.5, 0.5)]
    new, w, _, _ = oracle.new_cell2d(law, *parents, lamx, lamy, diagnostics=True)
    exact = dofs_at(0.0, 0.0, shift=1.0)
    assert np.max(np.abs(new[0] - exact)) <= 1e-12 * np.max(np.abs(exact)), (new[0], exact)
    if limiter and P >= 2:
        assert abs(w[0, 0] - 1.0) <= 1e-12


def _lift_1d(q1, nv2):
    """1D DOFs [cells, nv, P+1] -> y-independent 2D DOFs [ny=3, cells, nv2, nq]."""
    n, nv, nk = q1.shape
    P = nk - 1
    q = np.zeros((3, n, nv2, inputs.nq2d(P)))
    vmap = [0, 1, 3] if nv2 == 4 else [0]  # Euler: (rho, m, E) -> (rho, m, n = 0, E)
    for a, v in enumerate(vmap):
        for k in range(nk):
            q[:, :, v, inputs.idx2d(k, 0)] = q1[None, :, a, k]
    return q


@pytest.mark.parametrize("P", [1, 2, 3, 4])
def test_linear_scheme_reduces_to_1d(P):
    # without the limiter, y-independent data follow the 1D scheme exactly
    # (the g fluxes cancel, every y-derivative stays zero)
    for system in (oracle.ADVECTION, oracle.EULER):
        if system == oracle.ADVECTION:
            pr1 = inputs.advection_sine(40, P)
            law1 = oracle.make_law(oracle.ADVECTION, P, limiter=False, a=0.9)
            law2 = oracle.make_law2d(oracle.ADVECTION, P, limiter=False, ax=0.9, ay=0.6)
        else:
            pr1 = inputs.euler_density_wave(40, P)
            law1 = oracle.make_law(oracle.EULER, P, limiter=False)
            law2 = oracle.make_law2d(oracle.EULER, P, limiter=False)
        q1 = pr1.q0
        q2 = _lift_1d(q1, 4 if system == oracle.EULER else 1)
        lam = 0.2
        for parity in (0, 1):
            r1 = oracle.halfstep(law1, parity, q1, lam)
            r2 = oracle.halfstep2d(law2, parity, q2, lam, 0.37)
            want = _lift_1d(r1, q2.shape[2])
            scale = np.max(np.abs(want)) + 1e-300
            assert np.max(np.abs(r2 - want)) <= 1e-13 * scale, (system, parity)
            q1, q2 = r1, r2


def _transpose(q, euler):
    """Swap x and y: cell (j, i) -> (i, j), u_{kx,ly} -> u_{lx,ky}, and for
    Euler the two momentum components."""
    ny, nx, nv, nq = q.shape
    P = int(round((math.sqrt(8 * nq + 1) - 3) / 2))
    out = np.zeros((nx, ny, nv, nq))
    for k in range(P + 1):
        for l in range(P + 1 - k):
            out[:, :, :, inputs.idx2d(l, k)] = np.swapaxes(q[:, :, :, inputs.idx2d(k, l)], 0, 1)
    if euler:
        out[:, :, [1, 2]] = out[:, :, [2, 1]]
    return out


@pytest.mark.parametrize("P", [1, 2, 3])
def test_transpose_symmetry_with_limiter(P):
    # a vortex moved off the diagonal so that x and y differ
    pr = inputs.isentropic_vortex(24, P)
    q = np.roll(pr.q0, (3, -5), axis=(0, 1))
    law = oracle.make_law2d(oracle.EULER, P, limiter=True)
    a = oracle.halfstep2d(law, 0, q, 0.05, 0.05)
    b = oracle.halfstep2d(law, 0, _transpose(q, True), 0.05, 0.05)
    scale = np.max(np.abs(a), axis=(0, 1, 3))[None, None, :, None]
    assert np.max(np.abs(_transpose(a, True) - b) / scale) <= 1e-12


def _averages(q, P):
    w = np.zeros(inputs.nq2d(P))
    for k in range(0, P + 1, 2):
        for l in range(0, P + 1 - k, 2):
            w[inputs.idx2d(k, l)] = 1.0 / (math.factorial(k + 1) * 2 ** k * math.factorial(l + 1) * 2 ** l)
    return q @ w


@pytest.mark.parametrize("P", [1, 2, 3])
def test_conservation_with_limiter(P):
    pr = inputs.isentropic_vortex(20, P)
    law = oracle.make_law2d(oracle.EULER, P, limiter=True)
    s = oracle.Solver2D(law, pr.q0, pr.dx, pr.dy)
    before = _averages(s.q, P).sum(axis=(0, 1))
    s.step_cfl(12, CFL[P])
    after = _averages(s.q, P).sum(axis=(0, 1))
    assert np.max(np.abs(after - before) / np.abs(before).clip(1.0)) <= 1e-12


def _flux_rotated(U, nx, ny, gamma=1.4):
    rho, m, n, E = U
    u, v = m / rho, n / rho
    p = (gamma - 1) * (E - 0.5 * rho * (u * u + v * v))
    F = np.array([m, m * u + p, m * v, (E + p) * u])
    G = np.array([n, n * u, n * v + p, (E + p) * v])
    return nx * F + ny * G


def test_rotated_eigenvectors():
    U = np.array(inputs.vortex_conserved(np.array(0.7), np.array(-0.4))).astype(float)
    for theta in (0.0, 0.4, 1.9, -2.5):
        nx, ny = math.cos(theta), math.sin(theta)
        R, L = oracle.euler_eigenvectors2d(1.4, U, nx, ny)
        assert np.allclose(L @ R, np.eye(4), atol=1e-13)
        A = np.zeros((4, 4))
        for j in range(4):  # complex-step Jacobian of the rotated flux
            Uc = U.astype(complex)
            Uc[j] += 1e-30j
            A[:, j] = _flux_rotated(Uc, nx, ny).imag / 1e-30
        u, v = U[1] / U[0], U[2] / U[0]
        p = 0.4 * (U[3] - 0.5 * U[0] * (u * u + v * v))
        c = math.sqrt(1.4 * p / U[0])
        un = u * nx + v * ny
        assert np.allclose(L @ A @ R, np.diag([un - c, un, un, un + c]), atol=1e-12)


@pytest.mark.parametrize("P", [1, 2, 3, 4])
def test_smoothness_indicator_against_quadrature(P):
    rng = np.random.default_rng(500 + P)
    D = rng.standard_normal(inputs.nq2d(P))
    g, w = np.polynomial.legendre.leggauss(8)
    X, Y = np.meshgrid(0.5 * g, 0.5 * g)
    W = np.outer(0.5 * w, 0.5 * w)
    ref = 0.0
    for k in range(P + 1):
        for l in range(P + 1 - k):
            if k + l == 0:
                continue
            vals = np.vectorize(lambda x, y: _poly_deriv(D, P, k, l, x, y))(X, Y)
            ref += float(np.sum(W * vals ** 2))
    assert abs(oracle.smoothness2d(D, P) - ref) <= 1e-12 * ref


def _diag_dofs(n, P, u0_derivs):
    """DOFs of u0(x + y) on periodic [-1, 1]^2: u_{kx,ly} = dx^k dy^l u0^(k+l)(x + y)."""
    X, Y = inputs._grid2d(n, n, -1.0, 1.0, -1.0, 1.0, inputs.PERIODIC)
    d = 2.0 / n
    q = np.zeros((n, n, 1, inputs.nq2d(P)))
    for k in range(P + 1):
        for l in range(P + 1 - k):
            q[:, :, 0, inputs.idx2d(k, l)] = d ** (k + l) * u0_derivs(X + Y, k + l)
    return q, X, Y, d


def _orders(errs, ns):
    return [math.log(errs[i] / errs[i + 1]) / math.log(ns[i + 1] / ns[i]) for i in range(len(errs) - 1)]


@pytest.mark.parametrize("P", [1, 2, 3])
def test_advection_converges_at_order_p_plus_1(P):
    # u0 = sin(pi (x + y)) carried by (ax, ay) = (1, 0.5) to t = 0.5 (linear scheme)
    ax, ay, t_end = 1.0, 0.5, 0.5
    law = oracle.make_law2d(oracle.ADVECTION, P, limiter=False, ax=ax, ay=ay)
    ns, errs = (16, 32, 64), []
    for n in ns:
        q, X, Y, d = _diag_dofs(n, P, lambda s, k: math.pi ** k * np.sin(math.pi * s + k * math.pi / 2))
        s = oracle.Solver2D(law, q, d, d)
        s.step_until(t_end, CFL[P])
        errs.append(float(np.mean(np.abs(s.q[:, :, 0, 0] - np.sin(math.pi * (X - ax * s.t + Y - ay * s.t))))))
    o = _orders(errs, ns)
    assert all(P + 1 - 0.25 < oi < P + 1 + 0.8 for oi in o), (errs, o)


@pytest.mark.parametrize("P", [1, 2, 3])
def test_burgers_converges_before_the_shock(P):
    # f = g = u^2/2 with u0 = 0.5 + 0.25 sin(pi (x + y)): u depends on s = x + y
    # only and solves u_t + 2 u u_s = 0, so u = u0(xi) with xi + 2 t u0(xi) = s
    # (shock at t = 2 / pi); the linear scheme to t = 0.2 against it
    t_end = 0.2
    law = oracle.make_law2d(oracle.BURGERS, P, limiter=False)

    def u0d(s, k):
        return (0.5 if k == 0 else 0.0) + 0.25 * math.pi ** k * np.sin(math.pi * s + k * math.pi / 2)

    ns, errs = (16, 32, 64), []
    for n in ns:
        q, X, Y, d = _diag_dofs(n, P, u0d)
        s = oracle.Solver2D(law, q, d, d)
        s.step_until(t_end, CFL[P])
        ex = exact.burgers_characteristics(lambda z: u0d(z, 0), lambda z: u0d(z, 1), X + Y, 2.0 * s.t)
        errs.append(float(np.mean(np.abs(s.q[:, :, 0, 0] - ex))))
    o = _orders(errs, ns)
    assert all(P + 1 - 0.35 < oi < P + 1 + 0.6 for oi in o), (errs, o)


def _mirror_x(q, euler, sign=1.0):
    """x -> -x on a periodic mesh (cell i -> n - 1 - i): u_{kx,ly} picks up
    (-1)^k, and for Euler the x-momentum changes sign; `sign` multiplies
    the whole state (Burgers needs u -> -u)."""
    nq = q.shape[3]
    P = int(round((math.sqrt(8 * nq + 1) - 3) / 2))
    out = sign * q[:, ::-1].copy()
    for k in range(1, P + 1, 2):
        for l in range(P + 1 - k):
            out[:, :, :, inputs.idx2d(k, l)] *= -1.0
    if euler:
        out[:, :, 1] *= -1.0
    return out


def _mirror_y(q, euler, sign=1.0):
    return _transpose(_mirror_x(_transpose(q, euler), euler, sign), euler)


def _new_index_after_mirror(n, parity):
    # parity 0: new cell i sits between parents i and i + 1, which mirror to
    # n - 2 - i and n - 1 - i; parity 1: between i - 1 and i -> n - i
    return (n - 2 - np.arange(n)) % n if parity == 0 else (n - np.arange(n)) % n


@pytest.mark.parametrize("P", [1, 2, 3])
def test_mirror_symmetry_with_limiter(P):
    # x -> -x and y -> -y for Euler, (x, y, u) -> (-x, -y, -u) for Burgers, on
    # discontinuous data (a four-state Riemann problem made periodic, rolled
    # off-centre and stepped three times so that every derivative is in use):
    # the limited half-step commutes with each mirror.  Catches a sign error
    # in any odd-derivative, flux or rotated-direction term that the
    # transpose symmetry maps onto itself.
    n = 26
    for system in (oracle.EULER, oracle.BURGERS):
        euler = system == oracle.EULER
        law = oracle.make_law2d(system, P, limiter=True)
        if euler:
            q = np.roll(inputs.riemann2d(n - 1, P, 1).q0[: n, : n], (3, -5), axis=(0, 1)).copy()
        else:
            X, Y = inputs._grid2d(n, n, -1.0, 1.0, -1.0, 1.0, inputs.PERIODIC)
            q = np.zeros((n, n, 1, inputs.nq2d(P)))
            q[:, :, 0, 0] = np.where(X + 0.3 * Y > 0.1, 1.0, -0.4) + 0.3 * np.sin(math.pi * Y)
        s = oracle.Solver2D(law, q, 2.0 / n, 2.0 / n)
        s.step_cfl(3, CFL[P])
        q = s.q
        for parity in (1, 0):
            a = oracle.halfstep2d(law, parity, q, 0.11, 0.07)
            scale = np.max(np.abs(a), axis=(0, 1, 3))[None, None, :, None]
            idx = _new_index_after_mirror(n, parity)
            if euler:
                b = oracle.halfstep2d(law, parity, _mirror_x(q, True), 0.11, 0.07)
                assert np.max(np.abs(_mirror_x(a, True)[:, ::-1][:, idx] - b) / scale) <= 1e-12, (P, parity, "x")
                b = oracle.halfstep2d(law, parity, _mirror_y(q, True), 0.11, 0.07)
                assert np.max(np.abs(_mirror_y(a, True)[::-1][idx] - b) / scale) <= 1e-12, (P, parity, "y")
            else:
                qm = _mirror_y(_mirror_x(q, False, -1.0), False)
                b = oracle.halfstep2d(law, parity, qm, 0.11, 0.07)
                am = _mirror_y(_mirror_x(a, False, -1.0), False)[::-1, ::-1][idx][:, idx]
                assert np.max(np.abs(am - b) / scale) <= 1e-12, (P, parity, "xy")
            q = a


@pytest.mark.parametrize("bc", [oracle.PERIODIC, oracle.TRANSMISSIVE])
def test_sampled_new_cells_match_the_whole_stage(bc):
    # the one-cell route the full-size GPU tests use gives the whole-stage
    # half-step's cells bit for bit, corners and edges included
    from tests.gpu_common import sampled_new_cells2d
    P = 2
    pr = inputs.isentropic_vortex(12, P)
    q = np.roll(pr.q0, (2, -3), axis=(0, 1))
    law = oracle.make_law2d(oracle.EULER, P, limiter=True, bc=bc)
    for parity in (0, 1):
        want = oracle.halfstep2d(law, parity, q, 0.13, 0.09)
        cells = [(j, i) for j in range(want.shape[0]) for i in range(want.shape[1])]
        got = sampled_new_cells2d(law, q, parity, cells, 0.13, 0.09)
        assert np.array_equal(got.reshape(want.shape), want), (bc, parity)
        q = want  # transmissive: 11 x 11 cells, then 12 x 12 again


def test_sod_along_x_against_the_exact_riemann_solution():
    # Sod's tube (Sec. 5.2: [0, 2], jump at 1, t = 0.4) laid along x on a
    # 2D mesh of three rows, transmissive on every side, limiter on (rotated
    # characteristic limiting, Sec. 4): the rows stay bitwise identical, the
    # y-momentum stays at rounding level, the density's L1 error against the
    # exact Riemann solution falls at the first-order rate of a captured shock
    # and contact, and the higher degrees resolve it better (Sec. 5)
    left, right = (1.0, 0.0, 1.0), (0.125, 0.0, 0.1)
    errs = {}
    for P in (1, 2, 3):
        law = oracle.make_law2d(oracle.EULER, P, limiter=True, bc=oracle.TRANSMISSIVE)
        for N in (100, 200, 400):
            pr1 = inputs.sod(N, P)
            s = oracle.Solver2D(law, _lift_1d(pr1.q0, 4), pr1.dx, pr1.dx)
            s.step_until(0.4, CFL[P])
            assert s.parity == 0 and abs(s.t - 0.4) < 1e-12
            assert np.array_equal(s.q[1:], np.broadcast_to(s.q[:1], s.q[1:].shape))
            assert np.max(np.abs(s.q[:, :, 2])) <= 1e-14
            x = inputs.centres(N, 0.0, 2.0, inputs.TRANSMISSIVE)
            rho = exact.riemann_sample(left, right, (x - 1.0) / s.t)[0]
            errs[P, N] = float(np.mean(np.abs(s.q[0, :, 0, 0] - rho)))
        orders = [math.log2(errs[P, N] / errs[P, 2 * N]) for N in (100, 200)]
        assert all(0.6 < o < 1.2 for o in orders), (P, orders)
    for N in (100, 200, 400):
        assert errs[3, N] < errs[2, N] < errs[1, N], errs


@pytest.mark.parametrize("P", [1, 2, 3])
def test_limited_advection_commutes_with_a_constant_shift(P):
    # linear advection is unchanged by u -> u + c, and the limiter of Sec. 3.2
    # sees the data only through differences (one-sided slopes, vertex
    # residuals, derivatives) and keeps the average: the limited half-step
    # of the shifted data is the shifted half-step, on rough data where the
    # weights are far from the linear ones
    rng = np.random.default_rng(P)
    n = 20
    q = 0.3 * rng.standard_normal((n, n, 1, inputs.nq2d(P)))
    law = oracle.make_law2d(oracle.ADVECTION, P, limiter=True, ax=0.8, ay=-0.55)
    for parity in (0, 1):
        a = oracle.halfstep2d(law, parity, q, 0.2, 0.15)
        for c in (1.0, -37.5):
            qc = q.copy()
            qc[..., 0] += c
            b = oracle.halfstep2d(law, parity, qc, 0.2, 0.15)
            b[..., 0] -= c
            assert np.max(np.abs(b - a)) <= 1e-12 * (1.0 + abs(c)), (P, parity, c)
