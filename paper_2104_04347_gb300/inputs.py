"""Seeded, synthetic initial data for the 1D WCC workloads.

This module is the only code shared by the CUDA path's tests/bench and the CPU
oracle.  It holds no arithmetic of the scheme: it only evaluates initial
conditions and turns them into the paper's DOFs, the scaled derivatives
u_kx = dx^k d^k u0/dx^k at every cell centre of the integer stage
(Eqs. 1D_Derivative_DEF, 1DPolynomial_Space).  Piecewise-constant data get the
exact cell average of the data and zero derivatives.

Random numbers come from splitmix64 (Steele, Lea & Flood 2014), so every
workload is reproducible from its seed on any machine.

Array layout of every generator's result: float64 [cells, nv, P+1].
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

ADVECTION, BURGERS, EULER = 0, 1, 2
PERIODIC, TRANSMISSIVE = 0, 1
GAMMA = 1.4

_MASK = (1 << 64) - 1


class SplitMix64:
    """splitmix64 generator; ``uniform()`` gives doubles in [0, 1) from the top
    53 bits."""

    def __init__(self, seed: int):
        self.state = seed & _MASK

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & _MASK
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK
        return z ^ (z >> 31)

    def uniform(self, lo: float = 0.0, hi: float = 1.0) -> float:
        return lo + (hi - lo) * ((self.next_u64() >> 11) * (1.0 / (1 << 53)))


def num_cells(N: int, bc: int, parity: int = 0) -> int:
    """Cells of a stage: N for periodic; N+1 on the integer stage and N on the
    half stage for non-periodic boundaries (Sec. 2.1)."""
    if bc == PERIODIC:
        return N
    return N + 1 if parity == 0 else N


def centres(N: int, x_l: float, x_r: float, bc: int, parity: int = 0) -> np.ndarray:
    """Cell centres: x_L + i dx on the integer stage, x_L + (i + 1/2) dx on the
    half stage."""
    dx = (x_r - x_l) / N
    off = 0.0 if parity == 0 else 0.5
    return x_l + (np.arange(num_cells(N, bc, parity)) + off) * dx


def smooth_dofs(derivs, x: np.ndarray, dx: float, P: int) -> np.ndarray:
    """DOFs of smooth data: derivs(x, k) returns d^k u0/dx^k; result [cells, P+1]."""
    return np.stack([derivs(x, k) * dx ** k for k in range(P + 1)], axis=1)


# ---------------------------------------------------------------- problems


@dataclass
class Problem:
    """A workload: the conservation law, mesh, boundary and integer-stage DOFs."""

    system: int
    N: int
    P: int
    x_l: float
    x_r: float
    bc: int
    q0: np.ndarray  # [cells, nv, P+1]
    name: str = ""

    @property
    def dx(self) -> float:
        return (self.x_r - self.x_l) / self.N

    @property
    def nv(self) -> int:
        return 3 if self.system == EULER else 1


def sine_derivative(x, k, freq=math.pi, amp=1.0, phase=0.0):
    """k-th derivative of amp * sin(freq x + phase)."""
    return amp * freq ** k * np.sin(freq * x + phase + k * math.pi / 2)


def advection_sine(N: int, P: int, x_l: float = -1.0, x_r: float = 1.0) -> Problem:
    """u0 = sin(pi x) on a periodic domain (Sec. 5.1, first case)."""
    x = centres(N, x_l, x_r, PERIODIC)
    dx = (x_r - x_l) / N
    q = smooth_dofs(lambda xx, k: sine_derivative(xx, k), x, dx, P)[:, None, :]
    return Problem(ADVECTION, N, P, x_l, x_r, PERIODIC, q, "advection-sine")


def advection_polynomial(N: int, P: int, coeffs, x_l: float = 0.0, x_r: float = 1.0) -> Problem:
    """u0 = sum_j coeffs[j] x^j with transmissive boundaries."""
    x = centres(N, x_l, x_r, TRANSMISSIVE)
    dx = (x_r - x_l) / N
    poly = np.polynomial.Polynomial(coeffs)

    def d(xx, k):
        return poly.deriv(k)(xx) if k <= poly.degree() else np.zeros_like(xx)

    q = smooth_dofs(d, x, dx, P)[:, None, :]
    return Problem(ADVECTION, N, P, x_l, x_r, TRANSMISSIVE, q, "advection-polynomial")


@dataclass
class FourierData:
    mean: float
    amps: np.ndarray
    phases: np.ndarray

    def derivative(self, x, k):
        out = np.full_like(x, self.mean if k == 0 else 0.0, dtype=np.float64)
        for j, (A, ph) in enumerate(zip(self.amps, self.phases), start=1):
            out = out + sine_derivative(x, k, freq=float(j), amp=A, phase=ph)
        return out


def burgers_fourier_data(seed: int = 2104043470, modes: int = 8) -> FourierData:
    """u0 = 0.5 + sum_{k=1}^{8} A_k sin(k x + phi_k), A_k ~ U(-0.2, 0.2),
    phi_k ~ U(0, 2 pi)."""
    rng = SplitMix64(seed)
    amps = np.array([rng.uniform(-0.2, 0.2) for _ in range(modes)])
    phases = np.array([rng.uniform(0.0, 2 * math.pi) for _ in range(modes)])
    return FourierData(0.5, amps, phases)


def burgers_fourier(N: int, P: int, seed: int = 2104043470) -> Problem:
    """Burgers on periodic [0, 2 pi] with seeded Fourier initial data."""
    data = burgers_fourier_data(seed)
    x_l, x_r = 0.0, 2 * math.pi
    x = centres(N, x_l, x_r, PERIODIC)
    q = smooth_dofs(data.derivative, x, (x_r - x_l) / N, P)[:, None, :]
    return Problem(BURGERS, N, P, x_l, x_r, PERIODIC, q, "burgers-fourier")


def shock_time(data: FourierData) -> float:
    """t_s = -1 / min u0' (first gradient catastrophe of Burgers)."""
    x = np.linspace(0.0, 2 * math.pi, 200001)
    return -1.0 / float(np.min(data.derivative(x, 1)))


def primitive_to_conserved(rho, u, p, gamma=GAMMA):
    return np.stack([rho, rho * u, p / (gamma - 1.0) + 0.5 * rho * u * u], axis=-1)


def riemann_states(seed: int = 2104043471):
    """rho, p ~ U(0.1, 1), u ~ U(-0.5, 0.5) on each side: ((rl, ul, pl), (rr, ur, pr))."""
    rng = SplitMix64(seed)
    rl, ul, pl = rng.uniform(0.1, 1.0), rng.uniform(-0.5, 0.5), rng.uniform(0.1, 1.0)
    rr, ur, pr = rng.uniform(0.1, 1.0), rng.uniform(-0.5, 0.5), rng.uniform(0.1, 1.0)
    return (rl, ul, pl), (rr, ur, pr)


def euler_riemann(N: int, P: int, left, right, x_l: float = 0.0, x_r: float = 1.0,
                  x0: float = 0.5, gamma: float = GAMMA, name: str = "euler-riemann") -> Problem:
    """Piecewise-constant Euler data with a jump at x0, transmissive boundaries.
    Each cell holds the exact cell average of the data (a cell cut by x0 gets
    the length-weighted mix of the two states) and zero derivatives."""
    x = centres(N, x_l, x_r, TRANSMISSIVE)
    dx = (x_r - x_l) / N
    UL = primitive_to_conserved(*[np.float64(v) for v in left], gamma=gamma)
    UR = primitive_to_conserved(*[np.float64(v) for v in right], gamma=gamma)
    frac_left = np.clip((x0 - (x - 0.5 * dx)) / dx, 0.0, 1.0)
    q = np.zeros((x.size, 3, P + 1))
    q[:, :, 0] = frac_left[:, None] * UL[None, :] + (1.0 - frac_left[:, None]) * UR[None, :]
    return Problem(EULER, N, P, x_l, x_r, TRANSMISSIVE, q, name)


def euler_riemann_seeded(N: int, P: int, seed: int = 2104043471) -> Problem:
    left, right = riemann_states(seed)
    return euler_riemann(N, P, left, right)


def sod(N: int, P: int) -> Problem:
    """Sod shock tube on [0, 2], jump at x = 1 (Sec. 5.2)."""
    return euler_riemann(N, P, (1.0, 0.0, 1.0), (0.125, 0.0, 0.1), 0.0, 2.0, 1.0, name="sod")


def euler_density_wave(N: int, P: int, amp: float = 0.2, gamma: float = GAMMA) -> Problem:
    """rho = 1 + amp sin(2 pi x), u = 1, p = 1 on periodic [0, 1]: conserved
    variables rho, m = rho, E = p/(gamma-1) + rho/2."""
    x_l, x_r = 0.0, 1.0
    x = centres(N, x_l, x_r, PERIODIC)
    dx = (x_r - x_l) / N

    def rho_d(xx, k):
        base = sine_derivative(xx, k, freq=2 * math.pi, amp=amp)
        return base + (1.0 if k == 0 else 0.0)

    rho = smooth_dofs(rho_d, x, dx, P)
    E = 0.5 * rho.copy()
    E[:, 0] += 1.0 / (gamma - 1.0)
    q = np.stack([rho, rho.copy(), E], axis=1)
    return Problem(EULER, N, P, x_l, x_r, PERIODIC, q, "euler-density-wave")


# ------------------------------------------------ piecewise-smooth initial data


def projected_dofs(func, N: int, P: int, x_l: float, x_r: float, bc: int, breaks=(), nodes: int = 24) -> np.ndarray:
    """DOFs of piecewise-smooth data: in every cell of the integer stage the
    L2 projection of func (x -> [points, nv] values) onto polynomials of
    degree P, written as the paper's scaled derivatives at the centre.  With
    xi = (x - x_i) / dx on [-1/2, 1/2] the projection is sum_n c_n L_n(2 xi),
    L_n the Legendre polynomials (orthogonal there, int L_n(2 xi)^2 dxi =
    1 / (2n + 1)), so c_n = (2n + 1) int u L_n(2 xi) dxi; expanding L_n(2 xi)
    in powers of xi gives the Taylor coefficients e_k and u_kx = k! e_k.
    Each cell is integrated piece by piece between the break points (jumps
    and kinks of the data) with Gauss-Legendre nodes mapped by
    x = a0 + (a1 - a0)(1 - cos t)/2, t in [0, pi]: the nodes cluster at both
    ends, which keeps square-root endpoints (the half ellipses) accurate.
    Result [cells, nv, P+1]."""
    x = centres(N, x_l, x_r, bc)
    dx = (x_r - x_l) / N
    g, gw = np.polynomial.legendre.leggauss(nodes)
    brk = np.sort(np.asarray(breaks, dtype=np.float64))
    # A[n, k]: coefficient of xi^k in L_n(2 xi)
    A = np.zeros((P + 1, P + 1))
    for n in range(P + 1):
        c = np.polynomial.legendre.leg2poly(np.eye(P + 1)[n])
        A[n, :c.size] = c * 2.0 ** np.arange(c.size)
    fact = np.array([math.factorial(k) for k in range(P + 1)], dtype=np.float64)
    out = None
    th = 0.5 * math.pi * (g + 1.0)
    for i, xc in enumerate(x):
        # pieces in the cell's own coordinate xi, so that their lengths sum to
        # exactly 1 whatever the rounding of the cell's position
        lo, hi = xc - 0.5 * dx, xc + 0.5 * dx
        inner = brk[(brk > lo) & (brk < hi)]
        cuts = np.concatenate(([-0.5], np.clip((inner - xc) / dx, -0.5, 0.5), [0.5]))
        mom = None
        for a0, a1 in zip(cuts[:-1], cuts[1:]):
            xi = a0 + (a1 - a0) * 0.5 * (1.0 - np.cos(th))
            ws = gw * (a1 - a0) * 0.25 * math.pi * np.sin(th)
            xs = xc + dx * xi
            vals = np.atleast_2d(func(xs))  # [points, nv]
            if vals.shape[0] != xs.size:
                vals = vals.T
            leg = np.polynomial.legendre.legvander(2.0 * xi, P)  # [points, P+1]
            part = np.einsum("p,pv,pn->vn", ws, vals, leg)
            mom = part if mom is None else mom + part
        cn = mom * (2.0 * np.arange(P + 1) + 1.0)  # [nv, P+1]
        e = cn @ A  # Taylor coefficients
        if out is None:
            out = np.zeros((x.size, e.shape[0], P + 1))
        out[i] = e * fact
    return out


def composite_wave_data(x):
    """Jiang-Shu composite profile on [-1, 1] (Sec. 5.1, second case): three
    Gaussians, a square wave, a triangle and three half ellipses, with a =
    0.5, z = -0.7, delta = 0.005, alpha = 10, beta = log 2 / (36 delta^2)."""
    a, z, d, al = 0.5, -0.7, 0.005, 10.0
    be = math.log(2.0) / (36.0 * d * d)
    x = np.asarray(x, dtype=np.float64)

    def G(zz):
        return np.exp(-be * (x - zz) ** 2)

    def F(aa):
        return np.sqrt(np.maximum(1.0 - al * al * (x - aa) ** 2, 0.0))

    u = np.zeros_like(x)
    m = (x >= -0.8) & (x <= -0.6)
    u[m] = ((G(z - d) + 4.0 * G(z) + G(z + d)) / 6.0)[m]
    u[(x >= -0.4) & (x <= -0.2)] = 1.0
    m = (x >= 0.0) & (x <= 0.2)
    u[m] = (1.0 - 10.0 * np.abs(x - 0.1))[m]
    m = (x >= 0.4) & (x <= 0.6)
    u[m] = ((F(a - d) + 4.0 * F(a) + F(a + d)) / 6.0)[m]
    return u[:, None]


# jumps and kinks of the composite profile (piece ends, the triangle's apex,
# the ellipses' edges a +- delta +- 1/alpha inside [0.4, 0.6])
COMPOSITE_BREAKS = (-0.8, -0.6, -0.4, -0.2, 0.0, 0.1, 0.2, 0.4, 0.405, 0.5, 0.595, 0.6)


def advection_composite(N: int, P: int) -> Problem:
    """The composite wave advected on periodic [-1, 1] (a = 1)."""
    q = projected_dofs(composite_wave_data, N, P, -1.0, 1.0, PERIODIC, COMPOSITE_BREAKS)
    return Problem(ADVECTION, N, P, -1.0, 1.0, PERIODIC, q, "advection-composite")


def shu_osher_data(x, gamma: float = GAMMA):
    """Modified Shu-Osher problem (Sec. 5.2, second case): a Mach 1.1 shock at
    x = -4.5, (rho, u, p) = (1.515695, 0.523346, 1.805) behind it, and
    (1 + 0.1 sin(20 pi x), 0, 1) ahead.  Conserved variables [points, 3]."""
    x = np.asarray(x, dtype=np.float64)
    left = x < -4.5
    rho = np.where(left, 1.515695, 1.0 + 0.1 * np.sin(20.0 * math.pi * x))
    u = np.where(left, 0.523346, 0.0)
    p = np.where(left, 1.805, 1.0)
    return primitive_to_conserved(rho, u, p, gamma)


def shu_osher(N: int, P: int) -> Problem:
    """The modified Shu-Osher problem on [-5, 5], transmissive boundaries."""
    q = projected_dofs(shu_osher_data, N, P, -5.0, 5.0, TRANSMISSIVE, (-4.5,))
    return Problem(EULER, N, P, -5.0, 5.0, TRANSMISSIVE, q, "shu-osher")


def random_smooth_dofs(ncells: int, nv: int, P: int, seed: int, scale: float = 1.0) -> np.ndarray:
    """Uniform random DOFs in [-scale, scale] (for unit-level checks)."""
    rng = np.random.default_rng(seed)
    return rng.uniform(-scale, scale, size=(ncells, nv, P + 1))


def batch_workload(count: int = 4096, n_min: int = 256, n_max: int = 65536, degrees=(2, 3),
                   seed: int = 2104043472) -> list:
    """Independent 1D Euler problems: N_i = round(exp(U(ln n_min, ln n_max)))
    (log-uniform), P_i drawn from `degrees` with equal probability, and 50/50
    either a seeded Riemann problem on [0, 1] (transmissive; its own states,
    drawn as in riemann_states) or the density wave on periodic [0, 1]."""
    rng = SplitMix64(seed)
    out = []
    lo, hi = math.log(n_min), math.log(n_max)
    for i in range(count):
        N = int(round(math.exp(rng.uniform(lo, hi))))
        P = degrees[int(rng.uniform(0.0, len(degrees)))]
        if rng.uniform() < 0.5:
            sub = rng.next_u64()
            left, right = riemann_states(sub)
            pr = euler_riemann(N, P, left, right, name=f"riemann-{i}")
        else:
            pr = euler_density_wave(N, P)
            pr.name = f"density-wave-{i}"
        out.append(pr)
    return out


# ------------------------------------------------------------------- 2D data
#
# 2D DOFs are the scaled derivatives u_{kx,ly} = dx^k dy^l d^k_x d^l_y u0 at
# every cell centre of the integer stage (Eq. 2DPolynomial_Space), k + l <= P,
# stored float64 [ny, nx, nv, nq] with nq = (P+1)(P+2)/2 and u_{kx,ly} at
# position (k+l)(k+l+1)/2 + l (by total degree, then by l).


def nq2d(P: int) -> int:
    return (P + 1) * (P + 2) // 2


def idx2d(k: int, l: int) -> int:
    d = k + l
    return d * (d + 1) // 2 + l


class Taylor2:
    """Truncated Taylor series in two variables (X, Y), one per point:
    ``c[k, l, ...]`` is the coefficient of X^k Y^l, kept for k + l <= P (the
    coefficient axes come first, so that every operation on one coefficient
    runs over contiguous memory).  Enough arithmetic (+, -, *, exp, real
    powers) to evaluate initial data and read off every mixed derivative at
    once: d^k_x d^l_y u = k! l! c_kl."""

    def __init__(self, c: np.ndarray, P: int):
        self.c = c
        self.P = P

    @staticmethod
    def variable(x0, which: int, P: int) -> "Taylor2":
        x0 = np.asarray(x0, dtype=np.float64)
        c = np.zeros((P + 1, P + 1) + x0.shape)
        c[0, 0] = x0
        if P >= 1:
            c[(1, 0)[which], (0, 1)[which]] = 1.0
        return Taylor2(c, P)

    def _lift(self, o) -> "Taylor2":
        if isinstance(o, Taylor2):
            return o
        c = np.zeros_like(self.c)
        c[0, 0] = o
        return Taylor2(c, self.P)

    def __add__(self, o):
        return Taylor2(self.c + self._lift(o).c, self.P)

    __radd__ = __add__

    def __neg__(self):
        return Taylor2(-self.c, self.P)

    def __sub__(self, o):
        return self + (-self._lift(o))

    def __rsub__(self, o):
        return self._lift(o) - self

    def __mul__(self, o):
        if not isinstance(o, Taylor2):
            return Taylor2(self.c * np.asarray(o), self.P)  # a number per point
        P = self.P
        a, b = self.c, o.c
        out = np.zeros((P + 1, P + 1) + np.broadcast_shapes(a.shape[2:], b.shape[2:]))
        for k in range(P + 1):
            for l in range(P + 1 - k):
                for i in range(k + 1):
                    for j in range(l + 1):
                        out[k, l] += a[i, j] * b[k - i, l - j]
        return Taylor2(out, P)

    __rmul__ = __mul__

    def _series(self, coef) -> "Taylor2":
        """sum_n coef[n] h^n with h = self - self(0), which vanishes to order
        P + 1 after P factors."""
        h = self - self.c[0, 0]
        term = self._lift(1.0)
        acc = term * coef[0]
        for n in range(1, self.P + 1):
            term = term * h
            acc = acc + term * coef[n]
        return acc

    def exp(self) -> "Taylor2":
        a0 = self.c[0, 0]
        return self._series([1.0 / math.factorial(n) for n in range(self.P + 1)]) * np.exp(a0)

    def pow(self, s: float) -> "Taylor2":
        a0 = self.c[0, 0]
        coef = []
        b = 1.0
        for n in range(self.P + 1):
            coef.append(b)
            b *= (s - n) / (n + 1)
        h = self * (1.0 / a0)  # (a0 + h)^s = a0^s (1 + h/a0)^s
        return h._series(coef) * a0 ** s

    def scaled_dofs(self, dx: float, dy: float) -> np.ndarray:
        """[..., nq] scaled derivatives dx^k dy^l d^k_x d^l_y."""
        P = self.P
        out = np.zeros(self.c.shape[2:] + (nq2d(P),))
        for k in range(P + 1):
            for l in range(P + 1 - k):
                out[..., idx2d(k, l)] = (self.c[k, l] * math.factorial(k) * math.factorial(l)
                                         * dx ** k * dy ** l)
        return out


@dataclass
class Problem2D:
    """A 2D workload: the law, mesh, boundary and integer-stage DOFs."""

    system: int
    nx: int
    ny: int
    P: int
    x_l: float
    x_r: float
    y_l: float
    y_r: float
    bc: int
    q0: np.ndarray  # [ny', nx', nv, nq]
    name: str = ""
    ax: float = 1.0
    ay: float = 1.0

    @property
    def dx(self) -> float:
        return (self.x_r - self.x_l) / self.nx

    @property
    def dy(self) -> float:
        return (self.y_r - self.y_l) / self.ny

    @property
    def nv(self) -> int:
        return 4 if self.system == EULER else 1


def _grid2d(nx, ny, x_l, x_r, y_l, y_r, bc, parity=0):
    x = centres(nx, x_l, x_r, bc, parity)
    y = centres(ny, y_l, y_r, bc, parity)
    return np.meshgrid(x, y)  # [ny, nx] each


VORTEX_STRENGTH = 5.0


def vortex_conserved(X, Y, gamma: float = GAMMA, psi: float = VORTEX_STRENGTH):
    """Isentropic vortex of Sec. 5.3 centred at the origin: rho = 1, p = 1,
    (u, v) = (1, 1) plus (du, dv) = psi/(2 pi) e^{(1 - r^2)/2} (-y, x),
    dT = -(gamma - 1) psi^2 / (8 gamma pi^2) e^{1 - r^2}, dS = 0 with
    T = p/rho, S = p/rho^gamma; so rho = T^{1/(gamma-1)}, p = rho T.
    X, Y may be arrays or Taylor2 series; returns (rho, rho u, rho v, E)."""
    r2 = X * X + Y * Y
    f = (0.5 - 0.5 * r2).exp() if isinstance(r2, Taylor2) else np.exp(0.5 * (1.0 - r2))
    k = psi / (2.0 * math.pi)
    u = 1.0 - k * (Y * f)
    v = 1.0 + k * (X * f)
    T = 1.0 - ((gamma - 1.0) * psi ** 2 / (8.0 * gamma * math.pi ** 2)) * (f * f)
    if isinstance(T, Taylor2):
        rho = T.pow(1.0 / (gamma - 1.0))
    else:
        rho = T ** (1.0 / (gamma - 1.0))
    p = rho * T
    m, n = rho * u, rho * v
    E = p * (1.0 / (gamma - 1.0)) + 0.5 * (m * u + n * v)
    return rho, m, n, E


def _wrap(z, lo, hi):
    return np.mod(z - lo, hi - lo) + lo


def vortex_exact(x, y, t, gamma: float = GAMMA):
    """Conserved variables of the exact solution at time t on periodic
    [-5, 5]^2: the vortex carried by the mean flow (1, 1)."""
    return vortex_conserved(_wrap(x - t, -5.0, 5.0), _wrap(y - t, -5.0, 5.0), gamma)


def isentropic_vortex(n: int, P: int, gamma: float = GAMMA) -> Problem2D:
    """Sec. 5.3: periodic [-5, 5]^2, n x n cells (mesh size 10/n)."""
    X, Y = _grid2d(n, n, -5.0, 5.0, -5.0, 5.0, PERIODIC)
    dx = 10.0 / n
    U = vortex_conserved(Taylor2.variable(X, 0, P), Taylor2.variable(Y, 1, P), gamma)
    q = np.stack([u.scaled_dofs(dx, dx) for u in U], axis=2)  # [ny, nx, 4, nq]
    return Problem2D(EULER, n, n, P, -5.0, 5.0, -5.0, 5.0, PERIODIC, q, "isentropic-vortex")


def advection2d_sine(nx: int, ny: int, P: int, ax: float = 1.0, ay: float = 1.0,
                     kx: float = math.pi, ky: float = math.pi, phase: float = 0.0) -> Problem2D:
    """u0 = sin(kx x + ky y + phase) on periodic [-1, 1]^2; f = ax u, g = ay u."""
    X, Y = _grid2d(nx, ny, -1.0, 1.0, -1.0, 1.0, PERIODIC)
    dx, dy = 2.0 / nx, 2.0 / ny
    q = np.zeros((ny, nx, 1, nq2d(P)))
    for k in range(P + 1):
        for l in range(P + 1 - k):
            q[:, :, 0, idx2d(k, l)] = (kx ** k * ky ** l * np.sin(kx * X + ky * Y + phase + (k + l) * math.pi / 2)
                                       * dx ** k * dy ** l)
    return Problem2D(ADVECTION, nx, ny, P, -1.0, 1.0, -1.0, 1.0, PERIODIC, q, "advection2d-sine", ax, ay)


# (rho, u, v, p) in the quadrants [-1,0]x[-1,0], [-1,0]x[0,1], [0,1]x[0,1], [0,1]x[-1,0]
RIEMANN2D_STATES = {
    1: ((0.138, 1.206, 1.206, 0.029), (0.5323, 1.206, 0.0, 0.3), (1.5, 0.0, 0.0, 1.5), (0.5323, 0.0, 1.206, 0.3)),
    2: ((1.0, -0.75, 0.5, 1.0), (2.0, 0.75, 0.5, 1.0), (1.0, 0.75, -0.5, 1.0), (3.0, -0.75, -0.5, 1.0)),
}


def riemann2d(n: int, P: int, config: int = 1, gamma: float = GAMMA) -> Problem2D:
    """The 2D Riemann problems of Sec. 5.3 on [-1, 1]^2 with transmissive
    boundaries, n x n cells: four constant quadrant states (config 1: four
    shocks; config 2: four contacts).  Each integer-stage cell holds the exact
    cell average of the data (cells cut by an axis the area-weighted mix) and
    zero derivatives."""
    X, Y = _grid2d(n, n, -1.0, 1.0, -1.0, 1.0, TRANSMISSIVE)
    d = 2.0 / n
    # fraction of each cell with x < 0 (resp. y < 0)
    fx = np.clip((0.0 - (X - 0.5 * d)) / d, 0.0, 1.0)
    fy = np.clip((0.0 - (Y - 0.5 * d)) / d, 0.0, 1.0)
    cons = [np.array(primitive_conserved2d(*s, gamma=gamma)) for s in RIEMANN2D_STATES[config]]
    U = (fx * fy)[..., None] * cons[0] + (fx * (1 - fy))[..., None] * cons[1] + \
        ((1 - fx) * (1 - fy))[..., None] * cons[2] + ((1 - fx) * fy)[..., None] * cons[3]
    q = np.zeros(X.shape + (4, nq2d(P)))
    q[..., 0] = U
    return Problem2D(EULER, n, n, P, -1.0, 1.0, -1.0, 1.0, TRANSMISSIVE, q, f"riemann2d-{config}")


def primitive_conserved2d(rho, u, v, p, gamma: float = GAMMA):
    return rho, rho * u, rho * v, p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v)
