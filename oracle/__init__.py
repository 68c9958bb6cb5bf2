"""Plain FP64 CPU oracle for the WCC half-step (Shen & Parsani, arXiv 2104.04347),
1D (Sec. 2, 4) and 2D (Sec. 3, 4, Appendix B).

TEST INFRASTRUCTURE ONLY.  This package is imported by ``tests/``,
``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference`` legs
of ``bench.py`` -- nothing in the product package imports it, and it imports
nothing from the product package.  It shares no kernel, header, table or helper
with the CUDA path; the only code both sides see is the seeded initial-data
generator module, which holds none of the scheme's arithmetic.

The arithmetic lives in ``wcc_oracle.c`` (1D) and ``wcc_oracle2d.c`` (2D),
compiled here with ``gcc -O2 -ffp-contract=off``.  This module loads it through ``ctypes`` and
adds the time loop (Sec. 2.1: alternating integer / half stages) and the
CFL step rule.  Parity status of every function is stated in its docstring;
pins live in ``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRCS = [os.path.join(_HERE, "wcc_oracle.c"), os.path.join(_HERE, "wcc_oracle2d.c")]
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")

ADVECTION, BURGERS, EULER = 0, 1, 2
PERIODIC, TRANSMISSIVE = 0, 1

_lock = threading.Lock()
_lib = None


class Law(ctypes.Structure):
    """Mirror of ``or_law`` in wcc_oracle.c."""

    _fields_ = [
        ("system", ctypes.c_int),
        ("P", ctypes.c_int),
        ("limiter", ctypes.c_int),
        ("bc", ctypes.c_int),
        ("a", ctypes.c_double),
        ("gamma", ctypes.c_double),
        ("alpha", ctypes.c_double),
        ("eps", ctypes.c_double),
    ]


def build(force: bool = False) -> str:
    """Compile the oracle sources into oracle/_build/liboracle.so (gcc, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and all(os.path.getmtime(_LIB_PATH) >= os.path.getmtime(src) for src in _SRCS)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC", "-shared",
           "-std=c11", "-o", tmp, *_SRCS, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    """Load (building first if needed) the oracle shared library."""
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            dp = ctypes.POINTER(ctypes.c_double)
            lp = ctypes.POINTER(Law)
            L.oracle_new_cell.argtypes = [lp, dp, dp, ctypes.c_double, dp, dp, dp, dp]
            L.oracle_new_cell.restype = None
            L.oracle_halfstep.argtypes = [lp, ctypes.c_int, ctypes.c_long, dp, dp,
                                          ctypes.c_double, dp]
            L.oracle_halfstep.restype = ctypes.c_long
            L.oracle_new_count.argtypes = [lp, ctypes.c_int, ctypes.c_long]
            L.oracle_new_count.restype = ctypes.c_int
            L.oracle_max_speed.argtypes = [lp, ctypes.c_long, dp]
            L.oracle_max_speed.restype = ctypes.c_double
            L.oracle_ck_table.argtypes = [lp, dp, ctypes.c_double, dp, dp]
            L.oracle_ck_table.restype = None
            L.oracle_smoothness.argtypes = [dp, ctypes.c_int]
            L.oracle_smoothness.restype = ctypes.c_double
            L.oracle_euler_eigenvectors.argtypes = [ctypes.c_double, dp, dp, dp]
            L.oracle_euler_eigenvectors.restype = None
            lp2 = ctypes.POINTER(Law2D)
            L.oracle2d_new_cell.argtypes = [lp2, dp, dp, dp, dp, ctypes.c_double, ctypes.c_double, dp, dp, dp, dp]
            L.oracle2d_new_cell.restype = None
            L.oracle2d_parent_terms.argtypes = [lp2, dp, ctypes.c_double, ctypes.c_double, dp, dp, dp]
            L.oracle2d_parent_terms.restype = None
            L.oracle2d_ck_table.argtypes = [lp2, dp, ctypes.c_double, ctypes.c_double, dp, dp, dp]
            L.oracle2d_ck_table.restype = None
            L.oracle2d_smoothness.argtypes = [dp, ctypes.c_int]
            L.oracle2d_smoothness.restype = ctypes.c_double
            L.oracle2d_euler_eigenvectors.argtypes = [ctypes.c_double, dp, ctypes.c_double, ctypes.c_double, dp, dp]
            L.oracle2d_euler_eigenvectors.restype = None
            L.oracle2d_new_count.argtypes = [lp2, ctypes.c_int, ctypes.c_long]
            L.oracle2d_new_count.restype = ctypes.c_long
            L.oracle2d_halfstep.argtypes = [lp2, ctypes.c_int, ctypes.c_long, ctypes.c_long, dp, dp,
                                            ctypes.c_double, ctypes.c_double, dp]
            L.oracle2d_halfstep.restype = ctypes.c_long
            L.oracle2d_max_speeds.argtypes = [lp2, ctypes.c_long, dp, ctypes.c_double, ctypes.c_double, dp]
            L.oracle2d_max_speeds.restype = None
            L.oracle_set_threads.argtypes = [ctypes.c_int]
            L.oracle_get_threads.restype = ctypes.c_int
            _lib = L
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def nvars(system: int) -> int:
    return 3 if system == EULER else 1


def make_law(system: int, P: int, *, limiter: bool = True, bc: int = PERIODIC, a: float = 1.0,
             gamma: float = 1.4, alpha: float = 2.0, eps: float = 1e-40) -> Law:
    """Scheme options.  alpha = 2 and eps = 1e-40 follow Sec. 2.2 (alpha for
    P = 1 is not stated in the paper; 2 is the reading that reproduces Table 2)."""
    return Law(system, P, 1 if limiter else 0, bc, a, gamma, alpha, eps)


def set_threads(n: int) -> None:
    lib().oracle_set_threads(int(n))


def get_threads() -> int:
    return int(lib().oracle_get_threads())


def new_cell(law: Law, qL, qR, lam: float, *, diagnostics: bool = False):
    """One new staggered cell from its two parents (Eqs. SubEq:1DIntegral,
    Cal1DFlux, Cal_1D_Derivatives_2, 1DCalU and the limiter of Sec. 2.2 / 4).

    qL, qR: [nv, P+1] paper-scaled DOFs.  Returns the new [nv, P+1] DOFs, and
    with ``diagnostics`` also (candidates [3, nv, P+1], weights [nv, 3],
    ubar [nv])."""
    nv, nk = nvars(law.system), law.P + 1
    qL = np.ascontiguousarray(qL, dtype=np.float64).reshape(nv * nk)
    qR = np.ascontiguousarray(qR, dtype=np.float64).reshape(nv * nk)
    out = np.zeros(nv * nk)
    cand = np.zeros(3 * nv * nk)
    w = np.zeros(nv * 3)
    ub = np.zeros(nv)
    lib().oracle_new_cell(ctypes.byref(law), _dp(qL), _dp(qR), float(lam), _dp(out), _dp(cand),
                          _dp(w), _dp(ub))
    out = out.reshape(nv, nk)
    if diagnostics:
        return out, cand.reshape(3, nv, nk), w.reshape(nv, 3), ub
    return out


def ck_table(law: Law, q, lam: float):
    """Scaled Cauchy-Kovalewski table (Eq. 1DCauchy_Kovalewski; Sec. 4):
    returns U, F of shape [nv, P+1, P+1], entry (a, b) = dx^a dt^b d_x^a d_t^b."""
    nv, nk = nvars(law.system), law.P + 1
    q = np.ascontiguousarray(q, dtype=np.float64).reshape(nv * nk)
    U = np.zeros(nv * nk * nk)
    F = np.zeros(nv * nk * nk)
    lib().oracle_ck_table(ctypes.byref(law), _dp(q), float(lam), _dp(U), _dp(F))
    return U.reshape(nv, nk, nk), F.reshape(nv, nk, nk)


def smoothness(c) -> float:
    """Jiang-Shu smoothness indicator of Eq. 1DSmoothIndicator in scaled form."""
    c = np.ascontiguousarray(c, dtype=np.float64)
    return float(lib().oracle_smoothness(_dp(c), len(c) - 1))


def euler_eigenvectors(gamma: float, U):
    """Right (columns) and left eigenvector matrices of the Euler Jacobian at U."""
    U = np.ascontiguousarray(U, dtype=np.float64)
    R = np.zeros(9)
    L = np.zeros(9)
    lib().oracle_euler_eigenvectors(float(gamma), _dp(U), _dp(R), _dp(L))
    return R.reshape(3, 3), L.reshape(3, 3)


def new_count(law: Law, parity: int, n_old: int) -> int:
    return int(lib().oracle_new_count(ctypes.byref(law), int(parity), int(n_old)))


def halfstep(law: Law, parity: int, old: np.ndarray, lam: float, *, weights: bool = False):
    """One half-step over a whole stage; old is [cells, nv, P+1]."""
    nv, nk = nvars(law.system), law.P + 1
    old = np.ascontiguousarray(old, dtype=np.float64)
    n_old = old.shape[0]
    n_new = new_count(law, parity, n_old)
    out = np.empty((n_new, nv, nk))
    w = np.empty((n_new, nv, 3)) if weights else None
    r = lib().oracle_halfstep(ctypes.byref(law), int(parity), n_old, _dp(old), _dp(out),
                              float(lam), _dp(w) if weights else None)
    if r < 0:
        raise ValueError("oracle_halfstep rejected its arguments")
    return (out, w) if weights else out


def max_speed(law: Law, q: np.ndarray) -> float:
    """Largest characteristic speed over the centre point values of a stage."""
    q = np.ascontiguousarray(q, dtype=np.float64)
    return float(lib().oracle_max_speed(ctypes.byref(law), q.shape[0], _dp(q)))


class Solver:
    """Time loop of Sec. 2.1 over the oracle's half-step.

    ``parity`` is 0 when the current stage is an integer stage (cells centred
    on x_L + i dx) and 1 on a half stage.  ``step_cfl`` takes
    dt = cfl * dx / amax with amax over the current stage (the CFL number is
    the paper's nu of Table 1, defined with the half step); ``step_dt``
    replays a given list of half-step sizes."""

    def __init__(self, law: Law, q0: np.ndarray, dx: float, parity: int = 0, t: float = 0.0):
        self.law = law
        self.q = np.ascontiguousarray(q0, dtype=np.float64).copy()
        self.dx = float(dx)
        self.parity = int(parity)
        self.t = float(t)
        self.dts: list[float] = []

    def _advance(self, dt: float) -> None:
        self.q = halfstep(self.law, self.parity, self.q, dt / self.dx)
        self.parity ^= 1
        self.t += dt
        self.dts.append(dt)

    def step_cfl(self, nsteps: int, cfl: float) -> None:
        for _ in range(int(nsteps)):
            amax = max_speed(self.law, self.q)
            self._advance(cfl * self.dx / amax)

    def step_dt(self, dts) -> None:
        for dt in dts:
            self._advance(float(dt))


def constant_speed_dts(t_end: float, dt_cfl: float) -> list[float]:
    """Half-step sizes that reach t_end exactly on an integer stage when the
    wave speed is constant: the largest even number of CFL steps that fits,
    then the remainder split into two equal half-steps.  (The paper does not
    say how t_end is hit; this reading reproduces Table 2.)"""
    n = int(np.floor(t_end / dt_cfl + 1e-12))
    if n % 2:
        n -= 1
    dts = [dt_cfl] * n
    rem = t_end - n * dt_cfl
    if rem > 1e-14 * max(1.0, t_end):
        dts += [0.5 * rem, 0.5 * rem]
    return dts


# ------------------------------------------------------------------ 2D (Sec. 3)


class Law2D(ctypes.Structure):
    """Mirror of ``o2_law`` in wcc_oracle2d.c."""

    _fields_ = [
        ("system", ctypes.c_int),
        ("P", ctypes.c_int),
        ("limiter", ctypes.c_int),
        ("bc", ctypes.c_int),
        ("ax", ctypes.c_double),
        ("ay", ctypes.c_double),
        ("gamma", ctypes.c_double),
        ("alpha", ctypes.c_double),
        ("eps", ctypes.c_double),
    ]


def nvars2d(system: int) -> int:
    return 4 if system == EULER else 1


def nq2d(P: int) -> int:
    """DOFs per variable of a 2D cell: the scaled derivatives u_{kx,ly}, k + l <= P."""
    return (P + 1) * (P + 2) // 2


def idx2d(k: int, l: int) -> int:
    """Position of u_{kx,ly} among a variable's DOFs: by total degree, then by l."""
    d = k + l
    return d * (d + 1) // 2 + l


def make_law2d(system: int, P: int, *, limiter: bool = True, bc: int = PERIODIC, ax: float = 1.0,
               ay: float = 1.0, gamma: float = 1.4, alpha: float = 2.0, eps: float = 1e-40) -> Law2D:
    """2D scheme options (alpha and eps as in 1D, Sec. 2.2 / 3.2)."""
    return Law2D(system, P, 1 if limiter else 0, bc, ax, ay, gamma, alpha, eps)


def new_cell2d(law: Law2D, q1, q2, q3, q4, lamx: float, lamy: float, *, diagnostics: bool = False):
    """One new staggered cell from its four parents, in the vertex order of
    Eq. 2DTaylorSeries: 1 lower left, 2 lower right, 3 upper right, 4 upper
    left (each [nv, nq]).  Returns the new [nv, nq] DOFs; with
    ``diagnostics`` also (weights [nv, 5], ubar [nv], normal [2])."""
    nv, nq = nvars2d(law.system), nq2d(law.P)
    qs = [np.ascontiguousarray(q, dtype=np.float64).reshape(nv * nq) for q in (q1, q2, q3, q4)]
    out = np.zeros(nv * nq)
    w = np.zeros(nv * 5)
    ub = np.zeros(nv)
    nrm = np.zeros(2)
    lib().oracle2d_new_cell(ctypes.byref(law), *[_dp(q) for q in qs], float(lamx), float(lamy), _dp(out),
                            _dp(w), _dp(ub), _dp(nrm))
    out = out.reshape(nv, nq)
    if diagnostics:
        return out, w.reshape(nv, 5), ub, nrm
    return out


def parent_terms2d(law: Law2D, q, lamx: float, lamy: float):
    """What one old cell contributes (Appendix B, Eq. SubEq:2DUij): quarter
    averages [nv, 4] (RU, RD, LU, LD), time-averaged edge fluxes [nv, 4]
    (f_U, f_D, g_R, g_L) and the scaled derivatives at t^{n+1/2} [nv, nq]."""
    nv, nq = nvars2d(law.system), nq2d(law.P)
    q = np.ascontiguousarray(q, dtype=np.float64).reshape(nv * nq)
    qa, fl, V = np.zeros(nv * 4), np.zeros(nv * 4), np.zeros(nv * nq)
    lib().oracle2d_parent_terms(ctypes.byref(law), _dp(q), float(lamx), float(lamy), _dp(qa), _dp(fl), _dp(V))
    return qa.reshape(nv, 4), fl.reshape(nv, 4), V.reshape(nv, nq)


def ck_table2d(law: Law2D, q, lamx: float, lamy: float):
    """Scaled 2D Cauchy-Kovalewski tables U, F, G of one cell, each
    [nv, P+1, P+1, P+1], entry (k, l, m) = dx^k dy^l dt^m d^k_x d^l_y d^m_t."""
    nv, nq, nk = nvars2d(law.system), nq2d(law.P), law.P + 1
    q = np.ascontiguousarray(q, dtype=np.float64).reshape(nv * nq)
    U, F, G = (np.zeros(nv * nk ** 3) for _ in range(3))
    lib().oracle2d_ck_table(ctypes.byref(law), _dp(q), float(lamx), float(lamy), _dp(U), _dp(F), _dp(G))
    shape = (nv, nk, nk, nk)
    return U.reshape(shape), F.reshape(shape), G.reshape(shape)


def smoothness2d(c, P: int) -> float:
    """Smoothness indicator of Eq. 2DSmoothIndicator in scaled form; c holds
    nq2d(P) DOFs."""
    c = np.ascontiguousarray(c, dtype=np.float64)
    return float(lib().oracle2d_smoothness(_dp(c), int(P)))


def euler_eigenvectors2d(gamma: float, U, nx: float, ny: float):
    """Right (columns) and left eigenvectors of cos(theta) dF/dU + sin(theta) dG/dU."""
    U = np.ascontiguousarray(U, dtype=np.float64)
    R, L = np.zeros(16), np.zeros(16)
    lib().oracle2d_euler_eigenvectors(float(gamma), _dp(U), float(nx), float(ny), _dp(R), _dp(L))
    return R.reshape(4, 4), L.reshape(4, 4)


def new_count2d(law: Law2D, parity: int, n_old: int) -> int:
    return int(lib().oracle2d_new_count(ctypes.byref(law), int(parity), int(n_old)))


def halfstep2d(law: Law2D, parity: int, old: np.ndarray, lamx: float, lamy: float, *, weights: bool = False):
    """One 2D half-step over a whole stage; old is [ny, nx, nv, nq]."""
    nv, nq = nvars2d(law.system), nq2d(law.P)
    old = np.ascontiguousarray(old, dtype=np.float64)
    ny_old, nx_old = old.shape[:2]
    nx_new, ny_new = new_count2d(law, parity, nx_old), new_count2d(law, parity, ny_old)
    out = np.empty((ny_new, nx_new, nv, nq))
    w = np.empty((ny_new, nx_new, nv, 5)) if weights else None
    r = lib().oracle2d_halfstep(ctypes.byref(law), int(parity), nx_old, ny_old, _dp(old), _dp(out), float(lamx),
                                float(lamy), _dp(w) if weights else None)
    if r < 0:
        raise ValueError("oracle2d_halfstep rejected its arguments")
    return (out, w) if weights else out


def max_speeds2d(law: Law2D, q: np.ndarray, dx: float, dy: float):
    """(max s_x, max s_y, max over cells of s_x/dx + s_y/dy) over the centre
    point values of a stage, s the characteristic speed along each axis."""
    q = np.ascontiguousarray(q, dtype=np.float64)
    out = np.zeros(3)
    lib().oracle2d_max_speeds(ctypes.byref(law), q.shape[0] * q.shape[1], _dp(q), float(dx), float(dy), _dp(out))
    return float(out[0]), float(out[1]), float(out[2])


def cfl_dt2d(law: Law2D, q: np.ndarray, dx: float, dy: float, cfl: float) -> float:
    """Half-step size dt = cfl / max over cells of (s_x/dx + s_y/dy): the 2D
    CFL bound read for Sec. 5.3 (the paper does not spell it out)."""
    return cfl / max_speeds2d(law, q, dx, dy)[2]


class Solver2D:
    """Time loop of Sec. 3.1 over the 2D oracle half-step (alternating
    integer and half stages, as in 1D)."""

    def __init__(self, law: Law2D, q0: np.ndarray, dx: float, dy: float, parity: int = 0, t: float = 0.0):
        self.law = law
        self.q = np.ascontiguousarray(q0, dtype=np.float64).copy()
        self.dx, self.dy = float(dx), float(dy)
        self.parity = int(parity)
        self.t = float(t)
        self.dts: list[float] = []

    def _advance(self, dt: float) -> None:
        self.q = halfstep2d(self.law, self.parity, self.q, dt / self.dx, dt / self.dy)
        self.parity ^= 1
        self.t += dt
        self.dts.append(dt)

    def cfl_dt(self, cfl: float) -> float:
        return cfl_dt2d(self.law, self.q, self.dx, self.dy, cfl)

    def step_cfl(self, nsteps: int, cfl: float) -> None:
        for _ in range(int(nsteps)):
            self._advance(self.cfl_dt(cfl))

    def step_dt(self, dts) -> None:
        for dt in dts:
            self._advance(float(dt))

    def step_until(self, t_end: float, cfl: float) -> None:
        """Reach t_end on an integer stage: CFL half-steps in pairs while a
        pair fits, then the rest in two equal half-steps (the 1D reading of
        how t_end is hit, applied pair by pair)."""
        if self.parity != 0:
            raise ValueError("step_until starts on an integer stage")
        while True:
            left = t_end - self.t
            if left <= 1e-14 * max(1.0, abs(t_end)):
                return
            dt = self.cfl_dt(cfl)
            if left >= 2.0 * dt * (1.0 - 1e-12):
                self._advance(dt)
                left2 = t_end - self.t
                dt2 = self.cfl_dt(cfl)
                if left2 >= dt2 * (1.0 - 1e-12):
                    self._advance(dt2)
                else:
                    self._advance(left2)
                    return
            else:
                self._advance(0.5 * left)
                self._advance(t_end - self.t)
                return
