"""Plain FP64 CPU oracle for the 1D WCC half-step (Shen & Parsani, arXiv 2104.04347).

TEST INFRASTRUCTURE ONLY.  This package is imported by ``tests/``,
``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference`` legs
of ``bench.py`` -- nothing in the product package imports it, and it imports
nothing from the product package.  It shares no kernel, header, table or helper
with the CUDA path; the only code both sides see is the seeded initial-data
generator module, which holds none of the scheme's arithmetic.

The arithmetic lives in ``wcc_oracle.c`` (compiled here with
``gcc -O2 -ffp-contract=off``).  This module loads it through ``ctypes`` and
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
_SRC = os.path.join(_HERE, "wcc_oracle.c")
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
    """Compile wcc_oracle.c into oracle/_build/liboracle.so (gcc, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC", "-shared",
           "-std=c11", "-o", tmp, _SRC, "-lm"]
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
