"""Von Neumann analysis of the linear compact central scheme (Sec. 2.3).

Test infrastructure only.  The half-step matrices M_1, M_2 of
Eq. 1DSchemeMatrixForm are read off the oracle itself by applying one
half-step of linear advection (a = 1, limiter off) to unit DOF vectors of
the left and right parent; the candidate maps of Eq. 1D_U012 come from the
oracle's candidate diagnostics.  G(theta) = M_1 e^{-i theta/2} +
M_2 e^{i theta/2} (Eq. 1DFourierAnalysis) and the scheme is linearly stable
when the spectral radius of G is at most 1 for every theta
(Eq. LinearStabilityCondition).
"""
from __future__ import annotations

import numpy as np

from . import ADVECTION, make_law, new_cell


def half_step_matrices(P: int, nu: float, candidate: int = 0):
    """(M_1, M_2) for candidate polynomial u_0, u_1 or u_2 at CFL nu."""
    law = make_law(ADVECTION, P, limiter=False, a=1.0)
    nk = P + 1
    M1 = np.zeros((nk, nk))
    M2 = np.zeros((nk, nk))
    zero = np.zeros((1, nk))
    for j in range(nk):
        e = np.zeros((1, nk))
        e[0, j] = 1.0
        _, candL, _, _ = new_cell(law, e, zero, nu, diagnostics=True)
        _, candR, _, _ = new_cell(law, zero, e, nu, diagnostics=True)
        M1[:, j] = candL[candidate, 0]
        M2[:, j] = candR[candidate, 0]
    return M1, M2


def spectral_radius(P: int, nu: float, candidate: int = 0, ntheta: int = 2048) -> float:
    M1, M2 = half_step_matrices(P, nu, candidate)
    theta = np.linspace(0.0, 2 * np.pi, ntheta, endpoint=False)[1:]
    G = (M1[None] * np.exp(-0.5j * theta)[:, None, None]
         + M2[None] * np.exp(0.5j * theta)[:, None, None])
    return float(np.max(np.abs(np.linalg.eigvals(G))))


def stability_limit(P: int, candidate: int = 0, tol: float = 1e-9, hi: float = 1.0) -> float:
    """Largest nu in (0, hi] with spectral radius <= 1 + tol, by bisection
    (assumes the stable set is an interval starting at 0)."""
    lo = 1e-3
    if spectral_radius(P, lo, candidate) > 1.0 + tol:
        return 0.0
    for _ in range(40):
        mid = 0.5 * (lo + hi)
        if spectral_radius(P, mid, candidate) <= 1.0 + tol:
            lo = mid
        else:
            hi = mid
    return lo
