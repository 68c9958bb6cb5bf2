"""Initial data of the paper's piecewise-smooth 1D workloads: the L2
projection used for their DOFs (paper_2104_04347_gb300.inputs.projected_dofs)
must reproduce polynomials of degree <= P, keep every cell's exact average,
and match the paper's definitions of the composite wave (Sec. 5.1) and the
modified Shu-Osher problem (Sec. 5.2)."""
import math

import numpy as np

from paper_2104_04347_gb300 import inputs


def _avg_weights(P):
    # cell average of the polynomial with scaled derivatives q_k: sum over even k of q_k / ((k+1)! 2^k)
    return np.array([1.0 / (math.factorial(k + 1) * 2.0 ** k) if k % 2 == 0 else 0.0 for k in range(P + 1)])


def test_polynomials_are_reproduced():
    # every DOF is exact up to rounding: q_k is formed from moments of size
    # |u| whose rounding (~1e-16 |u|) the Legendre-to-Taylor change of basis
    # and the factor k! amplify by about k! 4^k; a wrong coefficient anywhere
    # gives an O(1) error
    c = np.array([1.0, 2.0, 3.0, -1.0, 0.5])
    for N in (8, 400):
        for P in range(1, 5):
            poly = np.polynomial.Polynomial(c[:P + 1])
            q = inputs.projected_dofs(lambda x: poly(x)[:, None], N, P, 0.0, 1.0, inputs.PERIODIC)
            x = inputs.centres(N, 0.0, 1.0, inputs.PERIODIC)
            ref = inputs.smooth_dofs(lambda xx, k: poly.deriv(k)(xx) if k else poly(xx), x, 1.0 / N, P)
            tol = 1e-14 * np.max(np.abs(poly(x))) * np.array([math.factorial(k) * 4.0 ** k for k in range(P + 1)])
            assert np.all(np.max(np.abs(q[:, 0, :] - ref), axis=0) <= tol), (N, P)


def test_cell_averages_are_exact_for_piecewise_data():
    # composite wave at N = 400: compare each cell's average from the DOFs with
    # an independent fine midpoint-rule average of the data
    N, P = 400, 3
    pr = inputs.advection_composite(N, P)
    avg = pr.q0[:, 0, :] @ _avg_weights(P)
    dx = 2.0 / N
    edges = -1.0 + dx * (np.arange(N) - 0.5)
    m = 4000
    fine = (np.arange(m) + 0.5) / m
    pts = edges[:, None] + dx * fine[None, :]
    pts = np.where(pts < -1.0, pts + 2.0, pts)  # periodic wrap of the first cell's left half
    ref = inputs.composite_wave_data(pts.ravel())[:, 0].reshape(N, m).mean(axis=1)
    # the midpoint rule on 4000 points per cell is accurate to ~1e-8 here
    assert np.max(np.abs(avg - ref)) < 1e-7
    assert abs(avg.sum() - ref.sum()) < 1e-5


def test_composite_wave_matches_the_definition():
    x = np.array([-0.7, -0.3, 0.1, 0.5, 0.9, -0.9, 0.15])
    u = inputs.composite_wave_data(x)[:, 0]
    assert abs(u[0] - (math.exp(-math.log(2) / 36 / 0.005 ** 2 * 0.005 ** 2) * 2 + 4) / 6) < 1e-12  # Gaussians
    assert u[1] == 1.0 and abs(u[2] - 1.0) < 1e-15 and abs(u[3] - (2 * math.sqrt(1 - (10 * 0.005) ** 2) + 4) / 6) < 1e-12
    assert u[4] == 0.0 and u[5] == 0.0 and abs(u[6] - 0.5) < 1e-12


def test_shu_osher_states():
    U = inputs.shu_osher_data(np.array([-4.9, -4.5, 0.025]))
    gm1 = inputs.GAMMA - 1.0
    assert np.allclose(U[0], [1.515695, 1.515695 * 0.523346, 1.805 / gm1 + 0.5 * 1.515695 * 0.523346 ** 2])
    assert np.allclose(U[1], [1.0 + 0.1 * math.sin(20 * math.pi * -4.5), 0.0, 1.0 / gm1])
    assert np.allclose(U[2], [1.0 + 0.1 * math.sin(20 * math.pi * 0.025), 0.0, 1.0 / gm1])
    pr = inputs.shu_osher(200, 2)
    assert pr.q0.shape == (201, 3, 3) and pr.bc == inputs.TRANSMISSIVE
