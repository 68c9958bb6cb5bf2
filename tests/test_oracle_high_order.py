"""Pins of the 1D oracle at P = 5 and 6 ("arbitrarily high order", Sec. 1 and
Sec. 2.1; the paper's tables stop at P = 3).

* The von Neumann limits of the linear scheme (Sec. 2.3) match the stored
  scan, the scheme is stable at the CFL numbers used here and unstable just
  above the limit.
* Order P + 1 on smooth data: advection of sin(pi x) (exact translate) and the
  Euler density wave (exact translate), with and without the limiter.
* The invariant and closed-form pins of the lower degrees, at P = 5, 6:
  polynomial data advected exactly, conservation, flat data, the limiter's
  weights and cell mean, mirror symmetry, the Euler CK on the translating
  density wave, the Burgers CK against brute-force differentiation.
"""
import math
import os

import numpy as np
import pytest

import oracle
from oracle import stability
from paper_2104_04347_gb300 import inputs

import tests.test_oracle_ck as ck_pins
import tests.test_oracle_invariants as inv_pins

HIGH = [5, 6]


def limits(golden_dir):
    out = {}
    with open(os.path.join(golden_dir, "stability_limits.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                P, lim, cfl = line.split()
                out[int(P)] = (float(lim), float(cfl))
    return out


@pytest.mark.parametrize("P", HIGH)
def test_stability_limit_and_cfl(golden_dir, P):
    lim, cfl = limits(golden_dir)[P]
    assert abs(stability.stability_limit(P, 0) - lim) < 1e-6
    assert stability.spectral_radius(P, cfl) <= 1.0 + 1e-12
    assert stability.spectral_radius(P, 1.05 * lim) > 1.0 + 1e-6
    for cand in (1, 2):  # the linear candidates of the limiter stay stable to 1/2
        assert abs(stability.stability_limit(P, cand) - 0.5) < 1e-3


def _orders(errs, Ns):
    return [math.log(errs[i] / errs[i + 1]) / math.log(Ns[i + 1] / Ns[i]) for i in range(len(errs) - 1)]


@pytest.mark.parametrize("P", HIGH)
def test_advection_order(golden_dir, P):
    cfl = limits(golden_dir)[P][1]
    Ns = (14, 20, 28, 40)
    errs = []
    for N in Ns:
        pr = inputs.advection_sine(N, P)
        s = oracle.Solver(oracle.make_law(oracle.ADVECTION, P, limiter=False), pr.q0, pr.dx)
        s.step_dt(oracle.constant_speed_dts(2.0, cfl * pr.dx))
        x = inputs.centres(N, -1.0, 1.0, inputs.PERIODIC)
        errs.append(float(np.mean(np.abs(s.q[:, 0, 0] - np.sin(math.pi * (x - s.t))))))
    o = _orders(errs, Ns)
    assert all(P + 1 - 0.15 < oi < P + 1 + 0.6 for oi in o), (errs, o)


@pytest.mark.parametrize("limiter", [False, True])
@pytest.mark.parametrize("P", HIGH)
def test_euler_density_wave_order(golden_dir, P, limiter):
    cfl = limits(golden_dir)[P][1]
    amax = 1.0 + math.sqrt(1.4 / 0.8)
    Ns = (16, 24, 32, 48)
    errs = []
    for N in Ns:
        pr = inputs.euler_density_wave(N, P)
        s = oracle.Solver(oracle.make_law(oracle.EULER, P, limiter=limiter), pr.q0, pr.dx)
        s.step_dt(oracle.constant_speed_dts(1.0, cfl * pr.dx / amax))
        x = inputs.centres(N, 0.0, 1.0, inputs.PERIODIC)
        errs.append(float(np.mean(np.abs(s.q[:, 0, 0] - (1.0 + 0.2 * np.sin(2 * math.pi * (x - 1.0)))))))
    o = _orders(errs, Ns)
    assert all(P + 1 - 0.15 < oi < P + 1 + 0.9 for oi in o), (errs, o)


@pytest.mark.parametrize("P", HIGH)
def test_lower_degree_pins_hold_at_high_order(P):
    inv_pins.test_polynomial_data_advected_exactly(P)
    inv_pins.test_flat_data_unchanged(P)
    inv_pins.test_conservation_periodic_burgers(P, True)
    inv_pins.test_conservation_periodic_euler(P)
    for system in (oracle.BURGERS, oracle.EULER):
        inv_pins.test_limiter_weights_and_mean(system, P)
        inv_pins.test_mirror_symmetry(P, system)
    ck_pins.test_euler_density_wave_translation(P)


def test_burgers_ck_brute_force_p5():
    # sympy differentiation of u^2/2 through the PDE (seconds at P = 5)
    ck_pins.test_burgers_ck_brute_force(5)
