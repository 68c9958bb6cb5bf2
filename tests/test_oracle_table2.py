"""Pin: the whole oracle (linear scheme and limiter) against Table 2 of the
paper (Sec. 5.1): advection of sin(pi x) on periodic [-1, 1] to t = 2.

Readings fixed here: dt is the half step and nu = a dt/dx (Table 1 caption);
CFL 0.4 / 0.3 / 0.25 for P = 1 / 2 / 3 (Sec. 5); t_end is met by the largest
even number of CFL half-steps plus two equal half-steps; L1 / Linf are the
mean / max error of the cell-centre point values (u_0x) against the exact
translate; alpha = 2 at P = 1."""
import math
import os

import numpy as np
import pytest

import oracle
from paper_2104_04347_gb300 import inputs

CFL = {1: 0.4, 2: 0.3, 3: 0.25}


def _rows(golden_dir):
    rows = []
    with open(os.path.join(golden_dir, "table2_advection.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                s, P, inv, l1, linf = line.split()
                rows.append((s, int(P), int(inv), float(l1), float(linf)))
    return rows


def _run(P, limiter, inv):
    N = 2 * inv
    pr = inputs.advection_sine(N, P)
    law = oracle.make_law(oracle.ADVECTION, P, limiter=limiter)
    s = oracle.Solver(law, pr.q0, pr.dx)
    s.step_dt(oracle.constant_speed_dts(2.0, CFL[P] * pr.dx))
    assert s.parity == 0 and abs(s.t - 2.0) < 1e-12
    x = inputs.centres(N, -1.0, 1.0, inputs.PERIODIC)
    err = np.abs(s.q[:, 0, 0] - np.sin(math.pi * (x - s.t)))
    return err.mean(), err.max()


def test_table2(golden_dir):
    rows = _rows(golden_dir)
    assert len(rows) == 24
    for scheme, P, inv, l1, linf in rows:
        got1, gotinf = _run(P, scheme == "WCCS", inv)
        # 3 % on the finer meshes; the coarsest mesh (dx = 1/25) is more
        # sensitive to how t_end is reached and gets 10 %.
        tol = 0.10 if inv == 25 else 0.03
        assert abs(got1 / l1 - 1) < tol, (scheme, P, inv, got1, l1)
        assert abs(gotinf / linf - 1) < tol, (scheme, P, inv, gotinf, linf)


@pytest.mark.parametrize("P", [1, 2, 3])
def test_convergence_order(P):
    e = [_run(P, False, inv)[0] for inv in (50, 100, 200)]
    orders = [math.log2(e[i] / e[i + 1]) for i in range(2)]
    for o in orders:
        assert abs(o - (P + 1)) < 0.05


def test_fourth_order_p4():
    # P = 4 is not in the paper; the scheme should still reach order 5 at
    # nu = 0.2 (inside the scanned stability limit ~0.28).
    def run(inv):
        N = 2 * inv
        pr = inputs.advection_sine(N, 4)
        s = oracle.Solver(oracle.make_law(oracle.ADVECTION, 4, limiter=False), pr.q0, pr.dx)
        s.step_dt(oracle.constant_speed_dts(2.0, 0.2 * pr.dx))
        x = inputs.centres(N, -1.0, 1.0, inputs.PERIODIC)
        return np.abs(s.q[:, 0, 0] - np.sin(math.pi * (x - s.t))).mean()
    e1, e2 = run(25), run(50)
    assert abs(math.log2(e1 / e2) - 5) < 0.2
