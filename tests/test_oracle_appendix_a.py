"""Pin: the oracle's linear half-step operator equals the printed matrices of
Appendix A (Eqs. 2ndOrderCoeMatrix) for P = 1, 2, 3, for the high-order
polynomial u_0 and for the two linear candidates u_1, u_2 (Eq. 1D_U012)."""
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle import stability


def _load(golden_dir):
    table = {}
    with open(os.path.join(golden_dir, "appendix_a_matrices.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            head, coeffs = line.split(":")
            P, name, r, c = head.split()
            table[(int(P), name, int(r), int(c))] = [float(Fraction(x)) for x in coeffs.split()]
    return table


def _printed(table, P, name, nu):
    nk = P + 1
    M = np.zeros((nk, nk))
    for (p, n, r, c), co in table.items():
        if p == P and n == name:
            M[r, c] = sum(ci * nu ** k for k, ci in enumerate(co))
    return M


@pytest.mark.parametrize("P", [1, 2, 3])
@pytest.mark.parametrize("nu", [0.1, 0.25, 0.37])
def test_half_step_matrices_match_appendix_a(golden_dir, P, nu):
    table = _load(golden_dir)
    for cand in (0, 1, 2):
        M1, M2 = stability.half_step_matrices(P, nu, candidate=cand)
        for s, M in ((1, M1), (2, M2)):
            expect = _printed(table, P, f"M{cand}{s}", nu)
            np.testing.assert_allclose(M, expect, rtol=0, atol=1e-14,
                                       err_msg=f"P={P} M{cand}{s} nu={nu}")


def test_fixture_is_complete(golden_dir):
    table = _load(golden_dir)
    for P in (1, 2, 3):
        for name in ("M01", "M02"):
            assert sum(1 for k in table if k[0] == P and k[1] == name) == (P + 1) ** 2
        for name in ("M11", "M12", "M21", "M22"):
            assert sum(1 for k in table if k[0] == P and k[1] == name) == 2 * (P + 1)
