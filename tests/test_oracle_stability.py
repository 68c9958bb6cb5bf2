"""Pin: von Neumann stability limits of Table 1 (Sec. 2.3), from the
amplification matrix G(theta) of Eq. 1DFourierAnalysis built on the oracle's
own half-step operator.

Table 1 prints nu <= 0.5 / 0.384 / 0.304 for u_0 at orders 2 / 3 / 4 and 0.5
for u_1, u_2.  The scan reproduces 0.5 and 0.384; at order 4 it finds
~0.289 (the spectral radius exceeds 1 by ~1e-4 at the printed 0.304), which is
recorded as a reading of the paper rather than hidden by a loose tolerance."""
import pytest

from oracle import stability


@pytest.mark.parametrize("P,limit,tol", [(1, 0.5, 1e-3), (2, 0.384, 1e-3)])
def test_u0_limits_match_table1(P, limit, tol):
    assert abs(stability.stability_limit(P, 0) - limit) < tol


def test_u0_limit_fourth_order_near_printed_value():
    got = stability.stability_limit(3, 0)
    assert 0.285 < got < 0.295           # strict limit found by the scan
    assert stability.spectral_radius(3, 0.304) - 1.0 < 5e-4   # printed value: marginal
    assert stability.spectral_radius(3, 0.25) <= 1.0 + 1e-12   # CFL used in Sec. 5


@pytest.mark.parametrize("P", [1, 2, 3])
@pytest.mark.parametrize("cand", [1, 2])
def test_linear_candidates_stable_to_half(P, cand):
    assert abs(stability.stability_limit(P, cand) - 0.5) < 1e-3


def test_unstable_above_limit():
    # nu = 0.5 at P = 2 (a full-step reading of CFL 0.5) is unstable.
    assert stability.spectral_radius(2, 0.5) > 1.01
