"""Writes tests/golden/stability_limits.txt: the von Neumann limits of the
linear scheme (Sec. 2.3, Eq. LinearStabilityCondition) for P = 1..6 from the
oracle's own half-step operator, and the CFL number the tests use at P >= 5
(0.8 of the limit, rounded down to two digits; the paper gives no CFL for
P > 3).  Calls only oracle/."""
import math
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import stability  # noqa: E402


def main():
    lines = ["# P  u0_limit  cfl  (von Neumann limit of the linear scheme, Sec. 2.3; cfl = floor(80 * limit) / 100)"]
    for P in range(1, 7):
        lim = stability.stability_limit(P, 0)
        lines.append(f"{P} {lim:.6f} {math.floor(80.0 * lim) / 100.0:.2f}")
    with open(os.path.join(HERE, "stability_limits.txt"), "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
