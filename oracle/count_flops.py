"""Floating-point operation counts of the oracle's 1D half-step per
cell-update (TEST INFRASTRUCTURE ONLY, like the rest of oracle/).

Compiles wcc_oracle.c a second time, as C++, with ``double`` replaced by the
counting type of count_flops.cpp (the oracle's source is not changed), runs
one half-step of smooth data and prints one JSON line per (system, P):

  per_new_cell_as_written  every data-dependent operation of oracle_new_cell,
                           which builds both parents' Cauchy-Kovalewski
                           tables for every new cell;
  ck_table                 one Cauchy-Kovalewski table;
  per_cell_update          the first minus the second: the scheme's work
                           with each parent's table built once (each parent
                           is a vertex of two new cells, Sec. 2.1).

Divisions by constants, which the oracle writes as divisions, count as
divisions.  Usage: python oracle/count_flops.py [system P limiter ...]."""
from __future__ import annotations

import json
import os
import subprocess
import sys
import tempfile

HERE = os.path.dirname(os.path.abspath(__file__))


def build() -> str:
    exe = os.path.join(HERE, "_build", "count_flops")
    os.makedirs(os.path.dirname(exe), exist_ok=True)
    src = '#include "count_flops.cpp"\n#include "wcc_oracle.c"\n#include "count_flops.cpp"\n'
    with tempfile.NamedTemporaryFile("w", suffix=".cpp", delete=False) as f:
        f.write(src)
        tu = f.name
    try:
        subprocess.run(["g++", "-std=c++17", "-O1", "-w", "-ffp-contract=off", "-I", HERE, tu, "-o", exe, "-lm"],
                       check=True)
    finally:
        os.unlink(tu)
    return exe


def count(system: int, P: int, limiter: int = 1, exe: str | None = None) -> dict:
    exe = exe or build()
    out = subprocess.run([exe, str(system), str(P), str(limiter)], check=True, capture_output=True, text=True)
    return json.loads(out.stdout)


def flops(c: dict) -> float:
    """add + mul + div + sqrt + pow of a count (each one operation)."""
    return sum(c[k] for k in ("add", "mul", "div", "sqrt", "pow"))


if __name__ == "__main__":
    exe = build()
    args = [int(a) for a in sys.argv[1:]]
    cases = [tuple(args[i:i + 3]) for i in range(0, len(args), 3)] or [(2, 3, 1), (1, 3, 1), (2, 2, 1), (2, 4, 1)]
    for system, P, lim in cases:
        c = count(system, P, lim, exe)
        c["flops_per_cell_update"] = flops(c["per_cell_update"])
        print(json.dumps(c))
