"""The documented maximum sizes on the device.  A mesh at the maximum whose
state cannot fit in device memory is refused by create with WCC_E_NOMEM
before any kernel runs (the first stage allocation already fails), and the
CUDA context stays usable: a small solver created right afterwards steps
and matches the oracle.

* 1D: N = 2^31 (the maximum), Euler, P = 6, FP64: 2 stages of 361 GB.
* 2D: 2^15 x 2^15 cells (the maximum), Euler, P = 3, FP64: 2 stages of 344 GB.
"""
import numpy as np
import pytest

import oracle
from paper_2104_04347_gb300 import inputs, wcc
from tests.gpu_common import gpu_solver, scales

pytestmark = pytest.mark.gpu


def _small_step_matches_the_oracle():
    pr = inputs.euler_riemann_seeded(300, 3)
    law = oracle.make_law(oracle.EULER, 3, limiter=True, bc=oracle.TRANSMISSIVE)
    dt = 0.1 * pr.dx / oracle.max_speed(law, pr.q0)
    with gpu_solver(pr) as s:
        s.set_initial(pr.q0)
        s.step_dt([dt])
        got = s.get_dofs()
    want = oracle.halfstep(law, 0, pr.q0, dt / pr.dx)
    assert float(np.max(np.abs(got - want) / scales(want)[None, :, None])) <= 1e-11


def test_1d_maximum_n_beyond_memory_is_refused():
    with pytest.raises(wcc.WCCError) as ei:
        wcc.Solver(inputs.EULER, 1 << 31, 6, (0.0, 1.0), inputs.TRANSMISSIVE, precision=wcc.FP64)
    assert ei.value.code == -3, ei.value
    _small_step_matches_the_oracle()


def test_2d_maximum_mesh_beyond_memory_is_refused():
    n = 1 << 15
    with pytest.raises(wcc.WCCError) as ei:
        wcc.Solver2D(inputs.EULER, n, n, 3, (-1.0, 1.0, -1.0, 1.0), inputs.TRANSMISSIVE, precision=wcc.FP64)
    assert ei.value.code == -3, ei.value
    _small_step_matches_the_oracle()
