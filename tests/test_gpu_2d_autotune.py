"""wcc2d_autotune: the strip height (rows_per_cta) timed on the handle's own
stage.  The tuner must put the stage, time, step count and dt history back,
keep the chosen height, and -- the strip height only changes how the new
rows are split among CTAs -- later half-steps must equal bit for bit those of
a handle created with that height, in every precision and boundary."""
import numpy as np
import pytest

from paper_2104_04347_gb300 import inputs, wcc
from tests.test_gpu_2d import CFL, EULER, _problem

pytestmark = pytest.mark.gpu

ROWS = {8, 10, 12, 13, 14, 15, 16, 17, 18, 19, 20, 22, 24}


def _solver(pr, precision, rows):
    return wcc.Solver2D(pr.system, pr.nx, pr.ny, pr.P, (pr.x_l, pr.x_r, pr.y_l, pr.y_r), pr.bc,
                        precision=precision, ax=pr.ax, ay=pr.ay, rows_per_cta=rows)


@pytest.mark.parametrize("precision", [wcc.FP32_MIXED, wcc.FP32, wcc.FP64])
@pytest.mark.parametrize("bc", [inputs.PERIODIC, inputs.TRANSMISSIVE])
def test_autotune_restores_the_state_and_keeps_results(precision, bc):
    P = 3
    pr = _problem(EULER, 150, 150 if bc == inputs.PERIODIC else 131, P, bc)
    with _solver(pr, precision, 16) as s:
        s.set_initial(pr.q0)
        s.step(5, CFL[P])
        before, state, dts = s.get_dofs(), s.state(), s.dt_history()
        rows = s.autotune(CFL[P])
        assert rows in ROWS
        assert np.array_equal(s.get_dofs(), before)
        assert s.state() == state
        assert np.array_equal(s.dt_history(), dts)
        s.step(12, CFL[P])
        qa, da = s.get_dofs(), s.dt_history()
    with _solver(pr, precision, rows) as r:
        r.set_initial(pr.q0)
        r.step(17, CFL[P])
        qb, db = r.get_dofs(), r.dt_history()
    assert np.array_equal(da, db)
    assert np.array_equal(qa, qb)


def test_autotune_needs_a_loaded_stage():
    pr = _problem(EULER, 32, 32, 2, inputs.PERIODIC)
    with _solver(pr, wcc.FP32_MIXED, 16) as s:
        with pytest.raises(wcc.WCCError) as ei:
            s.autotune(0.3)
        assert ei.value.code == -2
        s.set_initial(pr.q0)
        with pytest.raises(wcc.WCCError):
            s.autotune(-1.0)
        assert s.autotune(0.3) in ROWS
