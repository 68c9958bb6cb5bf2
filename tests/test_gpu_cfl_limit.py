"""CFL numbers above the linear stability limit of the degree (Sec. 2.3,
Table 1; wcc_stability_limit, the library's own von Neumann scan) are
refused with WCC_E_CFL before any half-step is taken: by wcc_step,
wcc_step_until, wcc_autotune, wcc_batch_step and wcc_advance_static.  The
limit itself is accepted, and the refused call leaves the handle as it was."""
import ctypes

import numpy as np
import pytest

from paper_2104_04347_gb300 import inputs, wcc

pytestmark = pytest.mark.gpu

E_CFL = -8


@pytest.mark.parametrize("precision", [wcc.FP64, wcc.FP32_MIXED])
@pytest.mark.parametrize("P", [1, 2, 3, 4, 5, 6])
def test_step_refuses_cfl_above_the_limit(P, precision):
    lim = wcc.stability_limit(P)
    pr = inputs.euler_density_wave(64, P)
    with wcc.Solver(pr.system, pr.N, P, (pr.x_l, pr.x_r), pr.bc, precision=precision) as s:
        s.set_initial(pr.q0)
        before = s.get_dofs()
        for call in (lambda: s.step(3, lim * (1 + 1e-9)), lambda: s.step_until(0.1, lim * 1.01),
                     lambda: s.autotune(lim * 1.5)):
            with pytest.raises(wcc.WCCError) as ei:
                call()
            assert ei.value.code == E_CFL
        assert s.state()[1] == 0 and np.array_equal(s.get_dofs(), before)
        s.step(2, lim)  # the limit itself is a valid CFL number
        assert s.state()[1] == 2


def test_batch_refuses_cfl_above_the_smaller_limit():
    probs = inputs.batch_workload(6, n_min=16, n_max=200, seed=4, degrees=(2, 3))
    lim = min(wcc.stability_limit(2), wcc.stability_limit(3))
    with wcc.Batch(probs) as b:
        b.set_initial()
        for call in (lambda: b.step(2, lim * 1.001), lambda: b.autotune(lim * 1.001)):
            with pytest.raises(wcc.WCCError) as ei:
                call()
            assert ei.value.code == E_CFL
        assert b.state() == (0, 0)
        b.step(2, lim)
        assert b.state() == (2, 0)


def test_static_entry_refuses_cfl_above_the_limit():
    torch = pytest.importorskip("torch")
    lib = wcc.load()
    a = torch.zeros((4, 128), dtype=torch.float64, device="cuda")
    b = torch.zeros_like(a)
    dom = (ctypes.c_double * 2)(0.0, 1.0)
    lim = wcc.stability_limit(3)
    rc = lib.wcc_advance_static(wcc.BURGERS, 3, wcc.PERIODIC, 64, dom, None, 0, ctypes.c_void_p(a.data_ptr()),
                                ctypes.c_void_p(b.data_ptr()), 128, 2, lim * 1.001, None)
    assert rc == E_CFL
