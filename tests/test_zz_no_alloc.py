"""The allocation-free entry point wcc_advance_static, checked against the
handle-based wcc_step on the same input, over two calls in a row.

wcc_advance_static serves callers that cannot allocate device memory when
they step (their own allocator owns the device pool, or they must avoid the
synchronisation an allocation can cause): the caller owns the two stage
buffers, and the kernels' scratch lives in a fixed array inside the library.
This file is named so that pytest collects it last."""
import ctypes
import math

import numpy as np
import pytest

from paper_2104_04347_gb300 import inputs, wcc
from tests.gpu_common import TOL64, scaled_error

pytestmark = pytest.mark.gpu

MAX_HALFSTEPS = 4096  # WCC_STATIC_MAX_HALFSTEPS in include/wcc.h


def _to_planes(q, pitch):
    """[cells, nv, P+1] paper DOFs -> [nv*(P+1), pitch] Taylor-coefficient planes."""
    cells, nv, K = q.shape
    out = np.zeros((nv * K, pitch))
    for v in range(nv):
        for k in range(K):
            out[v * K + k, :cells] = q[:, v, k] / math.factorial(k)
    return out


def _from_planes(planes, cells, nv, K):
    q = np.empty((cells, nv, K))
    for v in range(nv):
        for k in range(K):
            q[:, v, k] = planes[v * K + k, :cells] * math.factorial(k)
    return q


def test_static_entry_matches_wcc_step_two_calls():
    torch = pytest.importorskip("torch")
    lib = wcc.load()
    N, P, nsteps, cfl = 1000, 3, 40, 0.2
    pr = inputs.euler_riemann_seeded(N, P)
    pitch = (N + 1 + 63) // 64 * 64
    a = torch.tensor(_to_planes(pr.q0, pitch), dtype=torch.float64, device="cuda")
    b = torch.zeros_like(a)
    torch.cuda.synchronize()
    dom = (ctypes.c_double * 2)(pr.x_l, pr.x_r)
    dp = ctypes.POINTER(ctypes.c_double)

    with wcc.Solver(pr.system, N, P, (pr.x_l, pr.x_r), pr.bc) as ref:
        ref.set_initial(pr.q0)
        for call in range(2):
            dts = np.zeros(nsteps)
            rc = lib.wcc_advance_static(wcc.EULER, P, wcc.TRANSMISSIVE, N, dom, None, 0,
                                        ctypes.c_void_p(a.data_ptr()), ctypes.c_void_p(b.data_ptr()),
                                        pitch, nsteps, cfl, dts.ctypes.data_as(dp))
            assert rc == 0, rc
            # nsteps is even: the result is back in stage a
            got = _from_planes(a.cpu().numpy(), N + 1, 3, P + 1)
            ref.step(nsteps, cfl)
            want = ref.get_dofs()
            want_dts = ref.dt_history()[call * nsteps:(call + 1) * nsteps]
            np.testing.assert_allclose(dts, want_dts, rtol=1e-15, atol=0)
            assert scaled_error(got, want) <= TOL64


def test_static_entry_rejects_too_many_halfsteps():
    torch = pytest.importorskip("torch")
    lib = wcc.load()
    N = 64
    a = torch.zeros((4, 128), dtype=torch.float64, device="cuda")
    b = torch.zeros_like(a)
    dom = (ctypes.c_double * 2)(0.0, 1.0)
    rc = lib.wcc_advance_static(wcc.BURGERS, 3, wcc.PERIODIC, N, dom, None, 0, ctypes.c_void_p(a.data_ptr()),
                                ctypes.c_void_p(b.data_ptr()), 128, MAX_HALFSTEPS + 1, 0.2, None)
    assert rc == -7  # WCC_E_CAPACITY
