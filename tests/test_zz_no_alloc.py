"""The allocation-free entry point wcc_advance_static, checked against the
handle-based wcc_step on the same input, over two calls in a row.

wcc_advance_static serves callers that cannot allocate device memory when
they step (their own allocator owns the device pool, or they must avoid the
synchronisation an allocation can cause): the caller owns the two stage
buffers, and the kernels' scratch lives in a fixed array inside the library.
Both routes run the same FP64 half-step kernels with the same arguments, so
their results and half-step sizes are compared bit for bit; the stage
buffers are filled and read with the same FP64 scalings (1/k! and k!) as the
handle's own layout conversion.

This file is named so that pytest collects it last."""
import ctypes
import math

import numpy as np
import pytest

from paper_2104_04347_gb300 import inputs, wcc

pytestmark = pytest.mark.gpu

MAX_HALFSTEPS = 4096  # WCC_STATIC_MAX_HALFSTEPS in include/wcc.h
E_INVAL, E_CAPACITY = -1, -7


def _to_planes(q, pitch):
    """[cells, nv, P+1] paper DOFs -> [nv*(P+1), pitch] Taylor-coefficient planes."""
    cells, nv, K = q.shape
    out = np.zeros((nv * K, pitch))
    for v in range(nv):
        for k in range(K):
            out[v * K + k, :cells] = q[:, v, k] * (1.0 / math.factorial(k))
    return out


def _from_planes(planes, cells, nv, K):
    q = np.empty((cells, nv, K))
    for v in range(nv):
        for k in range(K):
            q[:, v, k] = planes[v * K + k, :cells] * float(math.factorial(k))
    return q


def _advance(lib, system, P, bc, N, domain, parity, a, b, pitch, nsteps, cfl):
    dts = np.zeros(max(nsteps, 1))
    dom = (ctypes.c_double * 2)(*domain)
    rc = lib.wcc_advance_static(system, P, bc, N, dom, None, parity, ctypes.c_void_p(a.data_ptr()),
                                ctypes.c_void_p(b.data_ptr()), pitch, nsteps, cfl,
                                dts.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    return rc, dts[:nsteps]


# (problem, P, half-steps of the first and the second call).  The first call
# starts on an integer stage (parity 0); with an odd count its result is in
# stage_b on a half stage, and the second call starts from there (parity 1).
CASES = [
    ("euler-riemann-transmissive", lambda: inputs.euler_riemann_seeded(1000, 3), 33, 31),
    ("burgers-periodic", lambda: inputs.burgers_fourier(1000, 2), 17, 16),
    ("euler-riemann-even", lambda: inputs.euler_riemann_seeded(1000, 3), 40, 40),
    ("euler-density-wave-p6", lambda: inputs.euler_density_wave(500, 6), 9, 12),
]


@pytest.mark.parametrize("name,make,n1,n2", CASES, ids=[c[0] for c in CASES])
def test_static_entry_matches_wcc_step_two_calls(name, make, n1, n2):
    torch = pytest.importorskip("torch")
    lib = wcc.load()
    pr = make()
    N, P = pr.N, pr.P
    cfl = 0.2 if P <= 4 else 0.14  # below the linear stability limit of P = 6 (0.185)
    nv, K = pr.q0.shape[1], P + 1
    pitch = (N + 1 + 63) // 64 * 64
    bufs = [torch.tensor(_to_planes(pr.q0, pitch), dtype=torch.float64, device="cuda"),
            torch.zeros((nv * K, pitch), dtype=torch.float64, device="cuda")]
    torch.cuda.synchronize()
    cur, parity = 0, 0
    with wcc.Solver(pr.system, N, P, (pr.x_l, pr.x_r), pr.bc) as ref:
        ref.set_initial(pr.q0)
        done = 0
        for nsteps in (n1, n2):
            rc, dts = _advance(lib, pr.system, P, pr.bc, N, (pr.x_l, pr.x_r), parity, bufs[cur], bufs[cur ^ 1],
                               pitch, nsteps, cfl)
            assert rc == 0, rc
            # the stages alternate a -> b -> a ...: an odd count ends in stage_b
            cur ^= nsteps & 1
            parity ^= nsteps & 1
            ref.step(nsteps, cfl)
            want = ref.get_dofs()
            got = _from_planes(bufs[cur].cpu().numpy(), want.shape[0], nv, K)
            assert ref.state()[2] == parity
            assert np.array_equal(dts, ref.dt_history()[done:done + nsteps])
            assert np.array_equal(got, want)
            done += nsteps


def test_static_entry_rejects_sizes_beyond_its_limits():
    torch = pytest.importorskip("torch")
    lib = wcc.load()
    a = torch.zeros((4, 128), dtype=torch.float64, device="cuda")
    b = torch.zeros_like(a)
    rc, _ = _advance(lib, wcc.BURGERS, 3, wcc.PERIODIC, 64, (0.0, 1.0), 0, a, b, 128, MAX_HALFSTEPS + 1, 0.2)
    assert rc == E_CAPACITY
    rc, _ = _advance(lib, wcc.BURGERS, 3, wcc.PERIODIC, (1 << 31) + 1, (0.0, 1.0), 0, a, b, 1 << 32, 2, 0.2)
    assert rc == E_INVAL
    rc, _ = _advance(lib, wcc.BURGERS, 3, wcc.PERIODIC, 64, (0.0, 1.0), 0, a, b, 64, 2, 0.2)
    assert rc == E_INVAL  # pitch < N + 1
    rc, _ = _advance(lib, wcc.BURGERS, 7, wcc.PERIODIC, 64, (0.0, 1.0), 0, a, b, 128, 2, 0.2)
    assert rc == E_INVAL  # P above 6
    # the context stays usable: a valid call after the rejected ones
    rc, _ = _advance(lib, wcc.BURGERS, 3, wcc.PERIODIC, 64, (0.0, 1.0), 0, a, b, 128, 0, 0.2)
    assert rc == 0
