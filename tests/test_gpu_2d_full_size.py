"""GPU parity of the 2D path at the size and in the launch configuration of
the 2D bench: the isentropic vortex of Sec. 5.3 on 2048 x 2048 periodic
cells, Euler, P = 3 (WCCS-4, rotated characteristic limiter on), 16 new rows
per CTA, CFL half-steps at nu = 0.25.  The whole-stage oracle would take
minutes at this size, so

* sampled new cells (the first and last columns of the FP64, FP32-mixed and
  FP32 strips, the rows where one CTA's strip hands over to the next, the
  periodic seams, random cells) are checked one by one against the oracle's
  new cell from its four parents, the parents read back from the GPU's own
  stage, within max(tol x scale, 50 x the oracle's spread when the parents
  carry relative noise): tol 1e-11 with 4e-16 noise for FP64, 2e-6 with
  1e-7 noise for FP32-mixed, both parities.  Plain FP32 (every value in
  float) is compared in L1 per variable over the samples, within
  max(2e-7, 50 x the oracle's L1 spread), as in the FP32 tests at small
  sizes: its limiter weights can switch on rounding-level slopes, so single
  entries are not compared;
* the CFL half-step equals the oracle's CFL step of the whole stage;
* over one bench step (8 half-steps) the FP32-mixed path keeps the summed
  cell averages to float-float rounding.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2104_04347_gb300 import inputs, wcc
from tests.gpu_common import sampled_new_cells2d

pytestmark = pytest.mark.gpu

N, P, CFL, ROWS, HALFSTEPS = 2048, 3, 0.25, 16, 8


@pytest.fixture(scope="module")
def vortex():
    return inputs.isentropic_vortex(N, P)


def _cells(seed):
    edges = {0, 1, N - 2, N - 1}
    for w in (63, 95, 127):  # new columns per strip: FP64, FP32-mixed, FP32
        for k in (1, 2, 7, N // w):
            edges |= {k * w - 1, k * w, k * w + 1}
    cols = sorted(c for c in edges if 0 <= c < N)
    rows = sorted({0, 1, ROWS - 1, ROWS, ROWS + 1, 5 * ROWS, 64 * ROWS - 1, 64 * ROWS, N - 2, N - 1})
    rng = np.random.default_rng(seed)
    rand = [(int(j), int(i)) for j, i in rng.integers(0, N, size=(300, 2))]
    return [(j, i) for j in rows for i in cols] + rand


def _check(law, prev, got, parity, lx, ly, tol, noise, seed, entrywise=True):
    cells = _cells(seed)
    want = sampled_new_cells2d(law, prev, parity, cells, lx, ly)
    rng = np.random.default_rng(seed + 1)
    g = np.array([got[j, i] for j, i in cells])
    sc = np.max(np.abs(prev[:, :, :, 0]), axis=(0, 1))[None, :, None]
    if not entrywise:  # L1 per variable over the samples
        spread = np.zeros(want.shape[1])
        for _ in range(3):
            pert = sampled_new_cells2d(law, prev, parity, cells, lx, ly, rng=rng, noise=noise)
            spread = np.maximum(spread, np.mean(np.abs(pert - want) / sc, axis=(0, 2)))
        l1 = np.mean(np.abs(g - want) / sc, axis=(0, 2))
        ratio = float(np.max(l1 / np.maximum(tol, 50.0 * spread)))
        assert ratio <= 1.0, (parity, l1, spread, ratio)
        return
    spread = np.zeros_like(want)
    for _ in range(3):
        pert = sampled_new_cells2d(law, prev, parity, cells, lx, ly, rng=rng, noise=noise)
        spread = np.maximum(spread, np.abs(pert - want))
    ratio = np.abs(g - want) / np.maximum(tol * sc, 50.0 * spread)
    k = int(np.argmax(ratio.max(axis=(1, 2))))
    assert float(ratio.max()) <= 1.0, (parity, cells[k], float(ratio.max()))


@pytest.mark.parametrize("precision", [wcc.FP64, wcc.FP32_MIXED, wcc.FP32])
def test_sampled_cells_at_full_size(vortex, precision):
    pr = vortex
    law = oracle.make_law2d(oracle.EULER, P, limiter=True)
    tol, noise, dt_tol = {wcc.FP64: (1e-11, 4e-16, 1e-12), wcc.FP32_MIXED: (2e-6, 1e-7, 1e-5),
                          wcc.FP32: (2e-7, 1e-7, 1e-5)}[precision]
    with wcc.Solver2D(pr.system, N, N, P, (pr.x_l, pr.x_r, pr.y_l, pr.y_r), pr.bc, precision=precision,
                      rows_per_cta=ROWS) as s:
        s.set_initial(pr.q0)
        prev = s.get_dofs()  # the stage as the GPU holds it
        for parity in (0, 1):
            s.step(1, CFL)
            dt = s.dt_history()[-1]
            want_dt = oracle.cfl_dt2d(law, prev, pr.dx, pr.dy, CFL)
            assert abs(dt - want_dt) <= dt_tol * want_dt, (parity, dt, want_dt)
            got = s.get_dofs()
            assert got.shape == prev.shape
            assert np.all(np.isfinite(got))
            _check(law, prev, got, parity, dt / pr.dx, dt / pr.dy, tol, noise, 100 * precision + parity,
                   entrywise=precision != wcc.FP32)
            prev = got


def test_mixed_conserves_over_a_bench_step(vortex):
    pr = vortex
    w = np.zeros(inputs.nq2d(P))
    for k in range(0, P + 1, 2):
        for l in range(0, P + 1 - k, 2):
            w[inputs.idx2d(k, l)] = 1.0 / (math.factorial(k + 1) * 2 ** k * math.factorial(l + 1) * 2 ** l)
    with wcc.Solver2D(pr.system, N, N, P, (pr.x_l, pr.x_r, pr.y_l, pr.y_r), pr.bc, precision=wcc.FP32_MIXED,
                      rows_per_cta=ROWS) as s:
        s.set_initial(pr.q0)
        m0 = (s.get_dofs() @ w).sum(axis=(0, 1))
        s.step(HALFSTEPS, CFL)
        assert s.state()[1] == HALFSTEPS
        m1 = (s.get_dofs() @ w).sum(axis=(0, 1))
    assert np.max(np.abs(m1 - m0) / np.abs(m0)) <= 1e-11, (m0, m1)
