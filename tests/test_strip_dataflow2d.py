"""Host-side model of the 2D half-step's strip marching (Sec. 3.1's staggered
mesh): the index arithmetic of `halfstep2d` / `halfstep2d_mx` replayed with
the oracle's per-cell update must reproduce the oracle's 2D half-step bit for
bit.

The launch grid has ceil(nx_new / (TW - 1)) x ceil(ny_new / R) CTAs for
strips of TW threads and R rows.  CTA (bx, by) starts at new column
i0 = bx (TW - 1) and new row j0 = by R.  Thread t owns parent column
i0 + t + off (off = -1 on an odd stage, through the boundary rule).  For
s = 0 .. min(R, ny_new - j0) it expands parent row j0 + off + s into ring
row s mod 2.  From s = 1 on, threads t < TW - 1 with i0 + t < nx_new build new
cell (j0 + s - 1, i0 + t) from the ring.  Its parents are, in the vertex
order 1..4 (lower left, lower right, upper right, upper left), columns t,
t + 1 of ring row s - 1 and columns t + 1, t of ring row s.

The geometry does not depend on the strip width or height, so narrow strips
and short heights on small meshes cover many strips, ragged last strips and
both boundaries cheaply.  The widths and heights the kernels use run on a
mesh wider than one strip."""
import numpy as np
import pytest

import oracle
from paper_2104_04347_gb300 import inputs

P = 2


def _parent(j, n, bc):
    if bc == inputs.PERIODIC:
        return j % n
    return min(max(j, 0), n - 1)


def _halfstep_by_strips(law, q, parity, lamx, lamy, bc, tw, rows):
    ny_old, nx_old = q.shape[:2]
    nx_new, ny_new = oracle.new_count2d(law, parity, nx_old), oracle.new_count2d(law, parity, ny_old)
    off = -1 if parity else 0
    out = np.full((ny_new, nx_new) + q.shape[2:], np.nan)
    writes = np.zeros((ny_new, nx_new), dtype=int)
    for by in range((ny_new + rows - 1) // rows):
        for bx in range((nx_new + tw - 2) // (tw - 1)):
            i0, j0 = bx * (tw - 1), by * rows
            cols = [_parent(i0 + t + off, nx_old, bc) for t in range(tw)]
            ring = [None, None]
            for s in range(min(rows, ny_new - j0) + 1):
                pr = _parent(j0 + off + s, ny_old, bc)
                ring[s & 1] = [q[pr, c] for c in cols]
                if s == 0:
                    continue
                lo, hi = ring[(s - 1) & 1], ring[s & 1]
                for t in range(tw - 1):
                    if i0 + t < nx_new:
                        out[j0 + s - 1, i0 + t] = oracle.new_cell2d(law, lo[t], lo[t + 1], hi[t + 1], hi[t],
                                                                    lamx, lamy)
                        writes[j0 + s - 1, i0 + t] += 1
    assert np.all(writes == 1)
    return out


def _rough_states(ny, nx, seed):
    """2D Euler DOFs that differ from cell to cell up to the boundary."""
    rng = np.random.default_rng(seed)
    shape = (ny, nx)
    rho = 1.0 + 0.3 * rng.random(shape)
    u, v = 0.5 * (rng.random(shape) - 0.5), 0.5 * (rng.random(shape) - 0.5)
    p = 1.0 + 0.3 * rng.random(shape)
    q = np.zeros(shape + (4, oracle.nq2d(P)))
    q[..., 0, 0] = rho
    q[..., 1, 0] = rho * u
    q[..., 2, 0] = rho * v
    q[..., 3, 0] = p / (inputs.GAMMA - 1.0) + 0.5 * rho * (u * u + v * v)
    q[..., 1:] = 0.01 * (rng.random(shape + (4, oracle.nq2d(P) - 1)) - 0.5)
    return q


def _stage(n, bc):
    return n + 1 if bc == inputs.TRANSMISSIVE else n


@pytest.mark.parametrize("bc", [inputs.TRANSMISSIVE, inputs.PERIODIC], ids=["transmissive", "periodic"])
@pytest.mark.parametrize("nx,ny", [(4, 6), (9, 5), (13, 11)])
@pytest.mark.parametrize("tw,rows", [(3, 1), (3, 4), (5, 2), (8, 3), (32, 7)])
def test_strips_equal_the_halfstep(bc, nx, ny, tw, rows):
    law = oracle.make_law2d(oracle.EULER, P, limiter=True, bc=bc)
    q0 = _rough_states(_stage(ny, bc), _stage(nx, bc), seed=100 * nx + ny)
    lamx, lamy = 0.04, 0.03
    for parity in (0, 1):
        q = q0 if parity == 0 else oracle.halfstep2d(law, 0, q0, lamx, lamy)
        want = oracle.halfstep2d(law, parity, q, lamx, lamy)
        got = _halfstep_by_strips(law, q, parity, lamx, lamy, bc, tw, rows)
        assert got.shape == want.shape
        assert np.array_equal(got, want), (parity, tw, rows)


@pytest.mark.parametrize("tw,rows", [(64, 16), (96, 19), (128, 16)])
def test_kernel_strip_shapes(tw, rows):
    # the kernels' strip widths (FP64 64, FP32-mixed Euler 96, FP32 128) and
    # the default and tuned heights, on a mesh of two strips and a ragged third
    bc = inputs.TRANSMISSIVE
    law = oracle.make_law2d(oracle.EULER, P, limiter=True, bc=bc)
    nx, ny = 2 * (tw - 1) + 5, rows + 3
    q0 = _rough_states(_stage(ny, bc), _stage(nx, bc), seed=tw)
    for parity in (0, 1):
        q = q0 if parity == 0 else oracle.halfstep2d(law, 0, q0, 0.04, 0.03)
        want = oracle.halfstep2d(law, parity, q, 0.04, 0.03)
        assert np.array_equal(_halfstep_by_strips(law, q, parity, 0.04, 0.03, bc, tw, rows), want)
