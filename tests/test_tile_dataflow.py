"""Host-side models of the FP32-mixed tiles (Sec. 2.1's staggered mesh): the
index arithmetic of `mixed_tile2` (one half-step) and `mixed_pair_tile` (two
half-steps per launch) replayed with the oracle's per-cell update must
reproduce oracle half-steps bit for bit.

One half-step: a tile owns the new cells f .. f + 2 T - 2 and reads the
parents f - p .. f - p + 2 T - 1 (slot s, through the boundary rule).  Thread
t holds slots t and t + T as a pair; the shared record row has T + 1 pairs,
the last one repeating slot T in both lanes, and new cell f + t (lane x) and
f + t + T (lane y, t < T - 1) are built from the pairs t and t + 1.

Two half-steps:
One tile owns the final cells f0 .. f0 + TILE - 1 (TILE = 2 T - 2 for T
threads with two cells each).  It reads the parents o0 = f0 - 1 ..
o0 + 2 T - 1 (wrapped or clamped at the boundary), builds the intermediate
cells m0 = o0 + p .. from neighbouring parent slots, replaces intermediate
slots outside a transmissive stage by the adjacent cell (the ghost rule), and
builds the final cells from neighbouring intermediate slots.  The thread
count is read from the kernel header, so the model follows the compiled
geometry.  Mesh sizes cover a few cells to two tiles, tile edges and both
stage parities."""
import os
import re

import numpy as np
import pytest

import oracle
from paper_2104_04347_gb300 import inputs

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                      "paper_2104_04347_gb300", "csrc", "wcc_mixed2.cuh")


def _geometry():
    text = open(HEADER).read()
    threads = int(re.search(r"#define WCC_MIXED_THREADS (\d+)", text).group(1))
    assert "constexpr int kTileMixed = 2 * kThreadsMixed - 1;" in text
    assert "constexpr int kTileTB = 2 * kThreadsMixed - 2;" in text
    assert "if (t == 0) r[kThreadsMixed] = make_float2(x.y(), x.y());" in text
    return threads, 2 * threads - 2


T, TILE = _geometry()


def _parent(idx, n, bc):
    if bc == inputs.PERIODIC:
        return idx % n
    return min(max(idx, 0), n - 1)


def _two_halfsteps_by_tiles(law, q, p, lam, bc):
    n_old = q.shape[0]
    n_mid = oracle.new_count(law, p, n_old)
    n_new = oracle.new_count(law, p ^ 1, n_mid)
    out = np.full((n_new,) + q.shape[1:], np.nan)
    writes = np.zeros(n_new, dtype=int)
    for b in range((n_new + TILE - 1) // TILE):
        f0 = b * TILE
        o0 = f0 - 1
        m0 = o0 + p
        par = [q[_parent(o0 + s, n_old, bc)] for s in range(2 * T)]
        # slot 2 T - 1 has no right neighbour; no final cell reads it
        mid = [np.asarray(oracle.new_cell(law, par[s], par[s + 1], lam)).reshape(q.shape[1:])
               for s in range(2 * T - 1)] + [par[2 * T - 1]]
        if bc == inputs.TRANSMISSIVE and (m0 < 0 or m0 + 2 * T - 1 > n_mid):
            mid = [mid[min(max(m0 + s, 0), n_mid - 1) - m0] for s in range(2 * T)]
        for s in range(TILE):
            if f0 + s < n_new:
                out[f0 + s] = oracle.new_cell(law, mid[s], mid[s + 1], lam)
                writes[f0 + s] += 1
    assert np.all(writes == 1)
    return out


def _one_halfstep_by_tiles(law, q, p, lam, bc):
    n_old = q.shape[0]
    n_new = oracle.new_count(law, p, n_old)
    tile = 2 * T - 1
    out = np.full((n_new,) + q.shape[1:], np.nan)
    writes = np.zeros(n_new, dtype=int)   # every cell written by exactly one thread lane
    for b in range((n_new + tile - 1) // tile):
        f = b * tile
        slot = [q[_parent(f - p + s, n_old, bc)] for s in range(2 * T)]
        rec = [(slot[t], slot[t + T]) for t in range(T)] + [(slot[T], slot[T])]
        for t in range(T):
            if f + t < n_new:
                out[f + t] = oracle.new_cell(law, rec[t][0], rec[t + 1][0], lam)
                writes[f + t] += 1
            if t < T - 1 and f + t + T < n_new:
                out[f + t + T] = oracle.new_cell(law, rec[t][1], rec[t + 1][1], lam)
                writes[f + t + T] += 1
    assert np.all(writes == 1)
    return out


def _rough_states(n, P, seed):
    """Euler DOFs that differ from cell to cell up to the boundary (rho and p
    in [1, 1.3], u in [-0.25, 0.25], small derivatives), so that a wrong
    ghost cell or parent slot changes the result."""
    rng = np.random.default_rng(seed)
    q = np.zeros((n, 3, P + 1))
    q[:, :, 0] = inputs.primitive_to_conserved(1.0 + 0.3 * rng.random(n), 0.5 * (rng.random(n) - 0.5),
                                               1.0 + 0.3 * rng.random(n))
    q[:, :, 1:] = 0.01 * (rng.random((n, 3, P)) - 0.5)
    return q


@pytest.mark.parametrize("bc", [inputs.TRANSMISSIVE, inputs.PERIODIC], ids=["transmissive", "periodic"])
@pytest.mark.parametrize("N", [4, 5, 6, 253, 254, 255, 256, 508, 510])
def test_pair_tiles_equal_two_halfsteps(bc, N):
    P = 3
    q0 = _rough_states(inputs.num_cells(N, bc, 0), P, seed=N)
    law = oracle.make_law(oracle.EULER, P, limiter=True, bc=bc)
    lam = 0.05
    for p in (0, 1):
        q = q0 if p == 0 else oracle.halfstep(law, 0, q0, lam)
        want = oracle.halfstep(law, p ^ 1, oracle.halfstep(law, p, q, lam), lam)
        got = _two_halfsteps_by_tiles(law, q, p, lam, bc)
        assert got.shape == want.shape
        assert np.array_equal(got, want), (N, p)


@pytest.mark.parametrize("bc", [inputs.TRANSMISSIVE, inputs.PERIODIC], ids=["transmissive", "periodic"])
@pytest.mark.parametrize("N", [4, 5, 126, 127, 128, 254, 255, 256, 509, 510, 511])
def test_halfstep_tiles_equal_one_halfstep(bc, N):
    P = 3
    q0 = _rough_states(inputs.num_cells(N, bc, 0), P, seed=1000 + N)
    law = oracle.make_law(oracle.EULER, P, limiter=True, bc=bc)
    lam = 0.05
    for p in (0, 1):
        q = q0 if p == 0 else oracle.halfstep(law, 0, q0, lam)
        want = oracle.halfstep(law, p, q, lam)
        got = _one_halfstep_by_tiles(law, q, p, lam, bc)
        assert got.shape == want.shape
        assert np.array_equal(got, want), (N, p)
