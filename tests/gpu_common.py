"""Helpers shared by the GPU parity tests: run a problem through the C ABI
and through the oracle with the same half-step sizes, and the parity bound.

Parity bound (FP64).  The target is max |gpu - oracle| <= 1e-11 x (scale of
each variable).  The WENO-type limiter of Sec. 2.2 is ill-conditioned where a
one-sided slope s_m is close to zero: the weight (sigma tau / s_m^4)^2 then
amplifies rounding differences, so two correct FP64 implementations that
round differently drift apart by far more than 1e-11 near discontinuities
(the oracle itself, fed inputs perturbed by a few ulps, scatters by up to
~6e-5 after 100 half-steps of Euler P = 2 Riemann data).  The bound is
therefore per cell:
    |gpu - oracle| <= max(1e-11 x scale_v, SCATTER_FACTOR x spread)
where spread is the largest deviation of the oracle from itself over a few
runs whose inputs are perturbed by PERTURB relative noise.  Where the scheme
is well conditioned the spread is ~1e-14 and the 1e-11 bound applies as is.
"""
import numpy as np

import oracle
from paper_2104_04347_gb300 import inputs, wcc

TOL64 = 1e-11
PERTURB = 4e-16
SCATTER_FACTOR = 50.0
TRIALS = 4


def gpu_solver(pr, *, limiter=True, precision=wcc.FP64, graph_chunk=32, stream=None, adv_speed=1.0):
    return wcc.Solver(pr.system, pr.N, pr.P, (pr.x_l, pr.x_r), pr.bc, precision=precision, limiter=limiter,
                      graph_chunk=graph_chunk, stream=stream, adv_speed=adv_speed)


def gpu_run(pr, nsteps, cfl, *, limiter=True, precision=wcc.FP64, graph_chunk=32, dts=None, stream=None,
            adv_speed=1.0):
    with gpu_solver(pr, limiter=limiter, precision=precision, graph_chunk=graph_chunk, stream=stream,
                    adv_speed=adv_speed) as s:
        s.set_initial(pr.q0)
        if dts is None:
            s.step(nsteps, cfl)
        else:
            s.step_dt(dts)
        q = s.get_dofs()
        t, k, parity = s.state()
        hist = s.dt_history()
    return q, hist, t, parity


def law_of(pr, limiter=True, adv_speed=1.0):
    return oracle.make_law(pr.system, pr.P, limiter=limiter, bc=pr.bc, a=adv_speed)


def oracle_run(pr, dts, *, limiter=True, adv_speed=1.0, parity0=0, q0=None):
    s = oracle.Solver(law_of(pr, limiter, adv_speed), pr.q0 if q0 is None else q0, pr.dx, parity=parity0)
    s.step_dt(dts)
    return s.q, s.t, s.parity


def scales(q_ref):
    """Per-variable solution scale: max |point value| over the cells."""
    return np.maximum(np.max(np.abs(q_ref[:, :, 0]), axis=0), 1e-300)


def scaled_error(q_gpu, q_ref):
    """max |diff| per variable divided by the variable's scale."""
    sc = scales(q_ref)
    return float(np.max(np.abs(q_gpu - q_ref) / sc[None, :, None]))


def oracle_spread(run, q_in, ref, seed=0):
    """Largest deviation, per entry, of run(perturbed q_in) from ref."""
    rng = np.random.default_rng(seed)
    spread = np.zeros_like(ref)
    for _ in range(TRIALS):
        qp = q_in * (1.0 + PERTURB * rng.standard_normal(q_in.shape))
        spread = np.maximum(spread, np.abs(run(qp) - ref))
    return spread


class Parity:
    """Outcome of one conditioning-aware comparison.

    violation: max over entries of |gpu - oracle| / bound (<= 1 passes);
    raw:       max |gpu - oracle| / scale, the plain relative difference;
    excused:   share of entries whose difference exceeds 1e-11 x scale and
               that pass only through the spread term of the bound;
    entries:   number of entries compared."""

    def __init__(self, violation, raw, excused, entries):
        self.violation, self.raw, self.excused, self.entries = violation, raw, excused, entries

    def as_dict(self):
        return {"violation": self.violation, "raw": self.raw, "excused": self.excused, "entries": self.entries}

    def __repr__(self):
        return (f"Parity(violation={self.violation:.3g}, raw={self.raw:.3g}, excused={self.excused:.3g}, "
                f"entries={self.entries})")


def parity_report(q_gpu, ref, spread):
    sc = scales(ref)[None, :, None]
    diff = np.abs(q_gpu - ref)
    bound = np.maximum(TOL64 * sc, SCATTER_FACTOR * spread)
    rep = Parity(float(np.max(diff / bound)), float(np.max(diff / sc)),
                 float(np.mean(diff > TOL64 * sc)), int(diff.size))
    _record(rep)
    return rep


def parity_violation(q_gpu, ref, spread):
    """Ratio of |gpu - oracle| to the per-cell bound (<= 1 passes)."""
    return parity_report(q_gpu, ref, spread).violation


def merge(reports):
    """The worst of several reports (per field)."""
    reports = list(reports)
    return Parity(max(r.violation for r in reports), max(r.raw for r in reports),
                  max(r.excused for r in reports), sum(r.entries for r in reports))


# the plain bound: nothing excused
PLAIN = dict(excused_max=0.0, raw_max=TOL64)


def assert_parity(rep, *, excused_max, raw_max):
    """The bound holds, and the spread term excuses no more than
    `excused_max` of the entries, none by more than `raw_max` x scale."""
    assert rep.violation <= 1.0, rep
    assert rep.excused <= excused_max, rep
    assert rep.raw <= raw_max, rep


def _record(rep):
    """Appends the report, with the running test's name, to the JSON-lines
    file named by WCC_PARITY_REPORT (if set)."""
    import json
    import os

    path = os.environ.get("WCC_PARITY_REPORT")
    if path:
        with open(path, "a") as f:
            f.write(json.dumps({"test": os.environ.get("PYTEST_CURRENT_TEST", "?"), **rep.as_dict()}) + "\n")


def trajectory_check(pr, q_gpu, dts, *, limiter=True, adv_speed=1.0):
    """Compare a GPU trajectory with the oracle replaying its dts; returns
    the Parity report."""
    law = law_of(pr, limiter, adv_speed)

    def run(q0):
        s = oracle.Solver(law, q0, pr.dx)
        s.step_dt(dts)
        return s.q

    ref = run(pr.q0)
    spread = oracle_spread(run, pr.q0, ref)
    return parity_report(q_gpu, ref, spread)


def fp32_pair_violation(pr, q_a, q_b, dts, *, floor=2e-6, perturb=1e-7, trials=3, seed=0):
    """Compare two FP32-mixed results of the same problem (e.g. a batch
    instance and the same problem run alone): per cell
    |a - b| <= max(floor x scale, 50 x the oracle's spread over `dts` when
    its inputs are perturbed by `perturb` relative, FP32 rounding level).
    Returns the largest ratio to that bound (<= 1 passes)."""
    law = law_of(pr)

    def run(q0):
        s = oracle.Solver(law, q0, pr.dx)
        s.step_dt(dts)
        return s.q

    ref = run(pr.q0)
    rng = np.random.default_rng(seed)
    spread = np.zeros_like(ref)
    for _ in range(trials):
        qp = pr.q0 * (1.0 + perturb * rng.standard_normal(pr.q0.shape))
        spread = np.maximum(spread, np.abs(run(qp) - ref))
    sc = scales(ref)
    bound = np.maximum(floor * sc[None, :, None], SCATTER_FACTOR * spread)
    return float(np.max(np.abs(q_a - q_b) / bound))


def oracle_l1_spread(pr, dts, perturb, *, trials=3, seed=0):
    """Largest L1 (centre point values, per variable over its scale) by
    which the oracle's own trajectory over `dts` moves when its inputs are
    perturbed by `perturb` relative noise."""
    law = law_of(pr)

    def run(q0):
        s = oracle.Solver(law, q0, pr.dx)
        s.step_dt(dts)
        return s.q

    ref = run(pr.q0)
    sc = scales(ref)
    rng = np.random.default_rng(seed)
    worst = 0.0
    for _ in range(trials):
        q = run(pr.q0 * (1.0 + perturb * rng.standard_normal(pr.q0.shape)))
        worst = max(worst, float(np.max(np.mean(np.abs(q[:, :, 0] - ref[:, :, 0]), axis=0) / sc)))
    return ref, worst


def sampled_new_cells2d(law, q, parity, cells, lamx, lamy, *, rng=None, noise=0.0):
    """The oracle's new cells (j, i) of one 2D half-step from the stage q
    [ny, nx, nv, nq], one at a time (oracle.new_cell2d) from their four
    parents, so that a few cells of a mesh too large for the whole-stage
    oracle can be checked.  New cell i of parity 0 lies between old cells
    i and i + 1, of parity 1 between i - 1 and i (Sec. 3.1); periodic meshes
    wrap, transmissive ones repeat the edge cell.  With ``rng`` each parent
    is multiplied by (1 + noise x N(0, 1)) entry by entry (the spread of the
    parity bound).  Returns [len(cells), nv, nq]."""
    ny, nx = q.shape[:2]

    def parent(j, n):
        return j % n if law.bc == oracle.PERIODIC else min(max(j, 0), n - 1)

    out = []
    for j, i in cells:
        il, jl = (i, j) if parity == 0 else (i - 1, j - 1)
        x0, x1, y0, y1 = parent(il, nx), parent(il + 1, nx), parent(jl, ny), parent(jl + 1, ny)
        ps = [q[y0, x0], q[y0, x1], q[y1, x1], q[y1, x0]]
        if rng is not None:
            ps = [p * (1.0 + noise * rng.standard_normal(p.shape)) for p in ps]
        out.append(oracle.new_cell2d(law, *ps, lamx, lamy))
    return np.array(out)
