"""Helpers shared by the GPU parity tests: run a problem through the C ABI
and through the oracle with the same half-step sizes."""
import numpy as np

import oracle
from paper_2104_04347_gb300 import inputs, wcc

# FP64 parity bound: max |gpu - oracle| <= TOL64 * (scale of the variable)
# after 100 half-steps (the oracle replays the GPU's realised dt sequence).
TOL64 = 1e-11


def gpu_run(pr, nsteps, cfl, *, limiter=True, precision=wcc.FP64, graph_chunk=32, dts=None, stream=None,
            adv_speed=1.0):
    with wcc.Solver(pr.system, pr.N, pr.P, (pr.x_l, pr.x_r), pr.bc, precision=precision, limiter=limiter,
                    graph_chunk=graph_chunk, stream=stream, adv_speed=adv_speed) as s:
        s.set_initial(pr.q0)
        if dts is None:
            s.step(nsteps, cfl)
        else:
            s.step_dt(dts)
        q = s.get_dofs()
        t, k, parity = s.state()
        hist = s.dt_history()
    return q, hist, t, parity


def oracle_run(pr, dts, *, limiter=True, adv_speed=1.0, parity0=0, q0=None):
    law = oracle.make_law(pr.system, pr.P, limiter=limiter, bc=pr.bc, a=adv_speed)
    s = oracle.Solver(law, pr.q0 if q0 is None else q0, pr.dx, parity=parity0)
    s.step_dt(dts)
    return s.q, s.t, s.parity


def scaled_error(q_gpu, q_ref):
    """max |diff| per variable divided by the variable's max |value|."""
    nv = q_ref.shape[1]
    out = []
    for v in range(nv):
        scale = max(np.max(np.abs(q_ref[:, v, 0])), 1e-300)
        out.append(np.max(np.abs(q_gpu[:, v, :] - q_ref[:, v, :])) / scale)
    return max(out)
