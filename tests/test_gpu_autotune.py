"""The single-grid autotuner (wcc_autotune) and the launch configurations it
chooses among: FP32-mixed with 255 or 510 new cells per CTA, one half-step
per launch, and two half-steps per launch.

Every candidate gives the scheme's results: within the FP32-mixed bounds of
the oracle replaying its dt list and of each other; tuning leaves the
handle's state as it was (the tuned handle then steps exactly like a fresh
one created with the chosen options)."""
import numpy as np
import pytest

from paper_2104_04347_gb300 import inputs, wcc
from tests.gpu_common import fp32_pair_violation, oracle_run, scales

pytestmark = pytest.mark.gpu

CANDIDATES = [(255, 1), (510, 1), (0, 2)]


def l1_rel(q, ref):
    return float(np.max(np.mean(np.abs(q[:, :, 0] - ref[:, :, 0]), axis=0) / scales(ref)))


def run(pr, nsteps, cfl, cpb, tb, dts=None):
    with wcc.Solver(pr.system, pr.N, pr.P, (pr.x_l, pr.x_r), pr.bc, precision=wcc.FP32_MIXED,
                    cells_per_block=cpb, tb_depth=tb) as s:
        s.set_initial(pr.q0)
        if dts is None:
            s.step(nsteps, cfl)
        else:
            s.step_dt(dts)
        return s.get_dofs(), s.dt_history()


@pytest.mark.parametrize("P", [2, 3])
@pytest.mark.parametrize("bc", [inputs.TRANSMISSIVE, inputs.PERIODIC])
def test_every_candidate_matches_the_oracle_and_the_others(P, bc):
    N = 3 * 510 + 77  # several CTAs of every tile size and a ragged tail
    pr = inputs.euler_riemann_seeded(N, P) if bc == inputs.TRANSMISSIVE else inputs.euler_density_wave(N, P)
    cfl = 0.3 if P == 2 else 0.25
    results = {}
    for cpb, tb in CANDIDATES:
        q, dts = run(pr, 64, cfl, cpb, tb)
        ref, _, _ = oracle_run(pr, dts)
        assert l1_rel(q, ref) <= 1e-6, (cpb, tb)
        results[(cpb, tb)] = (q, dts)
    # the one-half-step tile sizes take the same dt rule: same dt list, and
    # the same tile arithmetic
    (qa, da), (qb, db) = results[(255, 1)], results[(510, 1)]
    assert np.array_equal(da, db)
    assert fp32_pair_violation(pr, qa, qb, da) <= 1.0
    # the pairs' dt list differs; replay it one half-step per launch
    q2, d2 = results[(0, 2)]
    q1, _ = run(pr, None, None, 255, 1, dts=d2)
    assert fp32_pair_violation(pr, q2, q1, d2) <= 1.0


def test_autotune_restores_the_state_and_keeps_its_choice():
    pr = inputs.euler_riemann_seeded(1 << 16, 3)
    with wcc.Solver(pr.system, pr.N, 3, (pr.x_l, pr.x_r), pr.bc, precision=wcc.FP32_MIXED) as s:
        s.set_initial(pr.q0)
        s.step(10, 0.2)
        before, dts_before = s.get_dofs(), s.dt_history()
        state = s.state()
        cpb, tb = s.autotune(0.2)
        assert (cpb, tb) in CANDIDATES
        assert np.array_equal(s.get_dofs(), before)
        assert s.state() == state
        assert np.array_equal(s.dt_history(), dts_before)
    # tuned right after loading, then stepped: as a fresh handle created with
    # the chosen options
    with wcc.Solver(pr.system, pr.N, 3, (pr.x_l, pr.x_r), pr.bc, precision=wcc.FP32_MIXED) as s:
        s.set_initial(pr.q0)
        chosen = s.autotune(0.2)
        s.step(40, 0.2)
        q_tuned, d_tuned = s.get_dofs(), s.dt_history()
    with wcc.Solver(pr.system, pr.N, 3, (pr.x_l, pr.x_r), pr.bc, precision=wcc.FP32_MIXED,
                    cells_per_block=chosen[0], tb_depth=chosen[1]) as s:
        s.set_initial(pr.q0)
        s.step(40, 0.2)
        assert np.array_equal(s.dt_history(), d_tuned)
        assert np.array_equal(s.get_dofs(), q_tuned)


def test_autotune_of_fp64_returns_its_only_configuration():
    pr = inputs.euler_density_wave(512, 3)
    with wcc.Solver(pr.system, pr.N, 3, (pr.x_l, pr.x_r), pr.bc) as s:
        s.set_initial(pr.q0)
        assert s.autotune(0.25) == (0, 1)
