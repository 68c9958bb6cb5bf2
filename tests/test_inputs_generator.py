"""The seeded input generator: splitmix64 (Steele, Lea and Flood's SplitMix,
64-bit finaliser as published with the xoshiro generators) against its
reference outputs, and the workloads it seeds within their stated ranges."""
import numpy as np

from paper_2104_04347_gb300 import inputs


def test_splitmix64_reference_outputs():
    # the first outputs of the reference implementation started from state 0
    g = inputs.SplitMix64(0)
    assert [g.next_u64() for _ in range(5)] == [
        0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F, 0xF88BB8A8724C81EC, 0x1B39896A51A8749B]


def test_uniform_uses_the_top_53_bits():
    g, h = inputs.SplitMix64(2104043471), inputs.SplitMix64(2104043471)
    for _ in range(100):
        u = g.uniform()
        assert 0.0 <= u < 1.0
        assert u == (h.next_u64() >> 11) / 2.0 ** 53


def test_uniform_moments():
    g = inputs.SplitMix64(7)
    x = np.array([g.uniform(-0.5, 0.5) for _ in range(20000)])
    assert abs(x.mean()) < 0.01          # 4.9 standard errors
    assert abs(x.var() - 1.0 / 12.0) < 0.003


def test_riemann_states_in_their_ranges():
    # rho, p ~ U(0.1, 1), u ~ U(-0.5, 0.5) on each side
    for seed in (2104043471, 1, 2, 3):
        for rho, u, p in inputs.riemann_states(seed):
            assert 0.1 <= rho < 1.0 and 0.1 <= p < 1.0 and -0.5 <= u < 0.5


def test_bench_riemann_data_is_two_states_and_one_mixed_cell():
    pr = inputs.euler_riemann_seeded(1000, 3)
    avgs = pr.q0[:, :, 0]
    assert pr.q0.shape == (1001, 3, 4) and not np.any(pr.q0[:, :, 1:])
    distinct = np.unique(avgs, axis=0)
    assert len(distinct) <= 3      # left state, right state, the cell cut by the jump
    left, right = inputs.riemann_states()
    UL = inputs.primitive_to_conserved(*left)
    UR = inputs.primitive_to_conserved(*right)
    assert np.allclose(avgs[0], UL, rtol=0, atol=1e-15) and np.allclose(avgs[-1], UR, rtol=0, atol=1e-15)
