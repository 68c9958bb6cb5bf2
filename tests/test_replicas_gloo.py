"""The N > 1 path of bench.py runs independent replicas (the method has no
exchange step on one GPU) and reports the whole-job rate: units of all ranks
over the slowest rank's time.  Checked here with two gloo ranks on the CPU,
each advancing its own replica with the oracle."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as td  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import time

    import bench
    import oracle
    from paper_2104_04347_gb300 import inputs

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    td.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r advances a replica of a different size, so the work differs
        pr = inputs.euler_riemann_seeded(256 * (rank + 1), 3)
        law = oracle.make_law(oracle.EULER, 3, limiter=True, bc=oracle.TRANSMISSIVE)
        s = oracle.Solver(law, pr.q0, pr.dx)
        t0 = time.perf_counter()
        s.step_cfl(4, 0.2)
        secs = time.perf_counter() - t0
        units = 2 * ((pr.N + 1) + pr.N)
        value = bench.job_throughput(units, secs, "cpu")
        mx = bench.reduce_over_ranks(secs, "max", "cpu")
        sm = bench.reduce_over_ranks(units, "sum", "cpu")
        out[rank] = (units, secs, value, mx, sm)
    finally:
        td.destroy_process_group()


def test_two_gloo_ranks_report_whole_job_rate():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    units = [res[r][0] for r in range(world)]
    secs = [res[r][1] for r in range(world)]
    for r in range(world):
        _, _, value, mx, sm = res[r]
        assert mx == max(secs) and sm == sum(units)
        assert abs(value - sum(units) / max(secs)) <= 1e-9 * value


def test_without_a_group_the_rate_is_local():
    import bench
    assert bench.job_throughput(100.0, 2.0, "cpu") == 50.0
