"""The C-ABI library builds for sm_103a, loads, and exports every function
declared in include/*.h; host-side argument checks run without a GPU."""
import ctypes
import glob
import os

import pytest

from paper_2104_04347_gb300 import wcc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        names += wcc.header_functions(h)
    return sorted(set(names))


def test_library_exports_every_declared_function():
    lib = wcc.load()
    names = _declared()
    assert "wcc_create" in names and "wcc_step" in names and "wcc_get_dofs" in names
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_header():
    # every declared function has a ctypes signature in the binding
    assert set(_declared()) <= set(wcc._SIGS)


def test_default_options():
    o = wcc.default_options()
    assert o.precision == wcc.FP64 and o.limiter == 1
    assert o.alpha == 2.0 and o.eps == 1e-40 and o.gamma == 1.4 and o.graph_chunk == 32


@pytest.mark.parametrize("args,needle", [
    ((7, 64, 2, (0.0, 1.0), 0), "system"),
    ((0, 64, 0, (0.0, 1.0), 0), "P must"),
    ((0, 64, 7, (0.0, 1.0), 0), "P must"),
    ((0, 2, 2, (0.0, 1.0), 0), "N must"),
    ((0, 64, 2, (1.0, 0.0), 0), "domain"),
    ((0, 64, 2, (0.0, 1.0), 9), "bc"),
])
def test_create_rejects_bad_arguments(args, needle):
    with pytest.raises(wcc.WCCError) as ei:
        wcc.Solver(*args)
    assert ei.value.code == -1 and needle in str(ei.value)


@pytest.mark.parametrize("precision", [wcc.FP32_MIXED, wcc.FP32])
def test_every_precision_takes_p_up_to_6(precision):
    # P = 7 is refused by every precision; P = 5, 6 pass the argument checks of
    # the FP32 variants too (here, without a GPU, create then fails on the
    # missing device, not on P)
    with pytest.raises(wcc.WCCError) as ei:
        wcc.Solver(2, 64, 7, (0.0, 1.0), 1, precision=precision)
    assert ei.value.code == -1 and "P must" in str(ei.value)
    for P in (5, 6):
        try:
            wcc.Solver(2, 64, P, (0.0, 1.0), 1, precision=precision).close()
        except wcc.WCCError as e:
            assert e.code != -1, str(e)


@pytest.mark.parametrize("args,kw,code,needle", [
    ((7, 64, 64, 2, (0.0, 1.0, 0.0, 1.0), 0), {}, -1, "system"),
    ((2, 64, 64, 4, (0.0, 1.0, 0.0, 1.0), 0), {}, -1, "P must"),
    ((2, 3, 64, 2, (0.0, 1.0, 0.0, 1.0), 0), {}, -1, "nx and ny"),
    ((2, 64, 1 << 16, 2, (0.0, 1.0, 0.0, 1.0), 0), {}, -7, "2^15"),
    ((2, 64, 64, 2, (0.0, 1.0, 1.0, 0.0), 0), {}, -1, "domain"),
    ((2, 64, 64, 2, (0.0, 1.0, 0.0, 1.0), 5), {}, -1, "bc"),
    ((2, 64, 64, 2, (0.0, 1.0, 0.0, 1.0), 0), {"precision": 7}, -1, "precision"),
    ((2, 64, 64, 2, (0.0, 1.0, 0.0, 1.0), 0), {"rows_per_cta": 0}, -1, "options"),
])
def test_create2d_rejects_bad_arguments(args, kw, code, needle):
    with pytest.raises(wcc.WCCError) as ei:
        wcc.Solver2D(*args, **kw)
    assert ei.value.code == code and needle in str(ei.value)


def test_null_handle_calls_fail_cleanly():
    lib = wcc.load()
    assert lib.wcc_step(None, 1, 0.3) == -1
    assert lib.wcc_synchronize(None) == -1
    lib.wcc_destroy(None)
    assert lib.wcc2d_step(None, 1, 0.3) == -1
    assert lib.wcc2d_synchronize(None) == -1
    assert lib.wcc2d_destroy(None) == 0
    # the tuners, the pair statistics and the batch calls
    i, j = ctypes.c_int(), ctypes.c_int()
    n1, n2 = ctypes.c_int64(), ctypes.c_int64()
    nu = ctypes.c_double()
    assert lib.wcc_autotune(None, 0.2, ctypes.byref(i), ctypes.byref(j)) == -1
    assert lib.wcc_tb_stats(None, ctypes.byref(n1), ctypes.byref(n2), ctypes.byref(nu)) == -1
    assert lib.wcc_step_until(None, 1.0, 0.2, ctypes.byref(n1)) == -1
    assert lib.wcc2d_autotune(None, 0.2, ctypes.byref(i)) == -1
    assert lib.wcc_batch_step(None, 1, 0.2) == -1
    assert lib.wcc_batch_autotune(None, 0.2, ctypes.byref(i)) == -1
    assert lib.wcc_batch_get_tuning(None, ctypes.byref(i), ctypes.byref(j)) == -1
    assert lib.wcc_batch_tb_stats(None, ctypes.byref(n1), ctypes.byref(n2)) == -1
    assert lib.wcc_batch_synchronize(None) == -1
    lib.wcc_batch_destroy(None)


@pytest.mark.parametrize("kw,needle", [
    (dict(precision=wcc.FP64, tb_depth=2), "tb_depth = 2 needs"),
    (dict(precision=wcc.FP32_MIXED, tb_depth=3), "tb_depth must be"),
    (dict(precision=wcc.FP32_MIXED, tb_depth=2, tb_cfl_growth=-2.0), "tb_cfl_growth"),
])
def test_create_rejects_bad_temporal_blocking(kw, needle):
    with pytest.raises(wcc.WCCError) as ei:
        wcc.Solver(2, 64, 3, (0.0, 1.0), 1, **kw)
    assert ei.value.code == -1 and needle in str(ei.value)


def test_default_temporal_blocking_options():
    o = wcc.default_options()
    assert o.tb_depth == 1 and o.tb_cfl_growth == 0.1


@pytest.mark.parametrize("precision,cpb", [(wcc.FP64, 255), (wcc.FP32_MIXED, 127), (wcc.FP32_MIXED, 300),
                                           (wcc.FP32, 510)])
def test_create_rejects_tile_sizes_that_are_not_compiled(precision, cpb):
    # P = 3: FP64 tiles are 127 cells, FP32-mixed 255 or 510, plain FP32 255
    with pytest.raises(wcc.WCCError) as ei:
        wcc.Solver(2, 64, 3, (0.0, 1.0), 1, precision=precision, cells_per_block=cpb)
    assert ei.value.code == -1 and "cells_per_block" in str(ei.value)
