"""Without a GPU the library reports WCC_E_CUDA instead of computing on the CPU."""
import pytest

from paper_2104_04347_gb300 import wcc


def test_no_cpu_fallback():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(wcc.WCCError) as ei:
        wcc.Solver(wcc.EULER, 64, 3, (0.0, 1.0), wcc.TRANSMISSIVE)
    assert ei.value.code == -4
