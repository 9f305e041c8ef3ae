"""The pipe microbenchmark the bench's rooflines use as measured denominators."""
import pytest

pytestmark = pytest.mark.gpu


def test_measure_pipe_peaks():
    torch = pytest.importorskip("torch")
    assert torch.cuda.is_available()
    from paper_1303_4945_gb300 import build

    build.build()
    from paper_1303_4945_gb300 import sht

    p = sht.sht_measure_pipe_peaks()
    assert set(p) == {"fp64_fma_tflops", "fp32_fma_tops", "fp32_add_tops"}
    assert all(v > 0 for v in p.values())
    # the chains are issue-bound: FP32 issues many times the FP64 rate, adds as fast as FMAs
    assert p["fp32_fma_tops"] > 4 * p["fp64_fma_tflops"] / 2
    assert 0.5 < p["fp32_add_tops"] / p["fp32_fma_tops"] < 2.0
    with pytest.raises(sht.ShtError):
        sht.sht_measure_pipe_peaks(torch.cuda.device_count() + 5)
