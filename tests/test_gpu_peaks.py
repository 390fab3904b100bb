"""Peak-rate microbenchmarks (symft_measure_peaks) through the C-ABI: every
rate is measured, positive and ordered as the hardware's pipes are (FP64 FMA
far below FP32 FMA, a Philox block costing tens of integer operations)."""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_measure_peaks():
    import paper_2607_28600_b300 as S
    p = S.symft_measure_peaks()
    assert p["sm_count"] == torch.cuda.get_device_properties(0).multi_processor_count
    for k in ("int32_lop3_per_s", "int32_imad_wide_per_s", "philox_blocks_per_s", "fp32_fma_per_s",
              "fp64_fma_per_s", "smem_bytes_per_s"):
        assert p[k] > 0.0, k
    assert p["fp64_fma_per_s"] < p["fp32_fma_per_s"]
    # a Philox4x32-10 block is 20 32x32->64 multiplies plus logic: it cannot
    # run faster than the multiply pipe allows
    assert p["philox_blocks_per_s"] * 20 <= p["int32_imad_wide_per_s"] * 1.25
