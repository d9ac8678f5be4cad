"""The measured FP64 fused multiply-add rate (lfm_measure_fp64_fma_rate; GPU required): a
positive rate of the order a GB300 can issue (nominal 1.25 TFLOP/s dense FP64, 625 G FMA/s),
repeatable, and an invalid device reported as LFM_EINVAL."""
import pytest

from paper_2507_18268_gb300 import binding as B

pytestmark = pytest.mark.gpu


def test_fp64_fma_rate_is_plausible_and_repeatable():
    a = B.lfm_measure_fp64_fma_rate(0)
    b = B.lfm_measure_fp64_fma_rate(0)
    assert 5e10 < a < 5e13
    assert abs(a - b) <= 0.2 * max(a, b)


def test_fp64_fma_rate_rejects_a_bad_device():
    with pytest.raises(B.LfmError) as e:
        B.lfm_measure_fp64_fma_rate(4096)
    assert e.value.code == B.LFM_EINVAL
