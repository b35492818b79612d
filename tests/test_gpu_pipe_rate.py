"""ccg_pipe_rate: the measured issue rates the bench divides arithmetic-bound
sweeps by.  The checks are the GPU's known proportions, not its exact
figures: the FP32 pipe retires far more fused multiply-adds than the FP64
pipe, the 64-bit integer multiply-add runs well above the FP64 rate, and the
FP64 rate lies within a factor of two of the nominal 1.25 TFLOP/s."""
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ccg():
    from paper_1208_4869_gb300 import build as B
    B.build()
    from paper_1208_4869_gb300 import ccg as C
    return C


def test_pipe_rates_in_proportion(ccg):
    h = ccg.Handle()
    fp64 = h.pipe_rate(ccg.PIPE_FP64_FMA)      # Gop/s, one FMA = one op
    fp32 = h.pipe_rate(ccg.PIPE_FP32_FMA)
    imad = h.pipe_rate(ccg.PIPE_IMAD_WIDE)
    assert 0.625e3 / 2 < fp64 < 2 * 0.625e3
    assert fp32 > 16 * fp64
    assert imad > 4 * fp64
    assert h.pipe_rate(ccg.PIPE_MAD_WIDE_PTX) > 4 * fp64 and h.pipe_rate(ccg.PIPE_MAD_PAIR_PTX) > 4 * fp64
    before = h.launch_count()
    h.pipe_rate(ccg.PIPE_FP64_FMA)
    assert h.launch_count() == before + 6


def test_pipe_rate_rejects_bad_arguments(ccg):
    h = ccg.Handle()
    for pipe in (-1, 5):
        with pytest.raises(ccg.CcgError) as e:
            h.pipe_rate(pipe)
        assert e.value.status == ccg.ERR_INVALID
