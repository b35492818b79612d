"""The tensor-core block product's stream-K work split, run on the host by the
library's own cut functions (the ones its launcher and kernel use) with the
invariants the kernel relies on checked (`ccg_check_block_schedule`): every
unit computed once, one finisher per tile, only a range's first segment left
unfinished, waits only on lower CTAs whose pieces are the tile's earlier K
blocks, indexes inside the buffers.  No GPU needed."""
import pytest

from paper_1208_4869_gb300 import ccg

SHAPES = [(8192, 256), (4096, 130), (1000, 37), (132, 1), (512, 256), (256, 8), (512, 64), (640, 24),
          (2048, 256), (8192, 1), (4099, 200), (16384, 256), (16384, 1), (300, 17), (65536, 3), (1, 1)]


@pytest.mark.parametrize("n,k", SHAPES)
@pytest.mark.parametrize("terms", [2, 3])
@pytest.mark.parametrize("sms", [152, 148, 132, 7, 1])
def test_cut_is_sound(n, k, terms, sms):
    ctas, bad = ccg.check_block_schedule(n, k, terms, sms)
    assert bad == 0, (n, k, terms, sms, bad)
    assert 1 <= ctas


def test_cut_fills_every_sm_at_the_batched_size():
    """n = 8192, k = 256 on 152 SMs: 76 ranges of the two column tiles, one
    CTA per SM (the one-CTA-per-tile grid had 128)."""
    assert ccg.check_block_schedule(8192, 256, 2, 152) == (152, 0)
    assert ccg.check_block_schedule(8192, 256, 3, 152) == (152, 0)


def test_bad_arguments_are_refused():
    for args in ((0, 8, 2, 152), (256, 0, 2, 152), (256, 257, 2, 152), (256, 8, 4, 152), (256, 8, 2, 0)):
        with pytest.raises(ccg.CcgError) as e:
            ccg.check_block_schedule(*args)
        assert e.value.status == ccg.ERR_INVALID
