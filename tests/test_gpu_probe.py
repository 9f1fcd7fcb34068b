"""The reduction-rate probe (gtp_measure_reductions) that the bench's
roofline divides by: a positive, plausible rate for both widths, and the
argument checks."""
import pytest

pytestmark = pytest.mark.gpu


def test_reduction_probe_rates_and_rejections():
    from paper_2609_05960_gb300 import Engine, GtpError, gtpower
    e = Engine(0)
    try:
        r2 = gtpower.gtp_measure_reductions(e.ctx, 1 << 20, 2, 20_000_000)
        r4 = gtpower.gtp_measure_reductions(e.ctx, 1 << 20, 4, 20_000_000)
        # above 1 G/s and below one reduction per SM clock cycle of every SM
        assert 1e9 < r2 < 152 * 2.1e9 and 1e9 < r4 < 152 * 2.1e9
        for bad in ((0, 2, 10), (1024, 3, 10), (1024, 2, 0)):
            with pytest.raises(GtpError):
                gtpower.gtp_measure_reductions(e.ctx, *bad)
    finally:
        e.close()
