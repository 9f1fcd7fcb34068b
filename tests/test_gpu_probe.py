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


def test_replay_probe_times_a_window_and_rejects_bad_arguments():
    """gtp_measure_replay: a positive time that grows with the records, and
    the argument checks (no such window, a bin size that does not divide the
    window)."""
    import synth
    from paper_2609_05960_gb300 import Engine, GtpError, gtpower
    lib = synth.make_library(1)
    net = synth.make_netlist(lib, 20_000, seed=2)
    e = Engine(0)
    try:
        e.load_library(lib)
        e.load_netlist(net)
        times = []
        for w, n_ev in enumerate((200_000, 4_000_000)):
            tr = synth.make_trace(net, synth.zipf_counts(net.n_gates, n_ev, 1.2, None, 3 + w), 1_000_000, 3 + w)
            e.load_events(w, tr)
            times.append(gtpower.gtp_measure_replay(e.ctx, w, 10))
        assert 0.0 < times[0] < times[1]
        with pytest.raises(GtpError):
            gtpower.gtp_measure_replay(e.ctx, 7, 10)
        with pytest.raises(GtpError):
            gtpower.gtp_measure_replay(e.ctx, 0, 7)
    finally:
        e.close()
