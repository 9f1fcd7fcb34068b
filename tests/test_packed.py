"""The packed transfer form of the records (gtp_pack_events, host only):
round trip against a plain decoding, block spans at the limit, and the
rejections.  CPU only."""
import numpy as np
import pytest

from cases import small_random


def _unpack(pk, n):
    nb = (n + 31) // 32
    anchors, words = pk[:nb].astype(np.int64), pk[nb:nb + n].astype(np.int64)
    t = anchors[np.arange(n) // 32] + (words >> 5)
    return np.stack([t, words & 31], axis=1)


@pytest.mark.parametrize("n_events", [1, 31, 32, 33, 10_000])
def test_round_trip(n_events):
    from paper_2609_05960_gb300 import gtpower
    _, _, tr = small_random(n_gates=50, n_events=n_events, window_ps=100_000, seed=7, tie_p=0.1)
    n = tr.records.shape[0]
    pk = gtpower.gtp_pack_events(tr.records)
    assert pk.shape[0] == gtpower.packed_words(n) == (n + 31) // 32 + n
    np.testing.assert_array_equal(_unpack(pk, n), tr.records.astype(np.int64))
    # each anchor is the smallest time of its block
    for b in range((n + 31) // 32):
        assert pk[b] == tr.records[32 * b:32 * b + 32, 0].min()


def test_empty_trace():
    from paper_2609_05960_gb300 import gtpower
    assert gtpower.gtp_pack_events(np.zeros((0, 2), np.uint32)).shape == (0,)


def test_block_span_limit():
    from paper_2609_05960_gb300 import GtpError, gtpower
    rec = np.zeros((40, 2), np.uint32)
    rec[:, 0] = 5
    rec[31, 0] = 5 + (1 << 27) - 1  # widest span that fits
    rec[32:, 0] = 1 << 30           # the second block, far from the first
    pk = gtpower.gtp_pack_events(rec)
    np.testing.assert_array_equal(_unpack(pk, 40), rec.astype(np.int64))
    rec[31, 0] = 5 + (1 << 27)
    with pytest.raises(GtpError) as ei:
        gtpower.gtp_pack_events(rec)
    assert ei.value.code == gtpower.GTP_ERANGE


@pytest.mark.parametrize("bad", ["negative_time", "reserved_bits"])
def test_rejections(bad):
    from paper_2609_05960_gb300 import GtpError, gtpower
    rec = np.zeros((10, 2), np.int32)
    if bad == "negative_time":
        rec[3, 0] = -1
    else:
        rec[3, 1] = 1 << 5
    with pytest.raises(GtpError) as ei:
        gtpower.gtp_pack_events(rec)
    assert ei.value.code == gtpower.GTP_ERANGE
