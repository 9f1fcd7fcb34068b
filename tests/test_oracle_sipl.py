"""State-indexed lookup built from Liberty-style state patterns (Sec. 4.1):
the oracle's traversal pinned by a hand-worked multiplexer cell and closed
forms, and the engine's host-side expansion (gtp_sipl_expand, which
enumerates each pattern's don't-care pins) checked against the traversal.
CPU only."""
import numpy as np
import pytest

from oracle import sipl

NS, NL = 7, 7
A, B, S, Y = 0, 1, 2, 3  # MUX2 pins: Y = S ? B : A


def _mux2():
    """Internal power: A when !S 1 fJ, A when S 2 fJ, B when S 3 fJ on the
    rising edge only, otherwise (defaults) A 10, B 11 (fall) / 12 (rise),
    S 13 fJ.  Leakage: !A & !B 7 nW, then Y 9 nW (overlaps the first), else
    1 nW."""
    ip = [(A, -1, 1 << S, 0, 1.0), (A, -1, 1 << S, 1 << S, 2.0), (B, 1, 1 << S, 1 << S, 3.0)]
    dflt = [[10.0, 10.0], [11.0, 12.0], [13.0, 13.0]]
    lp = [((1 << A) | (1 << B), 0, 7.0), (1 << Y, 1 << Y, 9.0)]
    return ip, dflt, lp, 1.0


def _entry(e_int, n_in, pin, edge, side):
    T = NS * NL
    k = (pin * 2 + edge) * 2 ** (n_in - 1) + side
    return e_int[k * T:(k + 1) * T]


def test_hand_worked_multiplexer_by_traversal():
    ip, dflt, lp, ld = _mux2()
    e_int, p_leak = sipl.dense_cell(3, NS, NL, ip, dflt, lp, ld)
    # pin A: side bits are (B, S) in pin order; S is side bit 1
    for edge in (0, 1):
        for side, want in ((0b00, 1.0), (0b01, 1.0), (0b10, 2.0), (0b11, 2.0)):
            assert (_entry(e_int, 3, A, edge, side) == want).all()
    # pin B: side bits are (A, S); only the rising edge with S = 1 has a pattern
    for side in range(4):
        assert (_entry(e_int, 3, B, 0, side) == 11.0).all()
        assert (_entry(e_int, 3, B, 1, side) == (3.0 if side & 0b10 else 12.0)).all()
    # pin S: no pattern
    assert (e_int[(S * 2) * 4 * NS * NL:] == 13.0).all()
    # leakage: state bits A, B, S, Y; the first matching pattern wins
    for state in range(16):
        if not state & 0b0011:
            want = 7.0
        elif state & 0b1000:
            want = 9.0
        else:
            want = 1.0
        assert p_leak[state] == want, state


@pytest.mark.parametrize("n_in", [1, 2, 3, 5, 7])
def test_side_index_round_trip(n_in):
    """input_state inverts the compaction of the other input pins."""
    for pin in range(n_in):
        for side in range(2 ** (n_in - 1)):
            s = sipl.input_state(side, pin)
            assert not (s >> pin) & 1 and s < 2 ** n_in
            low, high = s & ((1 << pin) - 1), s >> (pin + 1)
            assert low | (high << pin) == side


def test_expansion_matches_traversal_on_the_multiplexer():
    from paper_2609_05960_gb300 import gtpower
    ip, dflt, lp, ld = _mux2()
    e1, l1 = gtpower.gtp_sipl_expand(3, NS, NL, ip, dflt, lp, ld)
    e2, l2 = sipl.dense_cell(3, NS, NL, ip, dflt, lp, ld)
    np.testing.assert_array_equal(e1, e2)
    np.testing.assert_array_equal(l1, l2)


def _random_patterns(rng, n_in):
    ip = []
    for _ in range(int(rng.integers(0, 3 * n_in + 1))):
        pin = int(rng.integers(0, n_in))
        allowed = ((1 << n_in) - 1) & ~(1 << pin)
        care = int(rng.integers(0, allowed + 1)) & allowed
        val = int(rng.integers(0, 1 << n_in)) & care
        tab = rng.uniform(0.5, 5.0, (NS, NL)).astype(np.float32)
        ip.append((pin, int(rng.integers(-1, 2)), care, val, tab))
    dflt = rng.uniform(0.5, 5.0, (n_in, 2, NS, NL)).astype(np.float32)
    lp = []
    full = (2 << n_in) - 1
    for _ in range(int(rng.integers(0, 2 ** n_in + 1))):
        care = int(rng.integers(0, full + 1))
        lp.append((care, int(rng.integers(0, full + 1)) & care, float(rng.uniform(1.0, 50.0))))
    return ip, dflt, lp, float(rng.uniform(1.0, 50.0))


@pytest.mark.parametrize("seed", range(12))
def test_expansion_matches_traversal_on_random_overlapping_patterns(seed):
    from paper_2609_05960_gb300 import gtpower
    rng = np.random.default_rng(seed)
    n_in = int(rng.integers(1, 8))
    ip, dflt, lp, ld = _random_patterns(rng, n_in)
    e1, l1 = gtpower.gtp_sipl_expand(n_in, NS, NL, ip, dflt, lp, ld)
    e2, l2 = sipl.dense_cell(n_in, NS, NL, ip, dflt, lp, ld)
    np.testing.assert_array_equal(e1, e2)
    np.testing.assert_array_equal(l1, l2)


def test_fully_specified_patterns_reproduce_a_dense_cell():
    """One pattern per state (every pin cared for) gives back the dense
    arrays the patterns were read from."""
    from paper_2609_05960_gb300 import gtpower
    rng = np.random.default_rng(5)
    n_in = 3
    dense = rng.uniform(0.5, 5.0, (n_in, 2, 4, NS, NL)).astype(np.float32)
    leak = rng.uniform(1.0, 50.0, 16).astype(np.float32)
    allowed = lambda p: ((1 << n_in) - 1) & ~(1 << p)
    ip = [(p, e, allowed(p), sipl.input_state(side, p), dense[p, e, side])
          for p in range(n_in) for e in range(2) for side in range(4)]
    lp = [(15, s, float(leak[s])) for s in range(16)]
    e_int, p_leak = gtpower.gtp_sipl_expand(n_in, NS, NL, ip, np.zeros((n_in, 2)), lp, 0.0)
    np.testing.assert_array_equal(e_int, dense.reshape(-1))
    np.testing.assert_array_equal(p_leak, leak)


@pytest.mark.parametrize("bad", ["own_pin", "output", "val_outside_care", "pin_range", "edge_range", "leak_bits"])
def test_expansion_rejects_malformed_patterns(bad):
    from paper_2609_05960_gb300 import GtpError, gtpower
    ip, dflt, lp, ld = _mux2()
    ip, lp = list(ip), list(lp)
    if bad == "own_pin":
        ip.append((A, 0, 1 << A, 0, 1.0))
    elif bad == "output":
        ip.append((A, 0, 1 << Y, 0, 1.0))
    elif bad == "val_outside_care":
        ip.append((A, 0, 1 << S, 1 << B, 1.0))
    elif bad == "pin_range":
        ip.append((3, 0, 0, 0, 1.0))
    elif bad == "edge_range":
        ip.append((A, 2, 0, 0, 1.0))
    else:
        lp.append((1 << 4, 0, 1.0))
    with pytest.raises(GtpError) as ei:
        gtpower.gtp_sipl_expand(3, NS, NL, ip, dflt, lp, ld)
    assert ei.value.code == gtpower.GTP_EINVAL
    with pytest.raises(GtpError) as ei:
        gtpower.gtp_sipl_expand(8, NS, NL, [], np.zeros((8, 2)), [], 0.0)
    assert ei.value.code == gtpower.GTP_ERANGE
