"""Gates split into pieces (the persistent walk's big items) against the
FP64 oracle, element by element, through the C ABI.

A gate with more than `piece_len` events is walked as several big items, each
starting from the state its earlier records leave (each pin's last earlier
value).  With the smallest piece length (4,096 events) the cases reach: a
timestamp group cut by a piece boundary, a pin idle over many pieces,
glitch detection across pieces (each pin's previous event time comes from the
earlier piece), component waveforms, the adjoint, batched windows, and a
malformed record in a later piece (still located exactly).  Bar as
everywhere: states and counts bit-exact, bins and per-gate energies within
1e-5 relative; adjoint gradients as in the adjoint tests."""
import numpy as np
import pytest

import oracle
import synth
from cases import netlist_from, single_cell_library, trace_from

pytestmark = pytest.mark.gpu

TOL = 1e-5
PIECE = 4096


@pytest.fixture(scope="module")
def engine():
    from paper_2609_05960_gb300 import Engine
    e = Engine(0)
    yield e
    e.close()


def setup(engine, lib, net, piece_len=PIECE, rpt=8):
    engine.load_library(lib)
    engine.load_netlist(net)
    for k in ("kernel", "records_per_thread", "dense_min", "ctas_per_sm", "tile_min", "piece_len", "group_bin_bytes"):
        engine.set_param(k, -1)
    engine.set_param("piece_len", piece_len)
    engine.set_param("records_per_thread", rpt)


def check(w, ge, ref, bin_ps, tol=TOL):
    want = oracle.waveform_w(ref["bins"], bin_ps)
    rel = np.abs(w - want) / np.abs(want)
    assert rel.max() <= tol, f"bin {rel.argmax()}: got {w[rel.argmax()]} want {want[rel.argmax()]} rel {rel.max()}"
    np.testing.assert_array_equal(ge["n_events"], ref["n_events"])
    np.testing.assert_array_equal(ge["final_state"], ref["final_state"])
    for k in ("e_leak", "e_int", "e_sw"):
        err = np.abs(ge[k] - ref[k])
        bad = err > tol * np.abs(ref[k]) + 1e-9
        assert not bad.any(), f"{k}: gate {np.argmax(bad)} got {ge[k][np.argmax(bad)]} want {ref[k][np.argmax(bad)]}"


def _hot_gates():
    """Three hot gates and a few cool ones on the 12-cell library: a MUX2 of
    60k events with ties at every piece boundary (records 4096k-1 and 4096k
    share a time), a NAND3 whose pin 2 toggles only near the start (so later
    pieces find its value far back), an inverter of 30k events, and cool
    gates below the piece length."""
    lib = synth.make_library(1)
    rng = np.random.default_rng(17)
    T = 2_000_000
    gates, cells = [], []

    def events(n, n_pins, pins=None, tie_at=()):
        t = np.sort(rng.integers(0, T - 10, n))
        for k in tie_at:
            if 0 < k < n:
                t[k] = t[k - 1]
        S, ev = 0, []
        for k in range(n):
            p = int(rng.integers(0, n_pins)) if pins is None else int(pins[k])
            v = 1 - ((S >> p) & 1)
            S ^= 1 << p
            ev.append((int(t[k]), p, v))
        return ev

    gates.append(events(60_000, 4, tie_at=[PIECE * k for k in range(1, 15)]))
    cells.append(11)
    pins = rng.integers(0, 2, 40_000)
    pins[5] = 2
    pins[::7] = 3
    gates.append(events(40_000, 4, pins=pins))
    cells.append(3)
    gates.append(events(30_000, 2))
    cells.append(0)
    for n in (10, 700, 3000):
        gates.append(events(n, 3))
        cells.append(6)
    net = netlist_from(lib, cells, [2.0, 0.8, 5.0, 1.0, 3.0, 1.2],
                       np.random.default_rng(3).uniform(10, 200, (len(cells), lib.max_in, 2)))
    tr = trace_from(gates, [0] * len(cells), T)
    return lib, net, tr


@pytest.mark.parametrize("rpt", [4, 8, 16])
def test_pieces_match_the_oracle(engine, rpt):
    lib, net, tr = _hot_gates()
    ref = oracle.walk(lib, net, tr, 100)
    for piece in (PIECE, 0, 100_000):
        setup(engine, lib, net, piece, rpt)
        engine.load_events(0, tr)
        w = engine.run_power(0, 100).cpu().numpy()
        ge = engine.gate_energy(0, device=False)
        check(w, ge, ref, 100)
        # no gate longer than the piece length: the walk compiled without pieces ran
        assert engine.get_param("run_whole") == (0 if piece == PIECE else 1)
    setup(engine, lib, net, PIECE, rpt)
    engine.load_events(0, tr)
    engine.run_power(0, 100)
    assert engine.get_param("run_piece_len") == PIECE


def test_pieces_with_glitch_detection_and_components(engine):
    """Glitch detection needs each pin's previous event time: across a piece
    boundary it comes from the earlier piece's records."""
    lib, net, tr = _hot_gates()
    out_slew = np.random.default_rng(5).uniform(5, 300, (len(net.cell), 2)).astype(np.float32)
    for clock in (997, 100_000):
        ref = oracle.walk(lib, net, tr, 100, glitch=(clock, out_slew), components=True)
        setup(engine, lib, net)
        engine.set_glitch(clock, out_slew)
        engine.load_events(0, tr)
        w = engine.run_power(0, 100).cpu().numpy()
        ge = engine.gate_energy(0, device=False)
        check(w, ge, ref, 100)
        e_gl = engine.gate_glitch(0, device=False)
        assert np.all(np.abs(e_gl - ref["e_gl"]) <= TOL * np.abs(ref["e_gl"]) + 1e-9)
        comp = engine.run_power_components(0, 100).cpu().numpy()
        want = ref["comp_bins"] * 1e-3 / 100
        den = np.abs(want).max(axis=1, keepdims=True)
        assert (np.abs(comp - want) / np.where(den > 0, den, 1.0)).max() <= TOL
        engine.set_glitch(0)


def test_pieces_adjoint(engine):
    import torch
    lib, net, tr = _hot_gates()
    g = np.random.default_rng(2).uniform(-1, 1, tr.window_ps // 100)
    rC, re, rl = oracle.adjoint(lib, net, tr, 100, g)
    setup(engine, lib, net)
    engine.load_events(0, tr)
    engine.run_power(0, 100)
    dC, de, dl = engine.run_power_backward(0, 100, torch.tensor(g, dtype=torch.float32, device=engine.device))
    for got, want in ((dC, rC), (de, re), (dl, rl)):
        got = got.cpu().numpy()
        scale = np.abs(want).max()
        assert np.all(np.abs(got - want) <= 1e-4 * np.abs(want) + 1e-5 * scale)


def test_pieces_in_batched_windows(engine):
    lib, net, tr = _hot_gates()
    tr2 = synth.make_trace(net, synth.zipf_counts(len(net.cell), 50_000, 2.0, None, 8), tr.window_ps, 8, 0.02)
    setup(engine, lib, net)
    engine.load_events(0, tr)
    engine.load_events(1, tr2)
    outs = engine.run_power_batched([0, 1], 100)
    for w, t in ((0, tr), (1, tr2)):
        ref = oracle.walk(lib, net, t, 100)
        check(outs[w].cpu().numpy(), engine.gate_energy(w, device=False), ref, 100)


@pytest.mark.parametrize("kind,code", [("order", -2), ("time", -3), ("toggle", -4)])
def test_malformed_record_in_a_later_piece(engine, kind, code):
    from paper_2609_05960_gb300 import GtpError
    lib = single_cell_library(2, lambda *a: 1.0, lambda s: 1.0 + s)
    net = netlist_from(lib, [0, 0], [1.0, 1.0])
    rng = np.random.default_rng(11)
    T = 500_000
    t = np.sort(rng.integers(0, T, 20_000))
    S, g1 = 0, []
    for k in range(20_000):
        p = int(rng.integers(0, 3))
        v = 1 - ((S >> p) & 1)
        S ^= 1 << p
        g1.append((int(t[k]), p, v))
    pos = 3 * PIECE + 77
    tt, pin, v = g1[pos]
    if kind == "order":
        g1[pos] = (g1[pos - 1][0] - 1, pin, v)
    elif kind == "time":
        g1[pos] = (T + 5, pin, v)
    else:
        g1[pos] = (tt, pin, 1 - v)
    tr = trace_from([[(5, 0, 1)], g1], [0, 0], T)
    with pytest.raises(oracle.OracleError) as eo:
        oracle.walk(lib, net, tr, 100)
    assert eo.value.code == code and eo.value.record == 1 + pos
    setup(engine, lib, net)
    engine.load_events(0, tr)
    with pytest.raises(GtpError) as ei:
        engine.run_power(0, 100)
    assert ei.value.code == code
    assert f"at record {1 + pos}" in str(ei.value)
