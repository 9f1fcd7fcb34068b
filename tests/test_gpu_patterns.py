"""Pattern gates on the GPU (gtp_pattern.cu) against the FP64 oracle, element
by element, through the C ABI.

Pattern cells are given by Liberty-style state patterns, up to 32 pins
(Sec. 4.1): those with at most "sipl_max_pins" pins are walked through
state-indexed arrays built on the device, wider ones by scanning their
patterns at every lookup (the paper's fallback).  The oracle is
oracle/patterns.py (every lookup a traversal by oracle/sipl.py) for the
pattern gates plus oracle.walk for the ordinary gates of the same window.
Cases: the 20-pin SRAM-like macro and the 21-pin multiplexer with busy
clock pins, gates of many items (512 records each) with ties across item
boundaries, every threshold from 0 (all traversal) to 24 (every cell
indexed), glitch detection, batched windows, graph replay, malformed records
in a later item, component waveforms, the adjoint (dL/dC of the pattern
gates against the oracle's chain rule, with the ordinary gates' gradients
unchanged), and the calls that refuse windows with pattern gates.
Bar as everywhere: states and counts bit-exact, bins and per-gate energies
within 1e-5 relative."""
import numpy as np
import pytest

import oracle
import synth
from cases import small_random
from oracle import patterns as opat
from synth import patterns as spat

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def engine():
    from paper_2609_05960_gb300 import Engine
    e = Engine(0)
    yield e
    e.close()


def _reset(engine):
    for k in ("kernel", "records_per_thread", "dense_min", "ctas_per_sm", "tile_min", "piece_len", "group_bin_bytes",
              "sipl_max_pins"):
        engine.set_param(k, -1)


def _design(seed=1, n_pat=40, pat_events=60_000, window_ps=200_000, weights=None, tie_p=0.05, clock_share=0.3,
            main_events=20_000):
    lib, net, tr = small_random(n_gates=300, n_events=main_events, window_ps=window_ps, seed=seed + 10, tie_p=0.02)
    plib = spat.make_pattern_library(seed)
    pnet = spat.make_pattern_netlist(plib, n_pat, seed=seed + 1, weights=weights)
    counts = synth.zipf_counts(n_pat, pat_events, 1.1, None, seed + 2)
    ptr = spat.make_pattern_trace(pnet, counts, window_ps, seed + 2, tie_p=tie_p, clock_pin_share=clock_share)
    return lib, net, tr, plib, pnet, ptr


def _load(engine, lib, net, tr, plib, pnet, ptr, window=0):
    engine.load_library(lib)
    engine.load_netlist(net)
    _reset(engine)
    engine.load_pattern_cells(plib)
    engine.load_pattern_netlist(pnet)
    engine.load_events(window, tr)
    engine.load_pattern_events(window, ptr)


def _check(engine, w, ref, pref, bin_ps, window=0, tol=TOL):
    want = oracle.waveform_w(ref["bins"] + pref["bins"], bin_ps)
    rel = np.abs(w - want) / np.abs(want)
    assert rel.max() <= tol, f"bin {rel.argmax()}: got {w[rel.argmax()]} want {want[rel.argmax()]} rel {rel.max()}"
    ge = engine.gate_energy(window, device=False)
    np.testing.assert_array_equal(ge["final_state"], ref["final_state"])
    pe = engine.pattern_gate_energy(window)
    np.testing.assert_array_equal(pe["n_events"], pref["n_events"])
    np.testing.assert_array_equal(pe["final_state"], pref["final_state"])
    for k in ("e_leak", "e_int", "e_sw", "e_gl"):
        bad = np.abs(pe[k] - pref[k]) > tol * np.abs(pref[k]) + 1e-9
        assert not bad.any(), f"{k}: gate {np.argmax(bad)} got {pe[k][np.argmax(bad)]} want {pref[k][np.argmax(bad)]}"


def test_every_threshold_matches_the_oracle(engine):
    """All eight pattern cells (4 to 21 pins); thresholds 0 (every cell by
    traversal), 4, 8, 12, 16 (the paper's), 20 and 24 (every cell indexed)
    give the oracle's results; graph replay too."""
    lib, net, tr, plib, pnet, ptr = _design()
    bin_ps = 50
    ref = oracle.walk(lib, net, tr, bin_ps)
    pref = opat.walk(plib, pnet, ptr, bin_ps)
    _load(engine, lib, net, tr, plib, pnet, ptr)
    pins = plib.n_in + 1
    for thr in (0, 4, 8, 12, 16, 20, 24):
        engine.set_param("sipl_max_pins", thr)
        for graph in (False, True, True):
            w = engine.run_power(0, bin_ps, graph=graph).cpu().numpy()
            _check(engine, w, ref, pref, bin_ps)
        assert engine.get_param("pattern_indexed_cells") == int((pins <= thr).sum())
        want_bytes = sum(4 * (int(n) * 2 ** int(n) + 2 ** (int(n) + 1)) for n in plib.n_in if n + 1 <= thr)
        assert engine.get_param("pattern_index_bytes") == want_bytes


@pytest.mark.parametrize("clock", [0, 700])
def test_sram_macros_many_items(engine, clock):
    """Eight 20-pin SRAM-like macros of 512-40k events (1 to 79 items each),
    the clock pin busy, ties at about a third of the records (so groups
    cross the nominal item boundaries), with and without glitch detection."""
    plib = spat.make_pattern_library(2)
    w = [1.0 if n == "SRAM20" else 0.0 for n in plib.names]
    lib, net, tr = small_random(n_gates=200, n_events=5000, window_ps=100_000, seed=21, tie_p=0.02)
    pnet = spat.make_pattern_netlist(plib, 8, seed=22, weights=w)
    counts = np.array([40_000, 5_000, 20_000, 512, 1024, 513, 12_345, 30_000])
    ptr = spat.make_pattern_trace(pnet, counts, 100_000, 23, tie_p=0.3, clock_pin_share=0.5)
    out_slew = np.random.default_rng(4).uniform(10, 200, (net.n_gates, 2)).astype(np.float32)
    ref = oracle.walk(lib, net, tr, 20, glitch=(clock, out_slew) if clock else None)
    pref = opat.walk(plib, pnet, ptr, 20, glitch_clock_ps=clock)
    _load(engine, lib, net, tr, plib, pnet, ptr)
    if clock:
        engine.set_glitch(clock, out_slew)
        assert pref["e_gl"].sum() > 0
    for thr in (16, 24):
        engine.set_param("sipl_max_pins", thr)
        w_ = engine.run_power(0, 20).cpu().numpy()
        _check(engine, w_, ref, pref, 20)
    assert int(pref["final_state"].max()) >= 1 << 16
    engine.set_glitch(0)


def test_batched_windows_with_pattern_gates(engine):
    """Three windows, each with its own pattern events (one with none
    loaded, so only its ordinary gates run), walked in one batched run and in
    one group per window."""
    lib, net, tr0, plib, pnet, ptr0 = _design(seed=3, n_pat=30, pat_events=20_000, window_ps=60_000)
    tr1 = synth.make_trace(net, synth.zipf_counts(net.n_gates, 12_000, 1.2, None, 8), 60_000, 8, 0.02)
    counts = synth.zipf_counts(30, 15_000, 1.3, None, 9)
    ptr1 = spat.make_pattern_trace(pnet, counts, 60_000, 9, tie_p=0.1)
    tr2 = synth.make_trace(net, synth.zipf_counts(net.n_gates, 8000, 1.1, None, 5), 40_000, 5)
    _load(engine, lib, net, tr0, plib, pnet, ptr0, window=0)
    engine.load_events(1, tr1)
    engine.load_pattern_events(1, ptr1)
    engine.load_events(2, tr2)
    for gb in (-1, 1):
        engine.set_param("group_bin_bytes", gb)
        outs = engine.run_power_batched([0, 1, 2], 20)
        for k, (t, p) in enumerate(((tr0, ptr0), (tr1, ptr1))):
            _check(engine, outs[k].cpu().numpy(), oracle.walk(lib, net, t, 20), opat.walk(plib, pnet, p, 20), 20,
                   window=k)
        want = oracle.waveform_w(oracle.walk(lib, net, tr2, 20)["bins"], 20)
        assert (np.abs(outs[2].cpu().numpy() - want) / want).max() <= TOL


def test_pattern_events_from_device_arrays_and_zero_events(engine):
    import torch
    lib, net, tr, plib, pnet, ptr = _design(seed=5, n_pat=12, pat_events=3000, window_ps=30_000)
    counts = np.diff(ptr.offsets)
    ptr_z = spat.make_pattern_trace(pnet, np.zeros_like(counts), 30_000, 5)
    _load(engine, lib, net, tr, plib, pnet, ptr_z)
    w = engine.run_power(0, 10).cpu().numpy()
    _check(engine, w, oracle.walk(lib, net, tr, 10), opat.walk(plib, pnet, ptr_z, 10), 10)
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    engine.load_pattern_events(0, offsets=d(ptr.offsets), t_ps=d(ptr.t_ps), pin=d(ptr.pin), value=d(ptr.value),
                               init_state=d(ptr.init_state.view(np.int32)))
    w = engine.run_power(0, 10).cpu().numpy()
    _check(engine, w, oracle.walk(lib, net, tr, 10), opat.walk(plib, pnet, ptr, 10), 10)


def test_design_power_includes_pattern_gates(engine):
    lib, net, tr, plib, pnet, ptr = _design(seed=6, n_pat=20, pat_events=10_000, window_ps=50_000)
    _load(engine, lib, net, tr, plib, pnet, ptr)
    w = engine.run_power(0, 50)
    dp = engine.design_power(0, w)
    ref = oracle.walk(lib, net, tr, 50)
    pref = opat.walk(plib, pnet, ptr, 50)
    to_w = 1e-3 / 50_000
    for key, k in (("p_leak", "e_leak"), ("p_int", "e_int"), ("p_sw", "e_sw")):
        want = (ref[k].sum() + pref[k].sum()) * to_w
        assert dp[key] == pytest.approx(want, rel=1e-6), key


@pytest.mark.parametrize("kind,code", [("order", -2), ("time", -3), ("pin", -3), ("toggle", -4), ("value", -3)])
def test_malformed_pattern_record_in_a_later_item(engine, kind, code):
    """One bad record deep in a 10k-event macro (its thirteenth item) and a later
    bad one in another gate: the run reports the first, as the oracle does."""
    from paper_2609_05960_gb300 import GtpError
    plib = spat.make_pattern_library(1)
    w = [1.0 if n in ("SRAM20", "MUX16P") else 0.0 for n in plib.names]
    lib, net, tr = small_random(n_gates=50, n_events=2000, window_ps=50_000, seed=31)
    pnet = spat.make_pattern_netlist(plib, 4, seed=32, weights=w)
    ptr = spat.make_pattern_trace(pnet, np.array([100, 10_000, 3000, 500]), 50_000, 33, tie_p=0.05)
    g = 1
    pos = int(ptr.offsets[g]) + 3 * 2048 + 77
    t, p, v = ptr.t_ps.copy(), ptr.pin.copy(), ptr.value.copy()
    if kind == "order":
        t[pos] = t[pos - 1] - 1
    elif kind == "time":
        t[pos:int(ptr.offsets[g + 1])] = 50_000
    elif kind == "pin":
        p[pos] = pnet.n_pins[g]
    elif kind == "toggle":
        v[pos] ^= 1
    else:
        v[pos] = 2
    q = int(ptr.offsets[2]) + 100
    p[q] = 40  # a later error in another gate
    bad = spat.PatternTrace(ptr.window_ps, ptr.offsets, t, p, v, ptr.init_state)
    if kind != "value":
        with pytest.raises(oracle.OracleError) as eo:
            opat.walk(plib, pnet, bad, 10)
        assert (eo.value.code, eo.value.record) == (code, pos)
    _load(engine, lib, net, tr, plib, pnet, bad)
    for thr in (0, 24):
        engine.set_param("sipl_max_pins", thr)
        with pytest.raises(GtpError) as ei:
            engine.run_power(0, 10)
        assert ei.value.code == code
        assert f"at pattern record {pos}" in str(ei.value)


@pytest.mark.parametrize("clock", [0, 500])
def test_component_waveforms_with_pattern_gates(engine, clock):
    """gtp_run_power_components on a window with pattern gates: each row
    (leakage, internal, switching, glitch) against the oracles' component
    bins (the C oracle for the ordinary gates plus oracle/patterns.py), and
    the total waveform."""
    lib, net, tr, plib, pnet, ptr = _design(seed=8, n_pat=30, pat_events=30_000, window_ps=100_000)
    out_slew = np.random.default_rng(3).uniform(10, 200, (net.n_gates, 2)).astype(np.float32)
    ref = oracle.walk(lib, net, tr, 50, glitch=(clock, out_slew) if clock else None, components=True)
    pref = opat.walk(plib, pnet, ptr, 50, glitch_clock_ps=clock, components=True)
    _load(engine, lib, net, tr, plib, pnet, ptr)
    if clock:
        engine.set_glitch(clock, out_slew)
    total = engine.run_power(0, 50).cpu().numpy()
    comp = engine.run_power_components(0, 50).cpu().numpy()
    want = (ref["comp_bins"] + pref["comp_bins"]) * 1e-3 / 50
    den = np.abs(want).max(axis=1, keepdims=True)
    assert (np.abs(comp - want) / np.where(den > 0, den, 1.0)).max() <= TOL
    assert (np.abs(comp.sum(axis=0) - total) / np.abs(total)).max() <= TOL
    if clock:
        assert pref["comp_bins"][3].sum() > 0
    engine.set_glitch(0)


def test_calls_without_pattern_support_refuse(engine):
    from paper_2609_05960_gb300 import GtpError
    lib, net, tr, plib, pnet, ptr = _design(seed=7, n_pat=5, pat_events=500, window_ps=20_000)
    _load(engine, lib, net, tr, plib, pnet, ptr)
    engine.run_power(0, 10)
    with pytest.raises(GtpError) as e2:
        engine.pattern_gate_gradient(0)  # no backward run yet
    with pytest.raises(GtpError) as e3:
        engine.run_power_scheme(0, 10, "fused")
    assert e2.value.code == e3.value.code == -1
    # loading the window's ordinary events again drops its pattern events: the window runs without them
    engine.load_events(0, tr)
    w = engine.run_power(0, 10).cpu().numpy()
    want = oracle.waveform_w(oracle.walk(lib, net, tr, 10)["bins"], 10)
    assert (np.abs(w - want) / want).max() <= TOL
    with pytest.raises(GtpError):
        engine.pattern_gate_energy(0)


def _grad_close(got, want, rtol=1e-4):
    got = np.asarray(got, np.float64)
    want = np.asarray(want, np.float64)
    bad = np.abs(got - want) > rtol * np.abs(want) + 1e-5 * np.abs(want).max()
    assert not bad.any(), f"{bad.sum()} off; first {np.argmax(bad)}: got {got[np.argmax(bad)]} want {want[np.argmax(bad)]}"


@pytest.mark.parametrize("clock", [0, 700])
def test_adjoint_with_pattern_gates(engine, clock):
    """gtp_run_power_backward on a window with pattern gates: the ordinary
    gates' dL/dC and scale gradients equal the C oracle's adjoint, the pattern
    gates' dL/dC (gtp_pattern_gate_gradient) the pattern oracle's, with many
    items per gate, ties across item boundaries, glitch detection and every
    threshold's lookups."""
    import torch
    plib = spat.make_pattern_library(2)
    lib, net, tr = small_random(n_gates=300, n_events=20_000, window_ps=100_000, seed=31, tie_p=0.02)
    pnet = spat.make_pattern_netlist(plib, 30, seed=32)
    counts = synth.zipf_counts(30, 60_000, 1.1, None, 33)
    ptr = spat.make_pattern_trace(pnet, counts, 100_000, 33, tie_p=0.3, clock_pin_share=0.4)
    bin_ps = 25
    g = (np.random.default_rng(7).normal(size=100_000 // bin_ps) * 1e3).astype(np.float32)
    out_slew = np.random.default_rng(4).uniform(10, 200, (net.n_gates, 2)).astype(np.float32)
    glitch = (clock, out_slew) if clock else None
    rC, rde, rdl = oracle.adjoint(lib, net, tr, bin_ps, g.astype(np.float64), glitch=glitch)
    pC = opat.adjoint(plib, pnet, ptr, bin_ps, g.astype(np.float64), glitch_clock_ps=clock)
    assert np.count_nonzero(pC) > 20
    _load(engine, lib, net, tr, plib, pnet, ptr)
    if clock:
        engine.set_glitch(clock, out_slew)
    gd = torch.from_numpy(g).to(engine.device)
    for thr in (0, 16, 24):
        engine.set_param("sipl_max_pins", thr)
        engine.run_power(0, bin_ps)
        dC, de, dl = engine.run_power_backward(0, bin_ps, gd)
        _grad_close(dC.cpu().numpy(), rC)
        _grad_close(de.cpu().numpy(), rde)
        _grad_close(dl.cpu().numpy(), rdl)
        _grad_close(engine.pattern_gate_gradient(0), pC)
        _grad_close(engine.pattern_gate_gradient(0, device=True).cpu().numpy(), pC)
    engine.set_glitch(0)


def test_adjoint_reports_malformed_pattern_record(engine):
    """A malformed pattern record makes the backward run fail with the
    forward run's code and record, and leaves no pattern gradient."""
    import torch
    from paper_2609_05960_gb300 import GtpError
    lib, net, tr, plib, pnet, ptr = _design(seed=9, n_pat=6, pat_events=4000, window_ps=50_000)
    g = int(np.argmax(np.diff(ptr.offsets)))
    pos = int(ptr.offsets[g]) + 700
    t = ptr.t_ps.copy()
    t[pos] = t[pos - 1] - 1  # out of order
    bad = spat.PatternTrace(ptr.window_ps, ptr.offsets, t, ptr.pin, ptr.value, ptr.init_state)
    with pytest.raises(oracle.OracleError) as eo:
        opat.adjoint(plib, pnet, bad, 10, np.ones(50_000 // 10))
    assert (eo.value.code, eo.value.record) == (-2, pos)
    _load(engine, lib, net, tr, plib, pnet, bad)
    gd = torch.ones(50_000 // 10, dtype=torch.float32, device=engine.device)
    with pytest.raises(GtpError) as ei:
        engine.run_power_backward(0, 10, gd)
    assert ei.value.code == -2 and f"at pattern record {pos}" in str(ei.value)
    with pytest.raises(GtpError):
        engine.pattern_gate_gradient(0)
