"""Pins of the state-pattern oracle walk (oracle/patterns.py), CPU only.

The walk restates the C oracle's walk for gates of up to 32 pins, with every
lookup a scan of the cell's state patterns (Sec. 4.1, the fallback path).
It is pinned three ways:
  * on cells of 3-5 inputs it must equal the C oracle walk (oracle.walk) on
    the state-indexed library that sipl.dense_cell builds from the same
    patterns, bin by bin and gate by gate, with and without glitch
    detection, and reject malformed traces with the same codes and records;
  * on the 20- and 21-pin cells it must equal the per-picosecond brute-force
    simulator (oracle/brute.py), which integrates leakage picosecond by
    picosecond and interpolates with scipy;
  * closed forms on the 20-pin SRAM-like cell: a disabled macro whose clock
    alone toggles, at transition times and a load on table knots, takes the
    disabled-clock-rise and clock-fall tables exactly and leaks at the
    standby power.
"""
import numpy as np
import pytest

import oracle
import synth
from oracle import brute, sipl
from oracle import patterns as opat
from synth import patterns as spat


def _dense_equivalent(plib, pnet, ptrace, cells):
    """synth.Library / Netlist / Trace for gates of small pattern cells: the
    patterns expanded by traversal at every state (sipl.dense_cell)."""
    ns, nl = len(plib.slew_axis), len(plib.load_axis)
    e_all, l_all, n_in = [], [], []
    for c in cells:
        n, ip, d, lp, ld = plib.cell(c)
        e, l = sipl.dense_cell(n, ns, nl, ip, d, lp, ld)
        e_all.append(e)
        l_all.append(l)
        n_in.append(n)
    lib = synth.Library([plib.names[c] for c in cells], np.array(n_in, np.int32), plib.vdd, plib.slew_axis,
                        plib.load_axis, np.concatenate(e_all), np.concatenate(l_all))
    remap = {c: i for i, c in enumerate(cells)}
    stride = int(max(n_in))
    G = pnet.n_gates
    net = synth.Netlist(np.array([remap[int(c)] for c in pnet.cell], np.int32), pnet.load_ff,
                        np.ascontiguousarray(pnet.slew_ps[:, :stride]), pnet.n_pins.astype(np.uint8),
                        np.zeros(G, np.int32), -np.ones((G, stride), np.int64))
    rec = np.stack([ptrace.t_ps.astype(np.uint32),
                    ptrace.pin.astype(np.uint32) | (ptrace.value.astype(np.uint32) << 4)], axis=1)
    tr = synth.Trace(ptrace.window_ps, ptrace.offsets, np.ascontiguousarray(rec),
                     ptrace.init_state.astype(np.uint8), 0, 0)
    return lib, net, tr


def _small_case(seed, n_gates=30, n_events=6000, window=20000, tie_p=0.1):
    plib = spat.make_pattern_library(seed)
    small = [c for c in range(plib.n_cells) if plib.n_in[c] <= 5]
    w = [1.0 if c in small else 0.0 for c in range(plib.n_cells)]
    pnet = spat.make_pattern_netlist(plib, n_gates, seed=seed + 1, weights=w)
    counts = synth.zipf_counts(n_gates, n_events, 1.1, None, seed + 2)
    ptr = spat.make_pattern_trace(pnet, counts, window, seed + 2, tie_p=tie_p)
    return plib, pnet, ptr, small


def _close(a, b, rtol=1e-12):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    np.testing.assert_allclose(a, b, rtol=rtol, atol=rtol * max(1.0, float(np.abs(b).max(initial=0.0))))


@pytest.mark.parametrize("bin_ps", [1, 50, 1000])
@pytest.mark.parametrize("seed", [3, 8])
def test_equals_c_oracle_on_small_cells(seed, bin_ps):
    plib, pnet, ptr, small = _small_case(seed)
    lib, net, tr = _dense_equivalent(plib, pnet, ptr, small)
    want = oracle.walk(lib, net, tr, bin_ps)
    for range_split in (True, False):
        got = opat.walk(plib, pnet, ptr, bin_ps, range_split=range_split)
        _close(got["bins"], want["bins"])
        for k in ("e_leak", "e_int", "e_sw"):
            _close(got[k], want[k])
        np.testing.assert_array_equal(got["final_state"], want["final_state"].astype(np.uint32))
        np.testing.assert_array_equal(got["n_events"], want["n_events"])


@pytest.mark.parametrize("clock", [97, 1000])
def test_equals_c_oracle_with_glitches(clock):
    plib, pnet, ptr, small = _small_case(5, n_events=8000, window=10000)
    lib, net, tr = _dense_equivalent(plib, pnet, ptr, small)
    want = oracle.walk(lib, net, tr, 20, glitch=(clock, pnet.out_slew_ps))
    got = opat.walk(plib, pnet, ptr, 20, glitch_clock_ps=clock)
    assert want["e_gl"].sum() > 0
    _close(got["bins"], want["bins"])
    for k in ("e_leak", "e_int", "e_sw", "e_gl"):
        _close(got[k], want[k])


@pytest.mark.parametrize("kind,code", [("order", -2), ("time", -3), ("pin", -3), ("toggle", -4)])
def test_rejects_like_the_c_oracle(kind, code):
    plib, pnet, ptr, small = _small_case(4, n_gates=6, n_events=600, window=5000)
    g = int(np.argmax(np.diff(ptr.offsets)))
    pos = int(ptr.offsets[g]) + 40
    t, p = ptr.t_ps.copy(), ptr.pin.copy()
    v = ptr.value.copy()
    if kind == "order":
        t[pos] = t[pos - 1] - 1
    elif kind == "time":
        t[pos:int(ptr.offsets[g + 1])] = 5000
    elif kind == "pin":
        p[pos] = pnet.n_pins[g]
    else:
        v[pos] ^= 1
    bad = spat.PatternTrace(ptr.window_ps, ptr.offsets, t, p, v, ptr.init_state)
    lib, net, tr = _dense_equivalent(plib, pnet, bad, small)
    with pytest.raises(oracle.OracleError) as ec:
        oracle.walk(lib, net, tr, 10)
    with pytest.raises(oracle.OracleError) as ep:
        opat.walk(plib, pnet, bad, 10)
    assert (ep.value.code, ep.value.record) == (ec.value.code, ec.value.record) == (code, pos)


@pytest.mark.parametrize("clock", [0, 150])
def test_wide_cells_equal_brute_force(clock):
    """SRAM-like (20 pins) and 16-to-1 multiplexer (21 pins) gates with ties,
    the clock pin busy, against the per-picosecond simulator."""
    plib = spat.make_pattern_library(2)
    wide = [c for c in range(plib.n_cells) if plib.n_in[c] >= 19]
    w = [1.0 if c in wide else 0.0 for c in range(plib.n_cells)]
    pnet = spat.make_pattern_netlist(plib, 4, seed=9, weights=w)
    counts = np.array([60, 45, 1, 30])
    ptr = spat.make_pattern_trace(pnet, counts, 1500, 11, tie_p=0.2, clock_pin_share=0.4)
    got = opat.walk(plib, pnet, ptr, 30, glitch_clock_ps=clock)
    want = brute.simulate_patterns(plib, pnet, ptr, 30, clock=clock)
    _close(got["bins"], want["bins"], 1e-9)
    for k in ("e_leak", "e_int", "e_sw", "e_gl"):
        _close(got[k], want[k], 1e-9)
    np.testing.assert_array_equal(got["final_state"], want["final_state"])
    assert int(got["final_state"].max()) >= 1 << 16  # states wider than 16 bits were reached


def test_disabled_sram_closed_form():
    """CEN = 1 (disabled) and Q = 1: every clock rise takes the disabled-clock
    table, every fall the clock-fall table, and the gate leaks at the
    standby-with-output-high power throughout."""
    plib = spat.make_pattern_library(1)
    c = plib.names.index("SRAM20")
    n_in, ip, dflt, lp, ld = plib.cell(c)
    i, j = 2, 3  # knots
    pnet = spat.PatternNetlist(np.array([c], np.int32), np.array([plib.load_axis[j]], np.float32),
                               np.full((1, plib.max_in, 2), plib.slew_axis[i], np.float32),
                               np.zeros((1, 2), np.float32), np.array([n_in + 1], np.int32))
    T = 10_000
    times = np.arange(50, T, 50)
    init = (1 << 1) | (1 << 2) | (1 << 19)  # CEN, WEN, Q high; CLK low
    vals = (np.arange(len(times)) + 1) & 1  # 1, 0, 1, ...: rise, fall, ...
    ptr = spat.PatternTrace(T, np.array([0, len(times)]), times.astype(np.int32), np.zeros(len(times), np.uint8),
                            vals.astype(np.uint8), np.array([init], np.uint32))
    r = opat.walk(plib, pnet, ptr, 100)
    rise = [t for p, e, care, val, t in ip if p == 0 and e == 1 and care == 2 and val == 2][0]
    fall = [t for p, e, care, val, t in ip if p == 0 and e == 0][0]
    n_rise = int(vals.sum())
    n_fall = len(vals) - n_rise
    assert r["e_int"][0] == pytest.approx(n_rise * float(rise[i, j]) + n_fall * float(fall[i, j]), rel=1e-14)
    p_standby = [pw for care, val, pw in lp if care == (2 | (1 << 19))][0]
    assert r["e_leak"][0] == pytest.approx(float(np.float32(p_standby)) * T * 1e-6, rel=1e-14)
    assert r["e_sw"][0] == 0.0 and r["final_state"][0] == init ^ (len(times) & 1)
    # the waveform's total is the sum of the parts
    assert r["bins"].sum() == pytest.approx(r["e_leak"][0] + r["e_int"][0], rel=1e-13)


def test_generator_toggles_every_pin():
    """The pattern trace generator: times sorted per gate and inside the
    window, pins below the gate's pin count, every value a toggle."""
    plib = spat.make_pattern_library(1)
    pnet = spat.make_pattern_netlist(plib, 50, seed=3)
    counts = synth.zipf_counts(50, 20000, 1.2, None, 4)
    ptr = spat.make_pattern_trace(pnet, counts, 100_000, 4, tie_p=0.1, clock_pin_share=0.3)
    for g in range(50):
        a, b = ptr.offsets[g], ptr.offsets[g + 1]
        t = ptr.t_ps[a:b]
        assert np.all(np.diff(t) >= 0) and (t.size == 0 or (t.min() >= 0 and t.max() < 100_000))
        S = int(ptr.init_state[g])
        assert S < 1 << int(pnet.n_pins[g])
        for p, v in zip(ptr.pin[a:b], ptr.value[a:b]):
            assert p < pnet.n_pins[g] and ((S >> int(p)) & 1) != v
            S ^= 1 << int(p)


@pytest.mark.parametrize("clock", [0, 300])
def test_components_equal_the_c_oracle_and_add_up(clock):
    """The per-component bins (leakage, internal, switching, glitch) on small
    cells equal the C oracle's, and on the wide cells they add up to the bins
    and, per component, to the per-gate energies."""
    plib, pnet, ptr, small = _small_case(6, n_events=5000, window=10000)
    lib, net, tr = _dense_equivalent(plib, pnet, ptr, small)
    want = oracle.walk(lib, net, tr, 20, glitch=(clock, pnet.out_slew_ps) if clock else None, components=True)
    got = opat.walk(plib, pnet, ptr, 20, glitch_clock_ps=clock, components=True)
    _close(got["comp_bins"], want["comp_bins"])
    plib = spat.make_pattern_library(2)
    w = [1.0 if plib.n_in[c] >= 11 else 0.0 for c in range(plib.n_cells)]
    pnet = spat.make_pattern_netlist(plib, 10, seed=5, weights=w)
    ptr = spat.make_pattern_trace(pnet, np.array([300, 20, 0, 900, 5, 40, 600, 1, 2, 77]), 20000, 6, tie_p=0.1,
                                  clock_pin_share=0.3)
    r = opat.walk(plib, pnet, ptr, 50, glitch_clock_ps=clock, components=True)
    _close(r["comp_bins"].sum(axis=0), r["bins"])
    for row, k in enumerate(("e_leak", "e_int", "e_sw", "e_gl")):
        _close(r["comp_bins"][row].sum(), r[k].sum())


@pytest.mark.parametrize("clock", [0, 97])
def test_adjoint_equals_c_oracle_on_small_cells(clock):
    """dL/dC of the pattern oracle equals the C oracle's adjoint on the
    state-indexed library built from the same patterns (unit scales)."""
    import dataclasses
    plib, pnet, ptr, small = _small_case(6, n_events=8000, window=10000)
    lib, net, tr = _dense_equivalent(plib, pnet, ptr, small)
    bin_ps = 20
    dLdP = np.random.default_rng(3).normal(size=tr.window_ps // bin_ps) * 1e3
    glitch = (clock, pnet.out_slew_ps) if clock else None
    want, _, _ = oracle.adjoint(lib, net, tr, bin_ps, dLdP, glitch=glitch)
    got = opat.adjoint(plib, pnet, ptr, bin_ps, dLdP, glitch_clock_ps=clock)
    assert np.abs(want).max() > 0
    _close(got, want, 1e-11)
    sel = np.array([3, 0, 17])
    _close(opat.adjoint(plib, pnet, ptr, bin_ps, dLdP, glitch_clock_ps=clock, gates=sel), want[sel], 1e-11)


@pytest.mark.parametrize("clock", [0, 150])
def test_adjoint_central_differences_on_wide_cells(clock):
    """On 20- and 21-pin cells (pattern traversal), dL/dC equals central
    differences of the walk's waveform: with the loads at mid-segment the
    energies are affine in the load, so the difference is exact up to
    rounding."""
    import dataclasses
    plib = spat.make_pattern_library(2)
    wide = [c for c in range(plib.n_cells) if plib.n_in[c] >= 19]
    w = [1.0 if c in wide else 0.0 for c in range(plib.n_cells)]
    pnet = spat.make_pattern_netlist(plib, 4, seed=9, weights=w)
    la = np.asarray(plib.load_axis, np.float64)
    mids = 0.5 * (la[:-1] + la[1:])
    pnet = dataclasses.replace(pnet, load_ff=mids[np.arange(4) % len(mids)].astype(np.float32))
    counts = np.array([60, 45, 1, 30])
    ptr = spat.make_pattern_trace(pnet, counts, 1500, 11, tie_p=0.2, clock_pin_share=0.4)
    bin_ps = 30
    dLdP = np.random.default_rng(4).normal(size=1500 // bin_ps)
    got = opat.adjoint(plib, pnet, ptr, bin_ps, dLdP, glitch_clock_ps=clock)
    for g in range(4):
        h = 1e-3 * float(pnet.load_ff[g])
        loss = []
        for sgn in (1.0, -1.0):
            lf = pnet.load_ff.astype(np.float64).copy()
            lf[g] += sgn * h
            bins = opat.walk(plib, dataclasses.replace(pnet, load_ff=lf), ptr, bin_ps, glitch_clock_ps=clock)["bins"]
            loss.append(float(np.dot(dLdP, bins * 1e-3 / bin_ps)))
        fd = (loss[0] - loss[1]) / (2 * h)
        assert got[g] == pytest.approx(fd, rel=1e-7, abs=1e-9 * max(1.0, abs(fd)))
    assert np.count_nonzero(got) >= 3
