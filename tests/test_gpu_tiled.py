"""The time-sliced walk (gtp_tiled.cu) against the FP64 oracle, element by
element, through the C ABI.

It owns gates with at least `tile_min` events; the window is cut into slices
of 16,384 bins whose sums are kept in shared memory as exact integers.  The
cases reach: many slices and a ragged last one, events exactly on slice
boundaries and ties there, a gate whose events all fall in one slice, a gate
whose events start in a late slice, a pin idle for most of a gate (the entry
state comes from far back), bins whose shared-memory words carry (thousands
of events at one timestamp), energies too large to quantise (sent to L2
directly), signed energies, and malformed traces inside tiled gates (the
first bad record is still located exactly).  Bar as everywhere: states and
counts bit-exact, bins and per-gate energies within 1e-5 relative."""
import numpy as np
import pytest

import oracle
import synth
from cases import netlist_from, single_cell_library, small_random, trace_from

pytestmark = pytest.mark.gpu

TOL = 1e-5
SLICE = 16384


@pytest.fixture(scope="module")
def engine():
    from paper_2609_05960_gb300 import Engine
    e = Engine(0)
    yield e
    e.close()


def run(engine, lib, net, tr, bin_ps, tile_min, escale=None, lscale=None, dense_min=-1):
    engine.load_library(lib)
    engine.load_netlist(net)
    for k in ("kernel", "records_per_thread", "dense_min", "ctas_per_sm", "tile_min", "piece_len", "group_bin_bytes"):
        engine.set_param(k, -1)
    engine.set_param("tile_min", tile_min)
    engine.set_param("dense_min", dense_min)
    engine.set_scales(escale, lscale)
    engine.load_events(0, tr)
    w = engine.run_power(0, bin_ps).cpu().numpy()
    ge = engine.gate_energy(0, device=False)
    return w, ge


def check(w, ge, ref, bin_ps, tol=TOL, mean_scale=False):
    want = oracle.waveform_w(ref["bins"], bin_ps)
    den = np.abs(want).mean() if mean_scale else np.abs(want)
    rel = np.abs(w - want) / den
    assert rel.max() <= tol, f"bin {rel.argmax()}: got {w[rel.argmax()]} want {want[rel.argmax()]} rel {rel.max()}"
    np.testing.assert_array_equal(ge["n_events"], ref["n_events"])
    np.testing.assert_array_equal(ge["final_state"], ref["final_state"])
    for k in ("e_leak", "e_int", "e_sw"):
        err = np.abs(ge[k] - ref[k])
        bad = err > tol * np.abs(ref[k]) + 1e-9
        assert not bad.any(), f"{k}: gate {np.argmax(bad)} got {ge[k][np.argmax(bad)]} want {ref[k][np.argmax(bad)]}"


def _toggles(n, n_pins, rng, t0, t1, pins=None):
    """n valid events on random pins (or the given pin sequence) with sorted
    random times in [t0, t1), ties allowed."""
    t = np.sort(rng.integers(t0, t1, n))
    S, ev = 0, []
    for k in range(n):
        pin = int(rng.integers(0, n_pins)) if pins is None else int(pins[k])
        v = 1 - ((S >> pin) & 1)
        S ^= 1 << pin
        ev.append((int(t[k]), pin, v))
    return ev


@pytest.mark.parametrize("tile_min", [1, 64, 2048])
@pytest.mark.parametrize("bin_ps", [7, 10])
def test_many_slices_and_a_ragged_last_one(engine, tile_min, bin_ps):
    n_bins = 3 * SLICE + 849  # odd: the last slice's bins are not a multiple of 2
    lib, net, tr = small_random(n_gates=1500, n_events=400_000, window_ps=n_bins * bin_ps, seed=61, tie_p=0.05,
                                zipf_s=1.0)
    w, ge = run(engine, lib, net, tr, bin_ps, tile_min)
    check(w, ge, oracle.walk(lib, net, tr, bin_ps), bin_ps)


def test_slice_boundaries_bursts_late_gates_and_idle_pins(engine):
    """Hand-built gates on the 12-cell library (gate cells chosen to cover 1-3
    inputs): events exactly at slice starts and ties there; a burst inside one
    slice; a gate starting in the third slice; a NAND3 whose pin 2 toggles
    once early and then stays idle for 20k events."""
    lib = synth.make_library(1)
    bin_ps = 5
    n_bins = 4 * SLICE
    T = n_bins * bin_ps
    rng = np.random.default_rng(5)
    B = SLICE * bin_ps  # time of a slice boundary
    gates, cells = [], []
    # 1: events on every slice boundary, with ties (two pins at once) there
    ev = _toggles(3000, 3, rng, 0, T)
    extra = []
    for k in range(1, 4):
        extra += [(k * B, 0), (k * B, 1), (k * B - 1, 2), (k * B + 1, 2)]
    pins_times = sorted([(t, p) for t, p, _ in ev] + extra)
    S, ev = 0, []
    for t, p in pins_times:
        v = 1 - ((S >> p) & 1)
        S ^= 1 << p
        ev.append((t, p, v))
    gates.append(ev)
    cells.append(11)  # MUX2: 3 inputs
    # 2: a burst inside slice 1
    gates.append(_toggles(5000, 2, rng, B + 100, B + 9000))
    cells.append(2)  # NAND2
    # 3: starts in slice 2
    gates.append(_toggles(4000, 3, rng, 2 * B + 17, T))
    cells.append(6)  # AND2
    # 4: NAND3 with pin 2 idle after its first toggle
    pins = rng.integers(0, 2, 20_000)
    pins[3] = 2
    pins[::9] = 3
    gates.append(_toggles(20_000, 4, rng, 0, T, pins=pins))
    cells.append(3)  # NAND3
    # 5: an inverter, and 6: a gate without events
    gates.append(_toggles(3000, 2, rng, 0, T))
    cells.append(0)
    gates.append([])
    cells.append(1)
    loads = [2.0, 1.5, 3.0, 0.7, 9.0, 1.0]
    net = netlist_from(lib, cells, loads, np.random.default_rng(2).uniform(10, 200, (6, lib.max_in, 2)))
    init = [0, 0, 0, 0, 0, 1]
    tr = trace_from(gates, init, T)
    ref = oracle.walk(lib, net, tr, bin_ps)
    for tile_min in (1, 3000, 0):
        w, ge = run(engine, lib, net, tr, bin_ps, tile_min)
        check(w, ge, ref, bin_ps)


def test_word_carries_and_terms_sent_to_l2(engine):
    """6,000 events of one gate at one timestamp (alternating pins: all legal
    toggles) put ~20,000 fJ in one bin, far past the 128 fJ a shared word holds
    before it carries; with escale 40 single internal energies exceed what
    is quantised in shared memory and go to L2 directly."""
    lib = synth.make_library(1)
    rng = np.random.default_rng(9)
    T = 2 * SLICE * 10
    burst = []
    S = 0
    for k in range(6000):
        p = k % 2
        v = 1 - ((S >> p) & 1)
        S ^= 1 << p
        burst.append((SLICE * 10 + 55, p, v))
    gates = [burst, _toggles(3000, 3, rng, 0, T), _toggles(2500, 4, rng, 0, T)]
    net = netlist_from(lib, [2, 7, 9], [2.0, 4.0, 8.0])
    tr = trace_from(gates, [0, 0, 0], T)
    ref = oracle.walk(lib, net, tr, 10)
    w, ge = run(engine, lib, net, tr, 10, tile_min=1)
    check(w, ge, ref, 10)
    es = np.full(lib.n_cells, 40.0, np.float32)
    ref = oracle.walk(lib, net, tr, 10, escale=es)
    w, ge = run(engine, lib, net, tr, 10, tile_min=1, escale=es)
    check(w, ge, ref, 10)


def test_signed_energies(engine):
    """Tables that go negative under extrapolation: shared words move both
    ways and carry downwards.  Bins are compared relative to the waveform's
    mean magnitude (single bins can cancel to near zero)."""
    lib = single_cell_library(2, lambda pin, edge, side: np.arange(49, dtype=np.float32).reshape(7, 7) - 30.0,
                              lambda s: 5.0 + s)
    rng = np.random.default_rng(4)
    T = 3 * SLICE * 3
    gates = [_toggles(4000, 3, rng, 0, T) for _ in range(6)]
    slews = np.full((6, 2, 2), 400.0, np.float32)  # past the last slew knot: extrapolated
    net = netlist_from(lib, [0] * 6, [0.1, 20.0, 3.0, 30.0, 0.2, 5.0], slews)
    tr = trace_from(gates, [0] * 6, T)
    ref = oracle.walk(lib, net, tr, 3)
    w, ge = run(engine, lib, net, tr, 3, tile_min=1)
    check(w, ge, ref, 3, mean_scale=True)


@pytest.mark.parametrize("kind,code", [("order", -2), ("slice_order", -2), ("time", -3), ("pin", -3),
                                       ("toggle", -4)])
def test_malformed_tiled_gate_reports_first_bad_record(engine, kind, code):
    """A tiled gate (3,000 events over three slices) with one bad record deep
    in a later slice, and a later bad record in another gate: the error is the
    first bad record, with the oracle's code."""
    from paper_2609_05960_gb300 import GtpError
    lib = single_cell_library(2, lambda *a: 1.0, lambda s: 1.0 + s)
    net = netlist_from(lib, [0, 0, 0], [1.0, 1.0, 1.0])
    T = 3 * SLICE * 10
    rng = np.random.default_rng(7)
    g0 = _toggles(40, 3, rng, 0, T)
    g1 = _toggles(3000, 3, rng, 0, T)
    g2 = _toggles(2500, 3, rng, 0, T)
    pos = 2100
    t, pin, v = g1[pos]
    if kind == "order":
        g1[pos] = (g1[pos - 1][0] - 1, pin, v)
    elif kind == "slice_order":  # a time far back, in an earlier slice
        g1[pos] = (100, pin, v)
    elif kind == "time":
        g1[pos] = (T + 5, pin, v)
    elif kind == "pin":
        g1[pos] = (t, 3, v)
    else:
        g1[pos] = (t, pin, 1 - v)
    g2[2000] = (g2[2000][0], 3, 0)  # a later error in another gate
    tr = trace_from([g0, g1, g2], [0, 0, 0], T)
    with pytest.raises(oracle.OracleError) as eo:
        oracle.walk(lib, net, tr, 10)
    assert eo.value.code == code and eo.value.record == 40 + pos
    for tile_min in (1, 1000):
        with pytest.raises(GtpError) as ei:
            run(engine, lib, net, tr, 10, tile_min)
        assert ei.value.code == code
        assert f"at record {40 + pos}" in str(ei.value)


def test_tile_min_does_not_change_results(engine):
    """The same window with tiling off, at a high threshold and for every
    gate: each run within the bar of the oracle, and the runs agree with one
    another per gate exactly in counts and states."""
    lib, net, tr = small_random(n_gates=4000, n_events=600_000, window_ps=2 * SLICE * 10 + 30, seed=71,
                                tie_p=0.02, zipf_s=1.2)
    bin_ps = 10
    ref = oracle.walk(lib, net, tr, bin_ps)
    outs = []
    for tile_min in (0, 5000, 256, 1):
        w, ge = run(engine, lib, net, tr, bin_ps, tile_min)
        check(w, ge, ref, bin_ps)
        outs.append(ge)
    for ge in outs[1:]:
        np.testing.assert_array_equal(ge["final_state"], outs[0]["final_state"])
