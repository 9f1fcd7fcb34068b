"""Pins of the oracle's range-mode leakage split and of its multi-core runner.

The range mode gives every bin an interval covers whole its share through a
difference array and one running sum (the split of Sec. 2.4.2 with the FP64
additions reordered).  It must equal the plain split bin by bin up to FP64
rounding, on cases that reach every branch: intervals inside one bin, across
two bins, across many, starting and ending on boundaries, ties, 1 ps bins,
bins wider than most intervals, glitch detection and component rows.  A
closed form pins it on its own too: a gate with no events leaks P * bin_ps
into every bin.  The runner (oracle/fullsize.py) must equal the serial walk
of the materialised trace."""
import numpy as np
import pytest

import oracle
import synth
from cases import netlist_from, single_cell_library, small_random, trace_from
from oracle import fullsize

RTOL = 1e-12


def _close(a, b):
    a, b = np.asarray(a), np.asarray(b)
    np.testing.assert_allclose(a, b, rtol=RTOL, atol=RTOL * max(1.0, float(np.abs(b).max(initial=0.0))))


@pytest.mark.parametrize("bin_ps", [1, 7, 50, 3000])
@pytest.mark.parametrize("seed", [3, 4])
def test_range_split_equals_plain_split(bin_ps, seed):
    window = bin_ps * (9000 // bin_ps) if bin_ps < 3000 else 30000
    lib, net, tr = small_random(n_gates=40, n_events=3000, window_ps=window, seed=seed, tie_p=0.1)
    es = np.linspace(0.5, 1.5, lib.n_cells)
    ls = np.linspace(1.3, 0.7, lib.n_cells)
    plain = oracle.walk(lib, net, tr, bin_ps, escale=es, lscale=ls)
    rng = oracle.walk(lib, net, tr, bin_ps, escale=es, lscale=ls, leak_range=True)
    _close(rng["bins"], plain["bins"])
    for k in ("e_leak", "e_int", "e_sw", "e_gl", "n_events", "final_state"):
        np.testing.assert_array_equal(rng[k], plain[k])


def test_range_split_with_glitches_components_and_gate_subsets():
    lib, net, tr = small_random(n_gates=60, n_events=5000, window_ps=20000, seed=9, tie_p=0.05)
    out_slew = np.random.default_rng(2).uniform(5, 300, (60, 2)).astype(np.float32)
    gates = np.array([3, 0, 59, 17, 17, 42])
    kw = dict(glitch=(700, out_slew), components=True, gates=gates)
    plain = oracle.walk(lib, net, tr, 16, **kw)
    rng = oracle.walk(lib, net, tr, 16, leak_range=True, **kw)
    _close(rng["bins"], plain["bins"])
    _close(rng["comp_bins"], plain["comp_bins"])
    np.testing.assert_array_equal(rng["e_gl"], plain["e_gl"])


def test_range_split_closed_forms():
    """No events: each bin holds P * bin_ps exactly.  One event at t = 35 in
    a 10-bin window of 10 ps bins: bins 0-2 hold P0 * 10, bin 3 holds
    P0 * 5 + P1 * 5 plus the event's energy, bins 4-9 hold P1 * 10."""
    lib = single_cell_library(1, lambda pin, edge, side: np.full((7, 7), 2.0), lambda s: [4.0, 6.0, 8.0, 10.0][s])
    net = netlist_from(lib, [0], [1.0])
    quiet = trace_from([[]], [1], 100)
    r = oracle.walk(lib, net, quiet, 10, leak_range=True)
    np.testing.assert_array_equal(r["bins"], np.full(10, 6.0 * 10 * 1e-6))
    one = trace_from([[(35, 0, 1)]], [0], 100)  # input 0 -> 1: state 0b00 -> 0b01
    r = oracle.walk(lib, net, one, 10, leak_range=True)
    want = np.array([4.0 * 10] * 3 + [4.0 * 5 + 6.0 * 5] + [6.0 * 10] * 6) * 1e-6
    want[3] += 2.0
    _close(r["bins"], want)


def test_fullsize_runner_equals_the_serial_walk():
    cfg = synth.scaled(synth.CONFIGS["tiny"], 3000, 300_000, tie_p=0.01)
    wl = fullsize.Workload.of(cfg)
    lib, net, tr = synth.make_inputs(cfg)
    es = np.linspace(0.8, 1.2, lib.n_cells)
    want = oracle.walk(lib, net, tr, cfg.bin_ps, escale=es)
    with fullsize.Pool(n_proc=3) as pool:
        got = pool.walk(wl, cfg.bin_ps, escale=es)
        got2 = pool.walk(wl, 2 * cfg.bin_ps, escale=es)
    _close(got["bins"], want["bins"])
    for k in ("e_leak", "e_int", "e_sw", "n_events", "final_state"):
        np.testing.assert_array_equal(got[k], want[k])
    _close(got2["bins"], want["bins"].reshape(-1, 2).sum(1))
    e = fullsize.bin_errors(oracle.waveform_w(want["bins"], cfg.bin_ps), got["bins"], cfg.bin_ps)
    assert e["max_rel_bin_err"] <= 1e-12 and e["bins"] == len(want["bins"])


def test_fullsize_runner_with_glitches():
    cfg = synth.scaled(synth.CONFIGS["tiny"], 500, 60_000)
    wl = fullsize.Workload.of(cfg, clock_ps=1000)
    lib, net, tr = synth.make_inputs(cfg)
    out_slew = np.random.default_rng(wl.out_slew_seed).uniform(10.0, 200.0, (cfg.n_gates, 2)).astype(np.float32)
    want = oracle.walk(lib, net, tr, cfg.bin_ps, glitch=(1000, out_slew), components=True)
    got = fullsize.walk(wl, cfg.bin_ps, n_proc=2, components=True)
    _close(got["bins"], want["bins"])
    _close(got["comp_bins"], want["comp_bins"])
    np.testing.assert_array_equal(got["e_gl"], want["e_gl"])
