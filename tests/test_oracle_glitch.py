"""Pins for the oracle's glitch detection and scaling (Sec. 2.4.1 clock-cycle
glitch detection; Eq. 2; Algorithm 1 GlitchDetectUpdate):
a hand-worked trace, closed forms, the per-picosecond counter simulator, the
conservation of energy when every ratio is one, and central differences of
the adjoint.  CPU only."""
import numpy as np
import pytest

import oracle
from oracle import brute
import synth
from cases import netlist_from, single_cell_library, small_random, trace_from

VDD = 0.8
HALF_V2 = 0.5 * np.float64(np.float32(VDD)) ** 2


def _inverter_case():
    """One 1-input cell (pin 0 in, pin 1 out), constant 2 fJ tables, 10 nW
    leakage, C = 1 fF; input slews fall 60 / rise 40 ps, output 30 / 20 ps."""
    lib = single_cell_library(1, lambda *a: 2.0, lambda s: 10.0, vdd=VDD)
    net = netlist_from(lib, [0], [1.0], slews=[[[60.0, 40.0]]])
    out_slew = np.array([[30.0, 20.0]], np.float32)
    ev = [(100, 0, 1), (130, 0, 0), (200, 1, 1), (210, 1, 0), (999, 0, 1), (1000, 0, 0),
          (1100, 1, 1), (1100, 0, 1), (1500, 0, 0), (1500, 0, 1)]
    tr = trace_from([ev], [0], 2000)
    return lib, net, tr, out_slew


def test_hand_worked_glitches():
    """Clock 1000 ps.  Per event: first event of a pin in a cycle is regular;
    later ones are glitches with r = min(1, (2 * width / (rise + fall))^2):
      130 in : width 30, r = (60/100)^2 = 0.36  -> 0.72 fJ
      210 out: width 10, r = (20/50)^2  = 0.16  -> 0.16 * 0.5*C*Vdd^2
      999 in : width 869, r = 1                 -> 2 fJ
      1000 in: new cycle, regular               -> internal 2 fJ
      1100 out: previous output event in cycle 0, regular
      1100 in: width 100, r = min(1, 4) = 1     -> 2 fJ
      1500 in (fall): width 400, r = 1          -> 2 fJ
      1500 in (rise, same timestamp): width 0, r = 0 -> 0."""
    lib, net, tr, out_slew = _inverter_case()
    r = oracle.walk(lib, net, tr, 100, glitch=(1000, out_slew))
    e_sw = HALF_V2 * 1.0
    assert r["e_int"][0] == pytest.approx(4.0, rel=1e-12)
    assert r["e_sw"][0] == pytest.approx(2 * e_sw, rel=1e-12)
    assert r["e_gl"][0] == pytest.approx(0.72 + 0.16 * e_sw + 2 + 2 + 2 + 0.0, rel=1e-12)
    assert r["final_state"][0] == 0b11  # input high (1500 rise), output high (1100 rise)
    leak_bin = 10.0 * 100 * 1e-6
    assert r["bins"][1] == pytest.approx(2.0 + 0.72 + leak_bin, rel=1e-12)
    assert r["bins"][2] == pytest.approx(e_sw + 0.16 * e_sw + leak_bin, rel=1e-12)
    assert r["bins"][9] == pytest.approx(2.0 + leak_bin, rel=1e-12)
    assert r["bins"][10] == pytest.approx(2.0 + leak_bin, rel=1e-12)
    assert r["bins"][11] == pytest.approx(e_sw + 2.0 + leak_bin, rel=1e-12)
    assert r["bins"][15] == pytest.approx(2.0 + leak_bin, rel=1e-12)


def test_without_a_clock_nothing_is_a_glitch():
    lib, net, tr, out_slew = _inverter_case()
    plain = oracle.walk(lib, net, tr, 100)
    off = oracle.walk(lib, net, tr, 100, glitch=(0, out_slew))
    assert plain["e_int"][0] == pytest.approx(14.0) and plain["e_sw"][0] == pytest.approx(3 * HALF_V2)
    for k in ("bins", "e_leak", "e_int", "e_sw"):
        np.testing.assert_array_equal(plain[k], off[k])
    assert off["e_gl"][0] == 0.0 and plain["e_gl"][0] == 0.0


def test_a_cycle_boundary_separates_events():
    """999 and 1000 ps lie in cycles 0 and 1 of a 1000 ps clock; 1000 and
    1999 share cycle 1."""
    lib = single_cell_library(1, lambda *a: 2.0, lambda s: 10.0, vdd=VDD)
    net = netlist_from(lib, [0], [1.0], slews=[[[60.0, 40.0]]])
    tr = trace_from([[(999, 0, 1), (1000, 0, 0), (1999, 0, 1)]], [0], 3000)
    r = oracle.walk(lib, net, tr, 100, glitch=(1000, np.zeros((1, 2), np.float32)))
    assert r["e_int"][0] == pytest.approx(4.0) and r["e_gl"][0] == pytest.approx(2.0)


@pytest.mark.parametrize("seed,tie_p", [(31, 0.0), (32, 0.1), (33, 0.4)])
def test_matches_the_per_cycle_counter_simulator(seed, tie_p):
    lib, net, tr = small_random(n_gates=6, n_events=300, window_ps=1500, seed=seed, tie_p=tie_p)
    rng = np.random.default_rng(seed)
    out_slew = rng.uniform(5.0, 80.0, (net.n_gates, 2)).astype(np.float32)
    es = rng.uniform(0.5, 2.0, lib.n_cells)
    for clock in (37, 250, 1500):
        got = oracle.walk(lib, net, tr, 50, escale=es, glitch=(clock, out_slew))
        want = brute.simulate(lib, net, tr, 50, escale=es, glitch=(clock, out_slew))
        np.testing.assert_allclose(got["bins"], want["bins"], rtol=1e-10, atol=1e-12)
        for k in ("e_leak", "e_int", "e_sw", "e_gl"):
            np.testing.assert_allclose(got[k], want[k], rtol=1e-10, atol=1e-12)


def test_full_ratio_moves_energy_without_losing_it():
    """With transition times near zero every glitch of width >= 1 ps has
    r = 1: glitch detection only moves energy from the internal and
    switching components to the glitch component; bins are unchanged."""
    lib, net, tr = small_random(n_gates=20, n_events=4000, window_ps=20_000, seed=34, tie_p=0.0)
    net.slew_ps[:] = 1e-3
    out_slew = np.full((net.n_gates, 2), 1e-3, np.float32)
    plain = oracle.walk(lib, net, tr, 100, load_ff=None)
    gl = oracle.walk(lib, net, tr, 100, glitch=(700, out_slew))
    assert gl["e_gl"].sum() > 0
    np.testing.assert_allclose(gl["e_int"] + gl["e_sw"] + gl["e_gl"], plain["e_int"] + plain["e_sw"], rtol=1e-12)
    np.testing.assert_allclose(gl["bins"], plain["bins"], rtol=1e-12)


def test_one_cycle_window_keeps_only_each_pins_first_event():
    """With the clock as long as the window, constant tables and a
    no-transition-time limit (r = 1), every event but each pin's first is a
    glitch: regular internal energy = 2 fJ per used input pin, regular
    switching energy = one output toggle."""
    lib = single_cell_library(2, lambda *a: 2.0, lambda s: 5.0, vdd=VDD)
    rng = np.random.default_rng(35)
    gates, used = [], []
    for g in range(8):
        S, ev, t = 0, [], 10
        for _ in range(int(rng.integers(1, 40))):
            pin = int(rng.integers(0, 3))
            v = 1 - ((S >> pin) & 1)
            S ^= 1 << pin
            ev.append((t, pin, v))
            t += int(rng.integers(1, 50))
        gates.append(ev)
        used.append({p for _, p, _ in ev})
    net = netlist_from(lib, [0] * 8, [1.5] * 8)
    tr = trace_from(gates, [0] * 8, 4000)
    r = oracle.walk(lib, net, tr, 100, glitch=(4000, np.zeros((8, 2), np.float32)))
    for g in range(8):
        assert r["e_int"][g] == pytest.approx(2.0 * len(used[g] - {2}))
        assert r["e_sw"][g] == pytest.approx(HALF_V2 * 1.5 * (2 in used[g]))


def test_adjoint_with_glitches_matches_central_differences():
    lib, net, tr = small_random(n_gates=15, n_events=2500, window_ps=20_000, seed=36, tie_p=0.05)
    rng = np.random.default_rng(36)
    out_slew = rng.uniform(20.0, 300.0, (net.n_gates, 2)).astype(np.float32)
    gl = (400, out_slew)
    bin_ps = 100
    la = np.array(synth.LOAD_AXIS_FF, np.float64)
    C = np.asarray(net.load_ff, np.float64).copy()
    for k in la:
        C[np.abs(C - k) < 0.01 * k] = k * 1.03
    w = rng.normal(size=tr.window_ps // bin_ps)
    dC, de, _ = oracle.adjoint(lib, net, tr, bin_ps, w, load_ff=C, glitch=gl)
    loss = lambda **kw: float(np.dot(w, oracle.waveform_w(oracle.walk(lib, net, tr, bin_ps, glitch=gl, **kw)["bins"],
                                                          bin_ps)))
    for g in range(net.n_gates):
        h = 1e-3 * C[g]
        Cp, Cm = C.copy(), C.copy()
        Cp[g] += h
        Cm[g] -= h
        assert dC[g] == pytest.approx((loss(load_ff=Cp) - loss(load_ff=Cm)) / (2 * h), rel=1e-6, abs=1e-12)
    # the energy scale enters linearly, so its derivative is exact by differences of unit steps
    for c in range(lib.n_cells):
        e1 = np.ones(lib.n_cells)
        e2 = e1.copy()
        e2[c] = 2.0
        assert de[c] == pytest.approx(loss(load_ff=C, escale=e2) - loss(load_ff=C, escale=e1), rel=1e-9, abs=1e-12)


def test_design_power_of_the_hand_worked_trace():
    """Averages over the 2000 ps window (fJ / ps = 1e-3 W) and the peak bin:
    bin 1 holds 2 + 0.72 fJ of dynamic energy plus 0.001 fJ of leakage."""
    lib, net, tr, out_slew = _inverter_case()
    r = oracle.walk(lib, net, tr, 100, glitch=(1000, out_slew))
    p = oracle.design_power(r, 2000, 100)
    e_sw = HALF_V2 * 1.0
    assert p["p_int"] == pytest.approx(4.0 * 1e-3 / 2000)
    assert p["p_sw"] == pytest.approx(2 * e_sw * 1e-3 / 2000)
    assert p["p_gl"] == pytest.approx((6.72 + 0.16 * e_sw) * 1e-3 / 2000)
    assert p["p_leak"] == pytest.approx(10.0 * 2000 * 1e-6 * 1e-3 / 2000)
    assert p["p_total"] == pytest.approx(p["p_leak"] + p["p_int"] + p["p_sw"] + p["p_gl"])
    assert p["peak_bin"] == 1 and p["p_peak"] == pytest.approx((2.72 + 0.001) * 1e-3 / 100)
