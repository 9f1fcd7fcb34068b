"""Pins for the oracle's per-component waveform (Sec. 2.2: the leakage,
internal, switching and glitch components of the power; Sec. 2.4.1 glitch
energy): a hand-worked trace, the per-picosecond simulator, and the
conservation identities that tie the components to the total waveform and to
the per-gate energies.  CPU only."""
import numpy as np
import pytest

import oracle
from oracle import brute
from cases import netlist_from, single_cell_library, small_random, trace_from

VDD = 0.8
HALF_V2 = 0.5 * np.float64(np.float32(VDD)) ** 2
LEAK, INT, SW, GL = range(4)


def test_hand_worked_components():
    """One inverter (pin 0 in, pin 1 out), constant 2 fJ tables, 10 nW
    leakage, C = 1 fF, clock 1000 ps, 100 ps bins.  Per bin:
      1:  in 100 regular (2 fJ int); in 130 glitch r = 0.36 (0.72 fJ gl)
      2:  out 200 regular (e_sw sw); out 210 glitch r = 0.16 (0.16 e_sw gl)
      9:  in 999 glitch r = 1 (2 fJ gl)
      10: in 1000 first of cycle 1 (2 fJ int)
      11: out 1100 regular (e_sw sw); in 1100 glitch r = 1 (2 fJ gl)
      15: in 1500 fall glitch r = 1 (2 fJ gl); in 1500 rise width 0 (0 gl)
    and 10 nW * 100 ps = 0.001 fJ of leakage in every bin."""
    lib = single_cell_library(1, lambda *a: 2.0, lambda s: 10.0, vdd=VDD)
    net = netlist_from(lib, [0], [1.0], slews=[[[60.0, 40.0]]])
    out_slew = np.array([[30.0, 20.0]], np.float32)
    ev = [(100, 0, 1), (130, 0, 0), (200, 1, 1), (210, 1, 0), (999, 0, 1), (1000, 0, 0),
          (1100, 1, 1), (1100, 0, 1), (1500, 0, 0), (1500, 0, 1)]
    tr = trace_from([ev], [0], 2000)
    c = oracle.walk(lib, net, tr, 100, glitch=(1000, out_slew), components=True)["comp_bins"]
    e_sw = HALF_V2 * 1.0
    want = np.zeros((4, 20))
    want[LEAK, :] = 10.0 * 100 * 1e-6
    want[INT, 1] = want[INT, 10] = 2.0
    want[GL, 1] = 0.72
    want[SW, 2] = want[SW, 11] = e_sw
    want[GL, 2] = 0.16 * e_sw
    want[GL, 9] = want[GL, 11] = want[GL, 15] = 2.0
    np.testing.assert_allclose(c, want, rtol=1e-12, atol=1e-15)


@pytest.mark.parametrize("seed,tie_p", [(41, 0.0), (42, 0.2)])
def test_components_match_the_per_picosecond_simulator(seed, tie_p):
    lib, net, tr = small_random(n_gates=6, n_events=300, window_ps=1500, seed=seed, tie_p=tie_p)
    rng = np.random.default_rng(seed)
    out_slew = rng.uniform(5.0, 80.0, (net.n_gates, 2)).astype(np.float32)
    es, ls = rng.uniform(0.5, 2.0, lib.n_cells), rng.uniform(0.5, 2.0, lib.n_cells)
    for glitch in (None, (37, out_slew), (400, out_slew)):
        got = oracle.walk(lib, net, tr, 50, escale=es, lscale=ls, glitch=glitch, components=True)
        want = brute.simulate(lib, net, tr, 50, escale=es, lscale=ls, glitch=glitch)
        np.testing.assert_allclose(got["comp_bins"], want["comp_bins"], rtol=1e-10, atol=1e-12)
        if glitch is None:
            assert not got["comp_bins"][GL].any()


def test_components_add_up_to_the_waveform_and_the_gate_energies():
    lib, net, tr = small_random(n_gates=80, n_events=20_000, window_ps=50_000, seed=43, tie_p=0.05, zipf_s=1.2)
    out_slew = np.random.default_rng(43).uniform(5.0, 150.0, (net.n_gates, 2)).astype(np.float32)
    r = oracle.walk(lib, net, tr, 100, glitch=(500, out_slew), components=True)
    c = r["comp_bins"]
    np.testing.assert_allclose(c.sum(0), r["bins"], rtol=1e-12)
    for k, e in ((LEAK, "e_leak"), (INT, "e_int"), (SW, "e_sw"), (GL, "e_gl")):
        assert c[k].sum() == pytest.approx(r[e].sum(), rel=1e-12), e
    assert (c >= 0).all() and c[GL].sum() > 0


def test_sampled_components_are_the_full_ones_at_the_samples():
    lib, net, tr = small_random(n_gates=40, n_events=5_000, window_ps=20_000, seed=44, tie_p=0.05)
    out_slew = np.full((net.n_gates, 2), 40.0, np.float32)
    full = oracle.walk(lib, net, tr, 100, glitch=(300, out_slew), components=True)["comp_bins"]
    sample = np.array([0, 3, 17, 99, 150, 199])
    part = oracle.walk(lib, net, tr, 100, glitch=(300, out_slew), components=True, sample_bins=sample)
    np.testing.assert_array_equal(part["comp_bins"], full[:, sample])
