"""Pins for the FP64 oracle: closed forms, a hand-worked example, library
interpolation and the state-indexed table layout.  CPU only."""
import numpy as np
import pytest
from scipy.interpolate import RegularGridInterpolator

import oracle
import synth
from cases import and2_worked, netlist_from, single_cell_library, trace_from

SA = np.array(synth.SLEW_AXIS_PS, np.float32)
LA = np.array(synth.LOAD_AXIS_FF, np.float32)


# ----------------------------------------------------------------- interpolation (NLDM, Sec. 2.2)
def test_bilinear_returns_table_at_knots():
    rng = np.random.default_rng(0)
    tab = rng.uniform(0.5, 5, (7, 7)).astype(np.float32)
    for i in range(7):
        for j in range(7):
            assert oracle.bilinear(SA, LA, tab, SA[i], LA[j]) == float(tab[i, j])


def test_bilinear_reproduces_affine_tables_everywhere():
    # a + b*s + c*l is exactly representable at every knot; bilinear
    # interpolation and linear extrapolation must reproduce it everywhere.
    a, b, c = 1.0, 0.25, 0.5
    tab = (a + b * SA[:, None].astype(np.float64) + c * LA[None, :]).astype(np.float32)
    assert np.all(tab == a + b * SA[:, None] + c * LA[None, :])
    rng = np.random.default_rng(1)
    for s, l in zip(rng.uniform(0.0, 500.0, 200), rng.uniform(0.0, 30.0, 200)):
        assert oracle.bilinear(SA, LA, tab, s, l) == pytest.approx(a + b * s + c * l, rel=1e-13, abs=1e-12)
    # below and above both axes: linear extrapolation
    assert oracle.bilinear(SA, LA, tab, 1.0, 0.1) == pytest.approx(a + b * 1.0 + c * 0.1, rel=1e-13)
    assert oracle.bilinear(SA, LA, tab, 1000.0, 40.0) == pytest.approx(a + b * 1000 + c * 40, rel=1e-13)


def test_bilinear_midpoint_is_mean_of_corners():
    rng = np.random.default_rng(2)
    tab = rng.uniform(0.5, 5, (7, 7)).astype(np.float32)
    for i in range(6):
        for j in range(6):
            s = 0.5 * (float(SA[i]) + float(SA[i + 1]))
            l = 0.5 * (float(LA[j]) + float(LA[j + 1]))
            mean = 0.25 * (float(tab[i, j]) + float(tab[i, j + 1]) + float(tab[i + 1, j]) + float(tab[i + 1, j + 1]))
            assert oracle.bilinear(SA, LA, tab, s, l) == pytest.approx(mean, rel=1e-14)


def test_bilinear_matches_scipy_including_extrapolation():
    rng = np.random.default_rng(3)
    tab = rng.uniform(0.5, 5, (7, 7)).astype(np.float32)
    ref = RegularGridInterpolator((SA.astype(np.float64), LA.astype(np.float64)), tab.astype(np.float64),
                                  method="linear", bounds_error=False, fill_value=None)
    pts = np.stack([rng.uniform(0.0, 400.0, 500), rng.uniform(0.0, 20.0, 500)], 1)
    want = ref(pts)
    got = np.array([oracle.bilinear(SA, LA, tab, s, l) for s, l in pts])
    np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-12)


def test_bilinear_load_derivative():
    rng = np.random.default_rng(4)
    tab = rng.uniform(0.5, 5, (7, 7)).astype(np.float32)
    for s, j, u in zip(rng.uniform(6, 300, 50), rng.integers(0, 6, 50), rng.uniform(0.1, 0.9, 50)):
        # a point inside load segment j, and a step that stays inside it
        w = float(LA[j + 1]) - float(LA[j])
        l = float(LA[j]) + u * w
        h = 1e-3 * w
        fd = (oracle.bilinear(SA, LA, tab, s, l + h) - oracle.bilinear(SA, LA, tab, s, l - h)) / (2 * h)
        assert oracle.bilinear_dload(SA, LA, tab, s, l) == pytest.approx(fd, rel=1e-8)


# ----------------------------------------------------------------- hand-worked example
def test_and2_hand_worked_example():
    fx, lib, net, tr = and2_worked()
    out = oracle.walk(lib, net, tr, fx["bin_ps"])
    exp = fx["expected"]
    np.testing.assert_allclose(out["bins"], exp["bins_fj"], rtol=1e-12, atol=1e-15)
    assert out["e_int"][0] == pytest.approx(exp["e_int_fj"], rel=1e-14)
    assert out["e_sw"][0] == pytest.approx(exp["e_sw_fj"], rel=1e-14)
    assert out["e_leak"][0] == pytest.approx(exp["e_leak_fj"], rel=1e-12)
    assert out["n_events"][0] == exp["n_events"]
    assert out["final_state"][0] == exp["final_state"]


# ----------------------------------------------------------------- closed forms
def _inverter(n_toggles, Tr=2.0, Tf=2.0, C=2.0, slew=40.0, leak=0.0, period=100, window=None):
    lib = single_cell_library(1, lambda pin, edge, side: Tr if edge else Tf, lambda s: leak)
    net = netlist_from(lib, [0], [C], np.full((1, 1, 2), slew, np.float32))
    ev = []
    S = 0  # input 0, output 0
    for k in range(n_toggles):
        t = k * period + 10
        vin = 1 - (S & 1)
        ev.append((t, 0, vin))
        S ^= 1
        vout = 1 - ((S >> 1) & 1)
        ev.append((t + 30, 1, vout))
        S ^= 2
    window = window or n_toggles * period + 100
    return lib, net, trace_from([ev], [0], window)


@pytest.mark.parametrize("n", [1, 2, 7, 40])
def test_inverter_n_toggles_closed_form(n):
    """n toggles of one inverter = n * (E_int + 0.5*C*Vdd^2), leakage off;
    C and slew on table knots (both edges share the table value)."""
    lib, net, tr = _inverter(n, Tr=2.5, Tf=2.5, C=2.0, slew=40.0)
    out = oracle.walk(lib, net, tr, 10)
    vdd = lib.vdd
    assert out["e_int"][0] + out["e_sw"][0] == pytest.approx(n * (2.5 + 0.5 * 2.0 * vdd * vdd), rel=1e-14)
    assert out["bins"].sum() == pytest.approx(n * (2.5 + 0.5 * 2.0 * vdd * vdd), rel=1e-13)
    assert out["e_leak"][0] == 0.0
    # rise and fall edges read different tables
    lib2, net2, tr2 = _inverter(n, Tr=3.0, Tf=1.0)
    out2 = oracle.walk(lib2, net2, tr2, 10)
    n_rise = (n + 1) // 2
    assert out2["e_int"][0] == pytest.approx(3.0 * n_rise + 1.0 * (n - n_rise), rel=1e-14)


def test_constant_state_leakage_closed_form():
    """No events: each bin holds P*bin_ps*1e-6 fJ and the total is P*T*1e-6."""
    P = 17.25
    lib = single_cell_library(2, lambda *a: 1.0, lambda s: P if s == 5 else 3.0)
    net = netlist_from(lib, [0, 0], [2.0, 3.0])
    tr = trace_from([[], []], [5, 5], 10_000)
    out = oracle.walk(lib, net, tr, 250)
    np.testing.assert_allclose(out["bins"], 2 * P * 250 * 1e-6, rtol=1e-14)
    np.testing.assert_allclose(out["e_leak"], P * 10_000 * 1e-6, rtol=1e-14)
    assert out["e_int"].sum() == 0 and out["e_sw"].sum() == 0


def test_single_event_leakage_split_by_hand():
    """One output event at t = 1234 in 100 ps bins: before it P0, after P1."""
    P0, P1 = 7.0, 31.0
    lib = single_cell_library(1, lambda *a: 0.0, lambda s: {0: P0, 2: P1}.get(s, 99.0), vdd=1.0)
    net = netlist_from(lib, [0], [2.0])
    tr = trace_from([[(1234, 1, 1)]], [0], 3000)
    out = oracle.walk(lib, net, tr, 100)
    want = np.zeros(30)
    want[:12] = P0 * 100e-6
    want[12] = P0 * 34e-6 + P1 * 66e-6 + 0.5 * 2.0 * 1.0
    want[13:] = P1 * 100e-6
    np.testing.assert_allclose(out["bins"], want, rtol=1e-13)


def test_event_on_bin_boundary_goes_to_later_bin():
    lib = single_cell_library(1, lambda *a: 0.0, lambda s: 0.0, vdd=1.0)
    net = netlist_from(lib, [0], [2.0])
    tr = trace_from([[(200, 1, 1)]], [0], 400)
    out = oracle.walk(lib, net, tr, 100)
    np.testing.assert_allclose(out["bins"], [0, 0, 1.0, 0], atol=0)


# ----------------------------------------------------------------- state-indexed layout (Sec. 4.1)
def test_state_indexed_table_layout():
    """Every table holds its own flat index as a constant; the energy of each
    event must be the index derived independently from (pin, edge, side)."""
    n_in = 3
    idx = iter(range(10_000))
    tables = {}
    for pin in range(n_in):
        for edge in range(2):
            for side in range(4):
                tables[(pin, edge, side)] = float(next(idx))
    lib = single_cell_library(n_in, lambda p, e, s: tables[(p, e, s)], lambda s: 0.0)
    net = netlist_from(lib, [0], [2.0])
    rng = np.random.default_rng(5)
    S = 0b0101
    ev, want = [], []
    for k in range(60):
        pin = int(rng.integers(0, n_in))
        v = 1 - ((S >> pin) & 1)
        others = [(S >> p) & 1 for p in range(n_in) if p != pin]
        side = others[0] | (others[1] << 1)
        want.append(pin * 8 + v * 4 + side)
        ev.append((10 * k + 5, pin, v))
        S ^= 1 << pin
    tr = trace_from([ev], [0b0101], 1000)
    out = oracle.walk(lib, net, tr, 10)
    np.testing.assert_array_equal(out["bins"][: len(want)], np.array(want, float))
    assert out["final_state"][0] == S


def test_leakage_indexed_by_full_state_including_output():
    lib = single_cell_library(2, lambda *a: 0.0, lambda s: float(s + 1) * 10.0)
    net = netlist_from(lib, [0], [1.0])
    tr = trace_from([[]], [0b110], 1000)
    out = oracle.walk(lib, net, tr, 1000)
    assert out["e_leak"][0] == pytest.approx(70.0 * 1000 * 1e-6, rel=1e-14)


# ----------------------------------------------------------------- validation
@pytest.mark.parametrize("events,code", [
    ([(100, 0, 1), (50, 1, 1)], oracle.EORDER),
    ([(100, 0, 1), (1000, 1, 1)], oracle.ERANGE),
    ([(-1, 0, 1)], oracle.ERANGE),
    ([(100, 3, 1)], oracle.ERANGE),
    ([(100, 0, 0)], oracle.ENOTOGGLE),
    ([(100, 0, 1), (100, 0, 1)], oracle.ENOTOGGLE),
])
def test_malformed_traces_are_rejected(events, code):
    lib = single_cell_library(2, lambda *a: 1.0, lambda s: 1.0)
    net = netlist_from(lib, [0], [1.0])
    tr = trace_from([events], [0], 1000)
    with pytest.raises(oracle.OracleError) as ei:
        oracle.walk(lib, net, tr, 100)
    assert ei.value.code == code


def test_reserved_meta_bits_rejected():
    lib = single_cell_library(1, lambda *a: 1.0, lambda s: 1.0)
    net = netlist_from(lib, [0], [1.0])
    tr = trace_from([[(100, 0, 1)]], [0], 1000)
    tr.records[0, 1] |= 1 << 7
    with pytest.raises(oracle.OracleError) as ei:
        oracle.walk(lib, net, tr, 100)
    assert ei.value.code == oracle.ERANGE


def test_same_pin_twice_in_one_group_counts_both():
    """Two events of one pin at one timestamp: both count, both use the
    pre-group side bits, the state ends at the last one."""
    lib = single_cell_library(2, lambda p, e, s: 1.0 + p + 2 * e + 4 * s, lambda s: 0.0)
    net = netlist_from(lib, [0], [1.0])
    tr = trace_from([[(300, 0, 1), (300, 1, 1), (300, 0, 0)]], [0], 1000)
    out = oracle.walk(lib, net, tr, 100)
    # pre-group state 0: A rise side 0 -> 3; B rise side 0 -> 4; A fall side 0 -> 1
    assert out["e_int"][0] == pytest.approx(8.0)
    assert out["final_state"][0] == 0b010
    assert out["n_events"][0] == 3
