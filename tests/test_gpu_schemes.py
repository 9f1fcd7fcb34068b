"""The paper's own GPU schemes (Naive-D + Naive-L with state-pattern
traversal, with state-indexed lookup, with event-density-aware partitioning,
and the fused kernel of Algorithm 1) against the FP64 oracle, through the
C ABI.  They compute the same definition as the engine's walk.

Bar: counts and final states bit-exact, bins and per-gate energies within
1e-5 relative."""
import numpy as np
import pytest

import oracle
import synth
from cases import netlist_from, single_cell_library, small_random, trace_from

pytestmark = pytest.mark.gpu

TOL = 1e-5
SCHEMES = ["naive", "sipl", "density", "fused"]


@pytest.fixture(scope="module")
def engine():
    from paper_2609_05960_gb300 import Engine
    e = Engine(0)
    yield e
    e.close()


def _setup(engine, lib, net, params=None):
    engine.load_library(lib)
    engine.load_netlist(net)
    for k in ("scheme_evt_tgt", "scheme_thr_floor", "scheme_ncyc_fix"):
        engine.set_param(k, -1)
    for k, v in (params or {}).items():
        engine.set_param(k, v)


def _close(got, want, name):
    bad = np.abs(got - want) > TOL * np.abs(want) + 1e-9
    assert not bad.any(), f"{name}: {np.argmax(bad)} got {got[np.argmax(bad)]} want {want[np.argmax(bad)]}"


def _check(engine, w, ref, bin_ps, window=0, glitch=False):
    want = oracle.waveform_w(ref["bins"], bin_ps)
    rel = np.abs(w - want) / np.abs(want)
    assert rel.max() <= TOL, f"bin {rel.argmax()}: rel {rel.max()}"
    ge = engine.gate_energy(window, device=False)
    np.testing.assert_array_equal(ge["n_events"], ref["n_events"])
    np.testing.assert_array_equal(ge["final_state"], ref["final_state"])
    for k in ("e_leak", "e_int", "e_sw"):
        _close(ge[k], ref[k], k)
    if glitch:
        _close(engine.gate_glitch(window, device=False), ref["e_gl"], "e_gl")


@pytest.mark.parametrize("scheme", SCHEMES)
@pytest.mark.parametrize("clock", [0, 400])
def test_scheme_matches_oracle(engine, scheme, clock):
    lib, net, tr = small_random(n_gates=300, n_events=60_000, window_ps=300_000, seed=61, tie_p=0.05, zipf_s=1.3)
    out_slew = np.random.default_rng(61).uniform(5.0, 150.0, (net.n_gates, 2)).astype(np.float32)
    _setup(engine, lib, net)
    engine.set_glitch(clock, out_slew if clock else None)
    engine.load_events(0, tr)
    w, ms = engine.run_power_scheme(0, 50, scheme)
    assert ms > 0
    ref = oracle.walk(lib, net, tr, 50, glitch=(clock, out_slew) if clock else None)
    _check(engine, w.cpu().numpy(), ref, 50, glitch=clock > 0)
    engine.set_glitch(0)


@pytest.mark.parametrize("scheme", SCHEMES)
def test_scheme_tiny_workload_equals_the_walk(engine, scheme):
    """The tiny workload: the scheme against the oracle and against the
    engine's own walk, run after it on the same window (host output)."""
    lib, net, tr = synth.make_inputs(synth.CONFIGS["tiny"])
    _setup(engine, lib, net)
    engine.load_events(1, tr)
    walk = engine.run_power(1, 100).cpu().numpy()
    host = np.empty(tr.window_ps // 100)
    engine.run_power_scheme(1, 100, scheme, out=host)
    _check(engine, host, oracle.walk(lib, net, tr, 100), 100, window=1)
    np.testing.assert_allclose(host, walk, rtol=2e-6)


@pytest.mark.parametrize("params", [dict(scheme_ncyc_fix=7), dict(scheme_evt_tgt=2, scheme_thr_floor=64),
                                    dict(scheme_evt_tgt=64, scheme_thr_floor=4)], ids=["ncyc7", "tgt2", "tgt64"])
def test_partitioning_parameters_do_not_change_results(engine, params):
    lib, net, tr = small_random(n_gates=200, n_events=40_000, window_ps=100_000, seed=62, tie_p=0.05, zipf_s=1.2)
    _setup(engine, lib, net, params)
    engine.load_events(0, tr)
    ref = oracle.walk(lib, net, tr, 20)
    for scheme in SCHEMES:
        w, _ = engine.run_power_scheme(0, 20, scheme)
        _check(engine, w.cpu().numpy(), ref, 20)


def test_hand_worked_glitches_by_every_scheme(engine):
    lib = single_cell_library(1, lambda *a: 2.0, lambda s: 10.0, vdd=0.8)
    net = netlist_from(lib, [0], [1.0], slews=[[[60.0, 40.0]]])
    out_slew = np.array([[30.0, 20.0]], np.float32)
    ev = [(100, 0, 1), (130, 0, 0), (200, 1, 1), (210, 1, 0), (999, 0, 1), (1000, 0, 0),
          (1100, 1, 1), (1100, 0, 1), (1500, 0, 0), (1500, 0, 1)]
    tr = trace_from([ev], [0], 2000)
    _setup(engine, lib, net)
    engine.set_glitch(1000, out_slew)
    engine.load_events(0, tr)
    ref = oracle.walk(lib, net, tr, 100, glitch=(1000, out_slew))
    for scheme in SCHEMES:
        w, _ = engine.run_power_scheme(0, 100, scheme)
        _check(engine, w.cpu().numpy(), ref, 100, glitch=True)
    engine.set_glitch(0)


@pytest.mark.parametrize("scheme", SCHEMES)
def test_scheme_on_a_wide_cell(engine, scheme):
    """A 6-input cell: 32 side patterns per (pin, edge) and 128 leakage
    patterns for the traversal."""
    rng = np.random.default_rng(63)
    lib = single_cell_library(6, lambda pin, edge, side: 1.0 + 0.1 * pin + 0.5 * edge + 0.01 * side,
                              lambda s: 1.0 + s % 7)
    gates, init = [], [0, 5, 77]
    for n, s0 in zip((3000, 40, 0), init):
        S, ev, t = s0, [], 5
        for _ in range(n):
            pin = int(rng.integers(0, 7))
            v = 1 - ((S >> pin) & 1)
            S ^= 1 << pin
            ev.append((t, pin, v))
            t += int(rng.integers(0, 9))
        gates.append(ev)
    net = netlist_from(lib, [0, 0, 0], [1.5, 3.0, 0.7], slews=rng.uniform(10.0, 120.0, (3, 6, 2)).astype(np.float32))
    tr = trace_from(gates, init, 40_000)
    _setup(engine, lib, net)
    engine.load_events(0, tr)
    w, _ = engine.run_power_scheme(0, 40, scheme)
    _check(engine, w.cpu().numpy(), oracle.walk(lib, net, tr, 40), 40)


def test_scheme_reports_the_first_bad_record(engine):
    from paper_2609_05960_gb300 import GtpError
    lib = single_cell_library(2, lambda *a: 1.0, lambda s: 1.0 + s)
    rng = np.random.default_rng(64)
    gates = []
    for g in range(30):
        S, ev, t = 0, [], 10
        for _ in range(int(rng.integers(20, 200))):
            pin = int(rng.integers(0, 3))
            v = 1 - ((S >> pin) & 1)
            S ^= 1 << pin
            ev.append((t, pin, v))
            t += int(rng.integers(1, 20))
        gates.append(ev)
    t_bad, p_bad, v_bad = gates[21][7]
    gates[21][7] = (t_bad, p_bad, 1 - v_bad)  # does not toggle
    gates[25][3] = (gates[25][3][0], 3, 0)    # a later pin error
    net = netlist_from(lib, [0] * 30, [1.0] * 30)
    tr = trace_from(gates, [0] * 30, 200_000)
    _setup(engine, lib, net)
    engine.load_events(0, tr)
    with pytest.raises(GtpError) as ei:
        engine.run_power_scheme(0, 100, "fused")
    want = int(tr.offsets[21]) + 7
    assert ei.value.code == -4 and f"at record {want}" in str(ei.value)
    with pytest.raises(oracle.OracleError) as eo:
        oracle.walk(lib, net, tr, 100)
    assert eo.value.code == -4 and eo.value.record == want


def test_scheme_empty_window_and_rejections(engine):
    from paper_2609_05960_gb300 import GtpError, gtpower
    lib, net, _ = small_random(n_gates=50, n_events=10, window_ps=10_000, seed=65)
    tr = trace_from([[] for _ in range(50)], np.random.default_rng(0).integers(0, 2, 50), 10_000)
    _setup(engine, lib, net)
    engine.load_events(0, tr)
    for scheme in SCHEMES:
        w, _ = engine.run_power_scheme(0, 100, scheme)
        _check(engine, w.cpu().numpy(), oracle.walk(lib, net, tr, 100), 100)
    with pytest.raises(GtpError):
        gtpower.gtp_run_power_scheme(engine.ctx, 0, 100, 7)
    with pytest.raises(GtpError):
        gtpower.gtp_run_power_scheme(engine.ctx, 0, 300, "fused")  # 10,000 ps is not a multiple of 300
