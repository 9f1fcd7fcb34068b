"""Glitch detection (Sec. 2.4.1) on the GPU against the FP64 oracle, through
the C ABI: every walk (one thread per gate, the density-split walk at three
segment lengths), the batched form, the adjoint, and the off switch.

Bar: as for the plain walk: counts and final states bit-exact, bins and
per-gate energies (including the glitch energy) within 1e-5 relative."""
import numpy as np
import pytest

import oracle
import synth
from cases import netlist_from, single_cell_library, small_random, trace_from

pytestmark = pytest.mark.gpu

TOL = 1e-5
KERNELS = [
    dict(kernel=1),
    dict(kernel=0, records_per_thread=4, dense_min=16),
    dict(kernel=0, records_per_thread=8),
    dict(kernel=0, records_per_thread=16, dense_min=64),
]
KID = ["per_gate", "seg_k4", "seg_k8", "seg_k16"]


@pytest.fixture(scope="module")
def engine():
    from paper_2609_05960_gb300 import Engine
    e = Engine(0)
    yield e
    e.close()


def _setup(engine, lib, net, params):
    engine.load_library(lib)
    engine.load_netlist(net)
    for k in ("kernel", "records_per_thread", "dense_min", "ctas_per_sm", "tile_min", "piece_len", "group_bin_bytes"):
        engine.set_param(k, -1)
    for k, v in (params or {}).items():
        engine.set_param(k, v)


def _close(got, want, name):
    err = np.abs(got - want)
    bad = err > TOL * np.abs(want) + 1e-9
    assert not bad.any(), f"{name}: gate {np.argmax(bad)} got {got[np.argmax(bad)]} want {want[np.argmax(bad)]}"


def _check(engine, w, ref, bin_ps, window=0):
    want = oracle.waveform_w(ref["bins"], bin_ps)
    rel = np.abs(w - want) / np.abs(want)
    assert rel.max() <= TOL, f"bin {rel.argmax()}: rel {rel.max()}"
    ge = engine.gate_energy(window, device=False)
    np.testing.assert_array_equal(ge["n_events"], ref["n_events"])
    np.testing.assert_array_equal(ge["final_state"], ref["final_state"])
    for k in ("e_leak", "e_int", "e_sw"):
        _close(ge[k], ref[k], k)
    _close(engine.gate_glitch(window, device=False), ref["e_gl"], "e_gl")


def _hot_case(seed):
    """Hot gates of thousands of events: many events per clock cycle, so the
    search for a pin's previous event crosses lanes, segments and chunks."""
    return small_random(n_gates=300, n_events=60_000, window_ps=300_000, seed=seed, tie_p=0.05, zipf_s=1.3)


@pytest.mark.parametrize("params", KERNELS, ids=KID)
@pytest.mark.parametrize("clock", [37, 400, 5000])
def test_glitch_walk_matches_oracle(engine, params, clock):
    lib, net, tr = _hot_case(71)
    out_slew = np.random.default_rng(71).uniform(5.0, 150.0, (net.n_gates, 2)).astype(np.float32)
    _setup(engine, lib, net, params)
    engine.set_glitch(clock, out_slew)
    engine.load_events(0, tr)
    w = engine.run_power(0, 50).cpu().numpy()
    ref = oracle.walk(lib, net, tr, 50, glitch=(clock, out_slew))
    assert ref["e_gl"].sum() > 0
    _check(engine, w, ref, 50)


def test_hand_worked_glitches_on_the_gpu(engine):
    """The oracle's hand-worked glitch trace (one inverter, clock 1000 ps)."""
    lib = single_cell_library(1, lambda *a: 2.0, lambda s: 10.0, vdd=0.8)
    net = netlist_from(lib, [0], [1.0], slews=[[[60.0, 40.0]]])
    out_slew = np.array([[30.0, 20.0]], np.float32)
    ev = [(100, 0, 1), (130, 0, 0), (200, 1, 1), (210, 1, 0), (999, 0, 1), (1000, 0, 0),
          (1100, 1, 1), (1100, 0, 1), (1500, 0, 0), (1500, 0, 1)]
    tr = trace_from([ev], [0], 2000)
    for params in KERNELS:
        _setup(engine, lib, net, params)
        engine.set_glitch(1000, out_slew)
        engine.load_events(0, tr)
        w = engine.run_power(0, 100).cpu().numpy()
        _check(engine, w, oracle.walk(lib, net, tr, 100, glitch=(1000, out_slew)), 100)


def test_glitch_off_is_the_plain_walk(engine):
    lib, net, tr = _hot_case(72)
    out_slew = np.full((net.n_gates, 2), 20.0, np.float32)
    _setup(engine, lib, net, None)
    engine.load_events(0, tr)
    plain = engine.run_power(0, 50).cpu().numpy()
    engine.set_glitch(700, out_slew)
    with_gl = engine.run_power(0, 50).cpu().numpy()
    assert np.abs(with_gl - plain).max() > 1e-3 * np.abs(plain).max()
    engine.set_glitch(0)
    again = engine.run_power(0, 50).cpu().numpy()
    # bins are FP32 reductions in arbitrary order: equal up to that rounding
    np.testing.assert_allclose(again, plain, rtol=2e-6)
    assert not engine.gate_glitch(0, device=False).any()


def test_glitch_batched_matches_single_runs(engine):
    import torch
    lib = synth.make_library(1)
    net = synth.make_netlist(lib, 400, seed=9)
    out_slew = np.random.default_rng(73).uniform(5.0, 150.0, (net.n_gates, 2)).astype(np.float32)
    _setup(engine, lib, net, None)
    engine.set_glitch(300, out_slew)
    trs = []
    for w in range(5):
        n_ev = [0, 5_000, 40_000, 12_000, 70_000][w]
        counts = synth.zipf_counts(net.n_gates, n_ev, 1.3, None, 80 + w) if n_ev else np.zeros(net.n_gates, np.int64)
        tr = synth.make_trace(net, counts, 2000 * (w + 1) * 20, 80 + w, tie_p=0.05)
        engine.load_events(w, tr)
        trs.append(tr)
    ids = [4, 1, 3, 0, 2]
    outs = [torch.empty(trs[w].window_ps // 20, dtype=torch.float64, device=engine.device) for w in ids]
    engine.run_power_batched(ids, 20, outs=outs, graph=True)
    for o, w in zip(outs, ids):
        ref = oracle.walk(lib, net, trs[w], 20, glitch=(300, out_slew))
        _check(engine, o.cpu().numpy(), ref, 20, window=w)


@pytest.mark.parametrize("rpt", [4, 8, 16])
def test_glitch_adjoint_matches_oracle_adjoint(engine, rpt):
    import torch
    lib, net, tr = small_random(n_gates=300, n_events=50_000, window_ps=300_000, seed=74, tie_p=0.05, zipf_s=1.3)
    out_slew = np.random.default_rng(74).uniform(5.0, 150.0, (net.n_gates, 2)).astype(np.float32)
    _setup(engine, lib, net, dict(records_per_thread=rpt, dense_min=64))
    engine.set_glitch(450, out_slew)
    engine.load_events(0, tr)
    bin_ps = 50
    g = np.random.default_rng(1).normal(size=tr.window_ps // bin_ps)
    dC, de, dl = engine.run_power_backward(0, bin_ps, torch.tensor(g, dtype=torch.float32, device=engine.device))
    rC, re, rl = oracle.adjoint(lib, net, tr, bin_ps, g.astype(np.float32).astype(np.float64),
                                glitch=(450, out_slew))
    for got, want in ((dC, rC), (de, re), (dl, rl)):
        got = got.cpu().numpy().astype(np.float64)
        scale = np.abs(want).max()
        bad = np.abs(got - want) > 1e-4 * np.abs(want) + 1e-5 * scale
        assert not bad.any(), f"{np.argmax(bad)}: got {got[np.argmax(bad)]} want {want[np.argmax(bad)]}"


@pytest.mark.parametrize("params", KERNELS, ids=KID)
def test_glitch_on_a_wide_cell(engine, params):
    """A 6-input cell (above the tabulated width: energies interpolated per
    event) with a dense gate and a sparse one."""
    rng = np.random.default_rng(75)
    lib = single_cell_library(6, lambda pin, edge, side: 1.0 + 0.1 * pin + 0.5 * edge + 0.01 * side,
                              lambda s: 1.0 + s % 7)
    gates = []
    for n in (3000, 40):
        S, ev, t = 0, [], 5
        for _ in range(n):
            pin = int(rng.integers(0, 7))
            v = 1 - ((S >> pin) & 1)
            S ^= 1 << pin
            ev.append((t, pin, v))
            t += int(rng.integers(0, 9))
        gates.append(ev)
    slews = rng.uniform(10.0, 120.0, (2, 6, 2)).astype(np.float32)
    net = netlist_from(lib, [0, 0], [1.5, 3.0], slews=slews)
    tr = trace_from(gates, [0, 0], 40_000)
    out_slew = np.array([[25.0, 35.0], [50.0, 10.0]], np.float32)
    _setup(engine, lib, net, params)
    engine.set_glitch(120, out_slew)
    engine.load_events(0, tr)
    w = engine.run_power(0, 40).cpu().numpy()
    ref = oracle.walk(lib, net, tr, 40, glitch=(120, out_slew))
    assert ref["e_gl"][0] > 0
    _check(engine, w, ref, 40)


@pytest.mark.parametrize("host_wave", [False, True])
def test_design_power_matches_oracle(engine, host_wave):
    lib, net, tr = _hot_case(76)
    out_slew = np.random.default_rng(76).uniform(5.0, 150.0, (net.n_gates, 2)).astype(np.float32)
    _setup(engine, lib, net, None)
    engine.set_glitch(600, out_slew)
    engine.load_events(0, tr)
    w = engine.run_power(0, 50)
    got = engine.design_power(0, w.cpu().numpy() if host_wave else w)
    ref_r = oracle.walk(lib, net, tr, 50, glitch=(600, out_slew))
    ref = oracle.design_power(ref_r, tr.window_ps, 50)
    for k in ("p_leak", "p_int", "p_sw", "p_gl", "p_total"):
        assert got[k] == pytest.approx(ref[k], rel=1e-6), k
    want_w = oracle.waveform_w(ref_r["bins"], 50)
    assert got["p_peak"] == pytest.approx(ref["p_peak"], rel=TOL)
    assert want_w[got["peak_bin"]] == pytest.approx(ref["p_peak"], rel=2 * TOL)
    none = engine.design_power(0)
    assert none["peak_bin"] == -1 and none["p_total"] == pytest.approx(ref["p_total"], rel=1e-6)
    engine.set_glitch(0)
