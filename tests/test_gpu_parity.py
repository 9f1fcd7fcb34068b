"""GPU engine vs the FP64 oracle, element by element, through the C ABI.

Bar (spec accuracy): per-gate event counts and final states bit-exact;
every waveform bin within 1e-5 relative of the oracle; per-gate energies
within 1e-5 relative (absolute floor 1e-9 fJ for exact zeros)."""
import numpy as np
import pytest

import oracle
import synth
from cases import and2_worked, netlist_from, single_cell_library, small_random, trace_from

pytestmark = pytest.mark.gpu

TOL = 1e-5

KERNELS = [
    dict(kernel=1),
    dict(kernel=0, records_per_thread=4, dense_min=16),
    dict(kernel=0, records_per_thread=8),
    dict(kernel=0, records_per_thread=16, dense_min=64),
    dict(kernel=0, records_per_thread=8, tile_min=1),    # every gate through the time-sliced walk
    dict(kernel=0, records_per_thread=4, dense_min=16, tile_min=40),
]
KID = ["per_gate", "seg_k4", "seg_k8", "seg_k16", "tiled_all", "tiled40"]


@pytest.fixture(scope="module")
def engine():
    from paper_2609_05960_gb300 import Engine
    e = Engine(0)
    yield e
    e.close()


def run(engine, lib, net, tr, bin_ps, params=None, escale=None, lscale=None, window=0):
    engine.load_library(lib)
    engine.load_netlist(net)
    for k in ("kernel", "records_per_thread", "dense_min", "ctas_per_sm", "tile_min", "piece_len", "group_bin_bytes"):
        engine.set_param(k, -1)
    for k, v in (params or {}).items():
        engine.set_param(k, v)
    if escale is not None or lscale is not None:
        engine.set_scales(escale, lscale)
    engine.load_events(window, tr)
    w = engine.run_power(window, bin_ps).cpu().numpy()
    ge = engine.gate_energy(window, device=False)
    return w, ge


def assert_matches(w, ge, ref, bin_ps, tol=TOL):
    want = oracle.waveform_w(ref["bins"], bin_ps)
    assert w.shape == want.shape
    rel = np.abs(w - want) / np.abs(want)
    assert rel.max() <= tol, f"bin {rel.argmax()}: got {w[rel.argmax()]}, want {want[rel.argmax()]}, rel {rel.max()}"
    np.testing.assert_array_equal(ge["n_events"], ref["n_events"])
    np.testing.assert_array_equal(ge["final_state"], ref["final_state"])
    for k in ("e_leak", "e_int", "e_sw"):
        err = np.abs(ge[k] - ref[k])
        bad = err > tol * np.abs(ref[k]) + 1e-9
        assert not bad.any(), f"{k}: gate {np.argmax(bad)} got {ge[k][np.argmax(bad)]} want {ref[k][np.argmax(bad)]}"


@pytest.mark.parametrize("params", KERNELS, ids=KID)
def test_hand_worked_example(engine, params):
    fx, lib, net, tr = and2_worked()
    w, ge = run(engine, lib, net, tr, fx["bin_ps"], params)
    np.testing.assert_allclose(w, np.array(fx["expected"]["bins_fj"]) * 1e-3 / fx["bin_ps"], rtol=TOL)
    assert ge["final_state"][0] == fx["expected"]["final_state"]
    assert ge["n_events"][0] == fx["expected"]["n_events"]


@pytest.mark.parametrize("params", KERNELS, ids=KID)
def test_tiny_workload_matches_oracle(engine, params):
    """2,000 gates, 200k events, Zipf 1.1, 1 us window, 100 ps bins."""
    lib, net, tr = synth.make_inputs(synth.CONFIGS["tiny"])
    w, ge = run(engine, lib, net, tr, 100, params)
    assert_matches(w, ge, oracle.walk(lib, net, tr, 100), 100)


@pytest.mark.parametrize("params", KERNELS, ids=KID)
@pytest.mark.parametrize("tie_p", [0.05, 0.5, 0.95])
def test_timestamp_ties(engine, params, tie_p):
    lib, net, tr = small_random(n_gates=60, n_events=40_000, window_ps=400_000, seed=71, tie_p=tie_p)
    w, ge = run(engine, lib, net, tr, 50, params)
    assert_matches(w, ge, oracle.walk(lib, net, tr, 50), 50)


@pytest.mark.parametrize("params", KERNELS, ids=KID)
def test_one_dense_gate_across_many_segments(engine, params):
    lib = synth.make_library(1)
    net = synth.make_netlist(lib, 3, seed=5)
    net.cell[:] = [3, 0, 11]  # NAND3, INV, MUX2
    net.n_pins[:] = (lib.n_in[net.cell] + 1).astype(np.uint8)
    tr = synth.make_trace(net, np.array([3, 70_001, 5]), 2_000_000, seed=9, tie_p=0.02)
    w, ge = run(engine, lib, net, tr, 1000, params)
    assert_matches(w, ge, oracle.walk(lib, net, tr, 1000), 1000)


@pytest.mark.parametrize("params", KERNELS, ids=KID)
@pytest.mark.parametrize("n_events", [0, 1, 255, 256, 257, 4097])
def test_ragged_sizes_and_empty_gates(engine, params, n_events):
    lib = synth.make_library(1)
    net = synth.make_netlist(lib, 50, seed=13)
    counts = np.zeros(50, np.int64)
    if n_events:
        counts[[3, 4, 17, 49]] = synth.zipf_counts(4, n_events, 1.0, None, 3)
    tr = synth.make_trace(net, counts, 100_000, seed=21)
    w, ge = run(engine, lib, net, tr, 100, params)
    assert_matches(w, ge, oracle.walk(lib, net, tr, 100), 100)


@pytest.mark.parametrize("params", KERNELS, ids=KID)
@pytest.mark.parametrize("bin_ps", [1, 7, 3000])
def test_bin_sizes_and_window_edges(engine, params, bin_ps):
    lib, net, tr = small_random(n_gates=40, n_events=5_000, window_ps=21_000, seed=31, tie_p=0.05)
    rec = tr.records
    for g in range(0, 40, 5):  # events at t = 0 and t = T - 1
        a, b = tr.offsets[g], tr.offsets[g + 1]
        if b - a >= 2:
            rec[a, 0] = 0
            rec[b - 1, 0] = tr.window_ps - 1
    w, ge = run(engine, lib, net, tr, bin_ps, params)
    assert_matches(w, ge, oracle.walk(lib, net, tr, bin_ps), bin_ps)


@pytest.mark.parametrize("params", KERNELS, ids=KID)
def test_scales_and_extrapolated_lookups(engine, params):
    # points outside both axes (linear extrapolation), kept where the tables
    # stay positive so that every bin is a sum of positive terms
    lib, net, tr = small_random(n_gates=200, n_events=30_000, window_ps=300_000, seed=41, tie_p=0.01)
    net.slew_ps[::3, :, 0] = 4.5
    net.slew_ps[1::3, :, 1] = 330.0
    net.load_ff[::4] = 0.24
    net.load_ff[1::4] = 16.5
    rng = np.random.default_rng(0)
    es = rng.uniform(0.3, 3.0, lib.n_cells).astype(np.float32)
    ls = rng.uniform(0.3, 3.0, lib.n_cells).astype(np.float32)
    w, ge = run(engine, lib, net, tr, 100, params, escale=es, lscale=ls)
    ref = oracle.walk(lib, net, tr, 100, escale=es.astype(np.float64), lscale=ls.astype(np.float64))
    assert_matches(w, ge, ref, 100)


@pytest.mark.parametrize("params", KERNELS, ids=KID)
def test_far_extrapolation_with_signed_energies(engine, params):
    """Far outside the axes the random tables extrapolate to negative
    energies, so bins are sums of signed terms; the bar is then relative to
    the waveform's mean magnitude."""
    lib, net, tr = small_random(n_gates=200, n_events=30_000, window_ps=300_000, seed=42, tie_p=0.01)
    net.slew_ps[::3, :, 0] = 1.0
    net.slew_ps[1::3, :, 1] = 700.0
    net.load_ff[::4] = 0.1
    net.load_ff[1::4] = 40.0
    w, ge = run(engine, lib, net, tr, 100, params)
    ref = oracle.walk(lib, net, tr, 100)
    want = oracle.waveform_w(ref["bins"], 100)
    assert np.abs(w - want).max() <= TOL * np.abs(want).mean()
    np.testing.assert_array_equal(ge["final_state"], ref["final_state"])
    for k in ("e_leak", "e_int", "e_sw"):
        assert np.abs(ge[k] - ref[k]).max() <= TOL * np.abs(ref[k]).mean()


@pytest.mark.parametrize("params", KERNELS[1:], ids=KID[1:])
def test_seed_fixup_for_idle_pin(engine, params):
    """Pin 2 of a NAND3 stays idle for most of a 30k-event gate, so the
    bounded backward seed scan cannot resolve it and the fix-up pass runs."""
    lib = synth.make_library(1)
    net = netlist_from(lib, [3, 0], [2.0, 1.0])
    S = 0b0101
    ev = []
    rng = np.random.default_rng(3)
    for k in range(30_000):
        pin = int(rng.integers(0, 2)) if k != 29_000 else 2
        if k % 7 == 0 and k != 29_000:
            pin = 3
        v = 1 - ((S >> pin) & 1)
        S ^= 1 << pin
        ev.append((k * 10 + (5 if k % 11 else 0), pin, v))
    ev2 = [(100, 0, 1), (200, 1, 0)]
    tr = trace_from([ev, ev2], [0b0101, 0b10], 400_000)
    w, ge = run(engine, lib, net, tr, 100, params)
    assert_matches(w, ge, oracle.walk(lib, net, tr, 100), 100)


@pytest.mark.parametrize("params", KERNELS, ids=KID)
@pytest.mark.parametrize("events,code", [
    ([(100, 0, 1), (50, 1, 1)], -2),
    ([(100, 0, 1), (5000, 1, 1)], -3),
    ([(100, 3, 1)], -3),
    ([(100, 0, 0)], -4),
    ([(100, 0, 1), (100, 0, 1)], -4),
])
def test_malformed_traces_are_rejected(engine, params, events, code):
    from paper_2609_05960_gb300 import GtpError
    lib = single_cell_library(2, lambda *a: 1.0, lambda s: 1.0)
    net = netlist_from(lib, [0, 0], [1.0, 1.0])
    tr = trace_from([[(10, 1, 1)], events], [0, 0], 1000)
    with pytest.raises(GtpError) as ei:
        run(engine, lib, net, tr, 100, params)
    assert ei.value.code == code
    with pytest.raises(oracle.OracleError) as eo:
        oracle.walk(lib, net, tr, 100)
    assert eo.value.code == code


def _toggling_events(n, n_pins, seed, t0=100, step=7):
    """n valid events (each toggles its pin) with increasing times."""
    rng = np.random.default_rng(seed)
    S, ev, t = 0, [], t0
    for _ in range(n):
        pin = int(rng.integers(0, n_pins))
        v = 1 - ((S >> pin) & 1)
        S ^= 1 << pin
        ev.append((t, pin, v))
        t += int(rng.integers(0, step))  # ties allowed
    return ev


@pytest.mark.parametrize("params", KERNELS, ids=KID)
@pytest.mark.parametrize("kind,code", [("order", -2), ("time", -3), ("pin", -3), ("toggle", -4)])
@pytest.mark.parametrize("pos", [0, 131, 2200])
def test_malformed_dense_gate_reports_first_bad_record(engine, params, kind, code, pos):
    """A 3000-event gate (big or medium, depending on the segment length)
    with one bad record, and a later bad record in another gate: the error is
    the first bad record, with the oracle's code, whichever kernel ran."""
    from paper_2609_05960_gb300 import GtpError
    lib = single_cell_library(2, lambda *a: 1.0, lambda s: 1.0 + s)
    net = netlist_from(lib, [0, 0, 0], [1.0, 1.0, 1.0])
    T = 40_000
    g0 = _toggling_events(40, 3, 1)
    g1 = _toggling_events(3000, 3, 2)
    g2 = _toggling_events(50, 3, 3)
    t, pin, v = g1[pos]
    if kind == "order":
        g1[pos] = (g1[pos - 1][0] - 1 if pos else -1, pin, v)
        if pos == 0:
            code = -3  # a negative time is out of range before it is out of order
    elif kind == "time":
        g1[pos] = (T + 5, pin, v)
    elif kind == "pin":
        g1[pos] = (t, 3, v)
    else:
        g1[pos] = (t, pin, 1 - v)
    g2[10] = (g2[10][0], 3, 0)  # a later pin error in another gate
    tr = trace_from([g0, g1, g2], [0, 0, 0], T)
    with pytest.raises(GtpError) as ei:
        run(engine, lib, net, tr, 100, params)
    assert ei.value.code == code
    assert f"at record {40 + pos}" in str(ei.value)
    with pytest.raises(oracle.OracleError) as eo:
        oracle.walk(lib, net, tr, 100)
    assert eo.value.code == code and eo.value.record == 40 + pos


def test_bad_bin_size_rejected(engine):
    from paper_2609_05960_gb300 import GtpError
    lib, net, tr = small_random(n_gates=5, n_events=100, window_ps=1000, seed=2)
    engine.load_library(lib)
    engine.load_netlist(net)
    engine.load_events(0, tr)
    with pytest.raises(GtpError) as ei:
        engine.run_power(0, 300)
    assert ei.value.code == -3


def test_gpu_generator_matches_host_generator():
    import torch
    cfg = synth.scaled(synth.CONFIGS["tiny"], 500, 150_000, tie_p=0.2)
    lib, net, tr = synth.make_inputs(cfg)
    counts = np.diff(tr.offsets)
    tr2, rec = synth.make_trace_gpu(net, counts, cfg.window_ps, cfg.seed_ev, cfg.tie_p, chunk=100)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(rec.cpu().numpy().view(np.uint32), tr.records)
    np.testing.assert_array_equal(tr2.init_state, tr.init_state)


@pytest.mark.parametrize("borrow", [False, True])
def test_device_resident_events(engine, borrow):
    import torch
    lib, net, tr = small_random(n_gates=100, n_events=20_001, window_ps=200_000, seed=51, tie_p=0.02)
    engine.load_library(lib)
    engine.load_netlist(net)
    for k in ("kernel", "records_per_thread", "dense_min", "ctas_per_sm", "tile_min", "piece_len", "group_bin_bytes"):
        engine.set_param(k, -1)
    dev = engine.device
    off = torch.from_numpy(tr.offsets).to(dev)
    rec = torch.from_numpy(tr.records.view(np.int32)).to(dev)
    init = torch.from_numpy(tr.init_state).to(dev)
    engine.load_events(3, window_ps=tr.window_ps, offsets=off, records=rec, init_state=init, borrow=borrow)
    w = engine.run_power(3, 100).cpu().numpy()
    ge = engine.gate_energy(3, device=True)
    ge = {k: v.cpu().numpy() for k, v in ge.items()}
    assert_matches(w, ge, oracle.walk(lib, net, tr, 100), 100)


def test_host_waveform_output_and_repeat_runs(engine):
    from paper_2609_05960_gb300 import gtpower
    lib, net, tr = small_random(n_gates=100, n_events=20_000, window_ps=200_000, seed=52)
    engine.load_library(lib)
    engine.load_netlist(net)
    engine.load_events(0, tr)
    host = np.zeros(2000)
    gtpower.gtp_run_power(engine.ctx, 0, 100, host)
    dev = engine.run_power(0, 100).cpu().numpy()
    ref = oracle.waveform_w(oracle.walk(lib, net, tr, 100)["bins"], 100)
    for w in (host, dev):
        assert (np.abs(w - ref) / ref).max() <= TOL


def test_bin_and_gate_totals_agree(engine):
    """Sum over bins of energy equals the sum over gates of their energies."""
    cfg = synth.scaled(synth.CONFIGS["large"], 20_000, 2_000_000)
    cfg = synth.dataclasses.replace(cfg, window_ps=1_000_000, bin_ps=10)
    lib, net, tr = synth.make_inputs(cfg)
    w, ge = run(engine, lib, net, tr, 10)
    e_bins = (w * 10 * 1e3).sum()
    e_gates = ge["e_leak"].sum() + ge["e_int"].sum() + ge["e_sw"].sum()
    assert e_bins == pytest.approx(e_gates, rel=1e-6)
    w2, _ = run(engine, lib, net, tr, 20)
    np.testing.assert_allclose(w.reshape(-1, 2).mean(1), w2, rtol=TOL)


@pytest.mark.parametrize("fault", ["decreasing", "first", "last"])
def test_device_offsets_checked_and_copied(engine, fault):
    """Device offsets and initial states are copied by the load's check pass:
    malformed offsets are rejected, and a later load of good device arrays
    (the caller's copies overwritten afterwards) walks as the oracle does."""
    import torch
    from paper_2609_05960_gb300 import GtpError, gtpower
    lib, net, tr = small_random(n_gates=300, n_events=30_001, window_ps=300_000, seed=53, tie_p=0.02)
    engine.load_library(lib)
    engine.load_netlist(net)
    for k in ("kernel", "records_per_thread", "dense_min", "ctas_per_sm", "tile_min", "piece_len", "group_bin_bytes"):
        engine.set_param(k, -1)
    dev = engine.device
    bad = tr.offsets.copy()
    if fault == "decreasing":
        bad[150] = bad[152] + 1
    elif fault == "first":
        bad[0] = 1
    else:
        bad[-1] -= 1
    rec = torch.from_numpy(tr.records.view(np.int32)).to(dev)
    with pytest.raises(GtpError) as ei:
        engine.load_events(2, window_ps=tr.window_ps, offsets=torch.from_numpy(bad).to(dev), records=rec,
                           init_state=torch.from_numpy(tr.init_state).to(dev), borrow=True)
    assert ei.value.code == gtpower.GTP_EINVAL
    off = torch.from_numpy(tr.offsets).to(dev)
    init = torch.from_numpy(tr.init_state).to(dev)
    engine.load_events(2, window_ps=tr.window_ps, offsets=off, records=rec, init_state=init, borrow=True)
    off.fill_(0)   # the window keeps its own copies of offsets and states
    init.fill_(0)
    w = engine.run_power(2, 100).cpu().numpy()
    ge = {k: v.cpu().numpy() for k, v in engine.gate_energy(2, device=True).items()}
    assert_matches(w, ge, oracle.walk(lib, net, tr, 100), 100)


def test_gate_energy_device_outputs_any_subset(engine):
    """Per-gate device outputs come from one pass that skips null outputs."""
    import torch
    from paper_2609_05960_gb300 import gtpower
    lib, net, tr = small_random(n_gates=500, n_events=40_000, window_ps=400_000, seed=54)
    engine.load_library(lib)
    engine.load_netlist(net)
    engine.load_events(0, tr)
    engine.run_power(0, 100)
    full = {k: v.cpu().numpy() for k, v in engine.gate_energy(0, device=True).items()}
    G = net.n_gates
    kw = dict(device=engine.device)
    sentinel = {"e_leak": torch.full((G,), -7.0, dtype=torch.float64, **kw),
                "e_int": torch.full((G,), -7.0, dtype=torch.float64, **kw),
                "e_sw": torch.full((G,), -7.0, dtype=torch.float64, **kw),
                "n_events": torch.full((G,), -7, dtype=torch.int64, **kw),
                "final_state": torch.full((G,), 77, dtype=torch.uint8, **kw)}
    names = list(sentinel)
    for keep in ([0], [3], [1, 4], [0, 2, 3], []):
        outs = {k: (sentinel[k].clone() if i in keep else None) for i, k in enumerate(names)}
        gtpower.gtp_gate_energy(engine.ctx, 0, outs["e_leak"], outs["e_int"], outs["e_sw"], outs["n_events"],
                                outs["final_state"])
        torch.cuda.synchronize()
        for i, k in enumerate(names):
            if i in keep:
                np.testing.assert_array_equal(outs[k].cpu().numpy(), full[k])
    np.testing.assert_array_equal(full["n_events"], np.diff(tr.offsets))


def test_timing_levels(engine):
    """Timing level 2 records only the walk's pair of events; 1 every phase."""
    from paper_2609_05960_gb300 import GtpError, gtpower
    lib, net, tr = small_random(n_gates=200, n_events=50_000, window_ps=500_000, seed=55)
    engine.load_library(lib)
    engine.load_netlist(net)
    engine.load_events(0, tr)
    for graph in (False, True):
        for level in (2, 1):
            engine.set_param("timing", level)
            assert engine.get_param("timing") == level
            engine.run_power(0, 100, graph=graph)
            w = engine.run_power(0, 100, graph=graph)
            assert engine.get_param("n_timed") == 2
            assert engine.get_param("t_walk_ns") > 0
            if level == 2:
                assert engine.get_param("t_plan_ns") == 0 and engine.get_param("t_merge_ns") == 0
            else:
                assert engine.get_param("t_merge_ns") > 0
            ref = oracle.waveform_w(oracle.walk(lib, net, tr, 100)["bins"], 100)
            assert (np.abs(w.cpu().numpy() - ref) / ref).max() <= TOL
    engine.set_param("timing", 0)
    with pytest.raises(GtpError) as ei:
        engine.set_param("timing", 3)
    assert ei.value.code == gtpower.GTP_ERANGE


@pytest.mark.parametrize("params", KERNELS, ids=KID)
def test_load_and_scale_changes_rebuild_lookups(engine, params):
    """gtp_set_load and gtp_set_scales between runs: the next run rebuilds the
    event descriptors and gate tables (one pass) and walks as the oracle does
    with the new loads and scales, in the forward walk and the adjoint."""
    import torch
    lib, net, tr = small_random(n_gates=400, n_events=60_000, window_ps=600_000, seed=56, tie_p=0.02)
    w, ge = run(engine, lib, net, tr, 100, params)
    assert_matches(w, ge, oracle.walk(lib, net, tr, 100), 100)
    rng = np.random.default_rng(5)
    load2 = (net.load_ff * rng.uniform(0.2, 6.0, net.n_gates)).astype(np.float32)  # off the axes too
    engine.set_load(torch.from_numpy(load2).to(engine.device))
    w = engine.run_power(0, 100).cpu().numpy()
    assert_matches(w, engine.gate_energy(0, device=False), oracle.walk(lib, net, tr, 100, load_ff=load2), 100)
    es = rng.uniform(0.5, 2.0, lib.n_cells).astype(np.float32)
    ls = rng.uniform(0.5, 2.0, lib.n_cells).astype(np.float32)
    engine.set_scales(es, ls)
    load3 = (net.load_ff * rng.uniform(0.5, 2.0, net.n_gates)).astype(np.float32)
    engine.set_load(load3)  # host array
    w = engine.run_power(0, 100).cpu().numpy()
    ref = oracle.walk(lib, net, tr, 100, escale=es, lscale=ls, load_ff=load3)
    assert_matches(w, engine.gate_energy(0, device=False), ref, 100)
    if params.get("kernel", 0) == 0 and not params.get("tile_min"):
        g = (rng.normal(size=tr.window_ps // 100) * 1e3).astype(np.float32)
        dC, de, dl = engine.run_power_backward(0, 100, torch.from_numpy(g).to(engine.device))
        rC, rde, rdl = oracle.adjoint(lib, net, tr, 100, g.astype(np.float64), escale=es.astype(np.float64),
                                      lscale=ls.astype(np.float64), load_ff=load3)
        for got, ref in ((dC, rC), (de, rde), (dl, rdl)):
            got = got.cpu().numpy()
            assert np.all(np.abs(got - ref) <= 1e-4 * np.abs(ref) + 1e-5 * np.abs(ref).max())
    engine.set_scales(None, None)


def test_dense_min_chosen_per_run(engine):
    """Unless set, dense_min follows the run: 256 for a small window and for
    the adjoint; a value set applies to both directions."""
    import torch
    lib, net, tr = small_random(n_gates=300, n_events=40_000, window_ps=400_000, seed=57)
    engine.load_library(lib)
    engine.load_netlist(net)
    engine.set_param("dense_min", -1)
    engine.load_events(0, tr)
    engine.run_power(0, 100)
    assert engine.get_param("dense_min") == 256
    engine.set_param("dense_min", 48)
    w = engine.run_power(0, 100).cpu().numpy()
    assert engine.get_param("dense_min") == 48
    assert_matches(w, engine.gate_energy(0, device=False), oracle.walk(lib, net, tr, 100), 100)
    engine.run_power_backward(0, 100, torch.ones(4000, dtype=torch.float32, device=engine.device))
    assert engine.get_param("dense_min") == 48
    engine.set_param("dense_min", -1)
    engine.run_power_backward(0, 100, torch.ones(4000, dtype=torch.float32, device=engine.device))
    assert engine.get_param("dense_min") == 256
