"""Streamed runs (records copied from host memory in gate-range chunks while
earlier chunks are walked) against the FP64 oracle and against the resident
run, through the C ABI."""
import numpy as np
import pytest

import oracle
import synth
from cases import netlist_from, single_cell_library, small_random, trace_from

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def engine():
    from paper_2609_05960_gb300 import Engine
    e = Engine(0)
    yield e
    e.close()


def _setup(engine, lib, net, params=None):
    engine.load_library(lib)
    engine.load_netlist(net)
    for k in ("kernel", "records_per_thread", "dense_min", "ctas_per_sm", "tile_min", "piece_len", "group_bin_bytes"):
        engine.set_param(k, -1)
    for k, v in (params or {}).items():
        engine.set_param(k, v)


def _pinned(tr):
    import torch
    rec = torch.from_numpy(np.ascontiguousarray(tr.records).view(np.int32)).pin_memory()
    return rec


def _packed(tr):
    import torch
    from paper_2609_05960_gb300 import gtpower
    return torch.from_numpy(gtpower.gtp_pack_events(tr.records).view(np.int32)).pin_memory()


def _check(engine, w, ref, bin_ps, window):
    want = oracle.waveform_w(ref["bins"], bin_ps)
    rel = np.abs(w - want) / np.abs(want)
    assert rel.max() <= TOL, f"bin {rel.argmax()}: rel {rel.max()}"
    ge = engine.gate_energy(window, device=False)
    np.testing.assert_array_equal(ge["n_events"], ref["n_events"])
    np.testing.assert_array_equal(ge["final_state"], ref["final_state"])
    for k in ("e_leak", "e_int", "e_sw"):
        bad = np.abs(ge[k] - ref[k]) > TOL * np.abs(ref[k]) + 1e-9
        assert not bad.any(), f"{k}: gate {np.argmax(bad)}"


@pytest.mark.parametrize("params", [dict(kernel=1), dict(kernel=0, records_per_thread=8),
                                    dict(kernel=0, records_per_thread=4, dense_min=16)], ids=["per_gate", "k8", "k4"])
@pytest.mark.parametrize("n_chunks", [1, 3, 8, 64])
def test_streamed_matches_oracle(engine, params, n_chunks):
    lib, net, tr = synth.make_inputs(synth.CONFIGS["tiny"])
    _setup(engine, lib, net, params)
    w = engine.run_power_streamed(3, tr, 100, n_chunks=n_chunks, records=_pinned(tr), window_ps=tr.window_ps,
                                  offsets=tr.offsets, init_state=tr.init_state).cpu().numpy()
    _check(engine, w, oracle.walk(lib, net, tr, 100), 100, 3)


def test_streamed_hot_gates_with_glitches_and_a_host_waveform(engine):
    lib, net, tr = small_random(n_gates=300, n_events=60_000, window_ps=300_000, seed=91, tie_p=0.05, zipf_s=1.3)
    out_slew = np.random.default_rng(91).uniform(5.0, 150.0, (net.n_gates, 2)).astype(np.float32)
    _setup(engine, lib, net, dict(records_per_thread=4, dense_min=32))
    engine.set_glitch(400, out_slew)
    host = np.empty(tr.window_ps // 50)
    engine.run_power_streamed(0, tr, 50, out=host, n_chunks=5, records=_pinned(tr), window_ps=tr.window_ps,
                              offsets=tr.offsets, init_state=tr.init_state)
    ref = oracle.walk(lib, net, tr, 50, glitch=(400, out_slew))
    _check(engine, host, ref, 50, 0)
    gl = engine.gate_glitch(0, device=False)
    bad = np.abs(gl - ref["e_gl"]) > TOL * np.abs(ref["e_gl"]) + 1e-9
    assert not bad.any()
    engine.set_glitch(0)


def test_streamed_equals_resident_run_and_then_needs_a_reload(engine):
    from paper_2609_05960_gb300 import GtpError
    lib, net, tr = small_random(n_gates=500, n_events=80_000, window_ps=200_000, seed=92, tie_p=0.02)
    _setup(engine, lib, net)
    engine.load_events(1, tr)
    resident = engine.run_power(1, 40).cpu().numpy()
    streamed = engine.run_power_streamed(1, tr, 40, n_chunks=7, records=_pinned(tr), window_ps=tr.window_ps,
                                         offsets=tr.offsets, init_state=tr.init_state).cpu().numpy()
    np.testing.assert_allclose(streamed, resident, rtol=2e-6)
    with pytest.raises(GtpError):
        engine.run_power(1, 40)
    engine.load_events(1, tr)
    np.testing.assert_allclose(engine.run_power(1, 40).cpu().numpy(), resident, rtol=2e-6)


@pytest.mark.parametrize("params", [dict(kernel=1), dict(kernel=0, records_per_thread=8)], ids=["per_gate", "k8"])
@pytest.mark.parametrize("n_chunks", [1, 3, 8, 64])
def test_packed_streamed_matches_oracle(engine, params, n_chunks):
    """The packed transfer form (4.125 B a record) streamed and unpacked on
    the device gives the oracle's results."""
    lib, net, tr = synth.make_inputs(synth.CONFIGS["tiny"])
    _setup(engine, lib, net, params)
    w = engine.run_power_streamed(3, tr, 100, n_chunks=n_chunks, packed=_packed(tr), window_ps=tr.window_ps,
                                  offsets=tr.offsets, init_state=tr.init_state).cpu().numpy()
    _check(engine, w, oracle.walk(lib, net, tr, 100), 100, 3)


def test_packed_streamed_equals_the_unpacked_run(engine):
    lib, net, tr = small_random(n_gates=700, n_events=123_457, window_ps=400_000, seed=96, tie_p=0.03, zipf_s=1.3)
    _setup(engine, lib, net)
    kw = dict(window_ps=tr.window_ps, offsets=tr.offsets, init_state=tr.init_state)
    plain = engine.run_power_streamed(1, tr, 40, n_chunks=5, records=_pinned(tr), **kw).cpu().numpy()
    e_plain = engine.gate_energy(1, device=False)
    packed = engine.run_power_streamed(1, None, 40, n_chunks=5, packed=_packed(tr), **kw).cpu().numpy()
    np.testing.assert_allclose(packed, plain, rtol=2e-6)
    e_packed = engine.gate_energy(1, device=False)
    np.testing.assert_array_equal(e_packed["n_events"], e_plain["n_events"])
    np.testing.assert_array_equal(e_packed["final_state"], e_plain["final_state"])
    np.testing.assert_allclose(e_packed["e_int"], e_plain["e_int"], rtol=1e-6)


@pytest.mark.parametrize("on_device", [False, True], ids=["host", "device"])
def test_packed_load_equals_the_record_load(engine, on_device):
    import torch
    from paper_2609_05960_gb300 import gtpower
    lib, net, tr = small_random(n_gates=300, n_events=50_001, window_ps=300_000, seed=97, tie_p=0.05, zipf_s=1.3)
    _setup(engine, lib, net)
    engine.load_events(2, tr)
    want = engine.run_power(2, 50).cpu().numpy()
    pk = gtpower.gtp_pack_events(tr.records)
    off, init = tr.offsets, tr.init_state
    if on_device:
        dev = engine.device
        pk = torch.from_numpy(pk.view(np.int32)).to(dev)
        off, init = torch.from_numpy(off).to(dev), torch.from_numpy(init).to(dev)
    engine.load_events(2, window_ps=tr.window_ps, offsets=off, init_state=init, packed=pk)
    np.testing.assert_allclose(engine.run_power(2, 50).cpu().numpy(), want, rtol=2e-6)
    _check(engine, engine.run_power(2, 50).cpu().numpy(), oracle.walk(lib, net, tr, 50), 50, 2)


def test_streamed_empty_window(engine):
    lib, net, _ = small_random(n_gates=50, n_events=10, window_ps=10_000, seed=93)
    tr = trace_from([[] for _ in range(50)], np.random.default_rng(0).integers(0, 2, 50), 10_000)
    _setup(engine, lib, net)
    w = engine.run_power_streamed(0, tr, 100, n_chunks=4, records=np.zeros((0, 2), np.uint32),
                                  window_ps=tr.window_ps, offsets=tr.offsets, init_state=tr.init_state)
    _check(engine, w.cpu().numpy(), oracle.walk(lib, net, tr, 100), 100, 0)


@pytest.mark.parametrize("packed", [False, True], ids=["records", "packed"])
@pytest.mark.parametrize("chunks", [1, 4])
def test_streamed_reports_the_first_bad_record(engine, chunks, packed):
    from paper_2609_05960_gb300 import GtpError
    lib = single_cell_library(2, lambda *a: 1.0, lambda s: 1.0 + s)
    rng = np.random.default_rng(94)
    gates = []
    for g in range(40):
        S, ev, t = 0, [], 10
        for _ in range(int(rng.integers(50, 400))):
            pin = int(rng.integers(0, 3))
            v = 1 - ((S >> pin) & 1)
            S ^= 1 << pin
            ev.append((t, pin, v))
            t += int(rng.integers(1, 20))
        gates.append(ev)
    t_bad, p_bad, v_bad = gates[27][100]
    gates[27][100] = (t_bad, p_bad, 1 - v_bad)  # does not toggle
    gates[33][5] = (gates[33][5][0], 3, 0)      # a later pin error
    net = netlist_from(lib, [0] * 40, [1.0] * 40)
    tr = trace_from(gates, [0] * 40, 200_000)
    _setup(engine, lib, net, dict(dense_min=64))
    src = dict(packed=_packed(tr)) if packed else dict(records=_pinned(tr))
    with pytest.raises(GtpError) as ei:
        engine.run_power_streamed(0, None, 100, n_chunks=chunks, window_ps=tr.window_ps, offsets=tr.offsets,
                                  init_state=tr.init_state, **src)
    want = int(tr.offsets[27]) + 100
    assert ei.value.code == -4 and f"at record {want}" in str(ei.value)
    with pytest.raises(oracle.OracleError) as eo:
        oracle.walk(lib, net, tr, 100)
    assert eo.value.code == -4 and eo.value.record == want


def test_streamed_rejects_bad_offsets_before_copying(engine):
    from paper_2609_05960_gb300 import GtpError
    lib, net, tr = small_random(n_gates=20, n_events=500, window_ps=5_000, seed=95)
    _setup(engine, lib, net)
    off = tr.offsets.copy()
    off[7], off[8] = off[8], off[7] - 1
    with pytest.raises(GtpError) as ei:
        engine.run_power_streamed(0, tr, 100, n_chunks=3, records=tr.records, window_ps=tr.window_ps,
                                  offsets=off, init_state=tr.init_state)
    assert ei.value.code == -1
